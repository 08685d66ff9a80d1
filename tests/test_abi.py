"""The C-ABI library builds, loads and exports every function include/pitn.h
declares; argument checks that happen on the host before any device work
return their codes without a GPU."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pitn.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(pitn_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_01465_gb300 import build, pitn
    if not os.path.exists(pitn.LIB_PATH) or not build.up_to_date():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libpitn.so")
        build.build()
    return pitn.lib()


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("pitn_solve", "pitn_solve_ex", "pitn_solve_batch", "pitn_backward",
              "pitn_status_string", "pitn_release_workspace", "pitn_num_params", "pitn_launch_count"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_params(lib):
    from paper_2511_01465_gb300 import pitn as P
    assert P.pitn_num_params(P.PITN_LORENZ63) == 3
    assert P.pitn_num_params(P.PITN_VDP) == 1
    assert P.pitn_num_params(P.PITN_LINEAR_OSC) == 2
    assert P.pitn_num_params(P.PITN_FKPP) == 1
    assert P.pitn_num_params(P.PITN_LOGISTIC) == 2
    assert P.pitn_num_params(P.PITN_DAHLQUIST) == 1
    assert P.pitn_num_params(P.PITN_ROBERTSON) == 3
    assert P.pitn_num_params(99) == -1
    for code in (0, 1, 2, -1, -2, -3, -4, -5):
        assert P.pitn_status_string(code)


def test_argument_errors_are_detected_on_the_host(lib):
    from paper_2511_01465_gb300 import pitn as P
    p = np.array([10.0, 28.0, 8 / 3])
    x0 = np.ones(3)
    out = np.zeros((10, 3))
    E = P.PITN_EINVAL
    assert P.pitn_solve(P.PITN_LORENZ63, p, x0, 1e-3, 0, 3, 1e-10, 5, out) == E        # N = 0
    assert P.pitn_solve(P.PITN_LORENZ63, p, x0, 1e-3, 10, 2, 1e-10, 5, out) == E       # d mismatch
    assert P.pitn_solve(P.PITN_LORENZ63, p, x0, -1e-3, 10, 3, 1e-10, 5, out) == E      # h < 0
    assert P.pitn_solve(P.PITN_LORENZ63, p, x0, float("nan"), 10, 3, 1e-10, 5, out) == E
    assert P.pitn_solve(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, -1.0, 5, out) == E        # tol < 0
    assert P.pitn_solve(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, 1e-10, -1, out) == E      # max_iter < 0
    assert P.pitn_solve(77, p, x0, 1e-3, 10, 3, 1e-10, 5, out) == E                    # system
    assert P.pitn_solve(P.PITN_LORENZ63, None, x0, 1e-3, 10, 3, 1e-10, 5, out) == E    # null
    assert P.pitn_solve(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, 1e-10, 5, None) == E
    assert P.pitn_solve(P.PITN_FKPP, np.ones(1), np.ones(200), 1e-3, 10, 200, 1e-10, 5,
                        np.zeros((10, 200))) == E                                        # d > 128
    # the option arrays marshal (residual and cut histories), the host check still fires
    opt = P.make_options(res_history=np.zeros(6), cut_history=np.zeros(6, dtype=np.int64))
    rc, _ = P.pitn_solve_ex(P.PITN_LORENZ63, p, x0, 1e-3, 0, 3, 1e-10, 5, out, opt)
    assert rc == E
    opt = P.make_options(precision=P.PITN_PREC_MIXED_BF16)
    rc, _ = P.pitn_solve_ex(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, 1e-10, 5, out, opt)
    assert rc == E                                                                       # mixed needs d >= 64
    for m in (4, -1):
        opt = P.make_options(method=m)
        rc, _ = P.pitn_solve_ex(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, 1e-10, 5, out, opt)
        assert rc == E                                                                   # unknown step map
    opt = P.make_options(method=P.PITN_STEP_BACKWARD_EULER)
    rc, _ = P.pitn_solve_ex(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, 1e-10, 5, out, opt)
    assert rc == P.PITN_EUNSUPPORTED                                                     # not instantiated
    opt = P.make_options(method=P.PITN_STEP_BACKWARD_EULER, precision=P.PITN_PREC_MIXED_FP32)
    rc, _ = P.pitn_solve_ex(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, 1e-10, 5, out, opt)
    assert rc == E                                                                       # FP32 form: no implicit Lorenz
    opt = P.make_options(method=P.PITN_STEP_TRAPEZOID, precision=P.PITN_PREC_FP64_FF)
    rc, _ = P.pitn_solve_ex(P.PITN_LORENZ63, p, x0, 1e-3, 10, 3, 1e-10, 5, out, opt)
    assert rc == E                                                                       # float-float: no implicit Lorenz
    assert not out.any()  # nothing written on an argument error


def test_tune_cache_file_is_read(tmp_path, lib):
    """The autotuner's cache file (PITN_TUNE_CACHE) is loaded on first use."""
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    cache.write_text("small:2:2:22:1 128 3\nbatch:1:3:27:1 256 16\n")
    code = ("from paper_2511_01465_gb300 import pitn as P; "
            "print(P.pitn_tune_get('small:2:2:22:1'), P.pitn_tune_get('batch:1:3:27:1'), "
            "P.pitn_tune_get('nope'))")
    env = dict(os.environ, PITN_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "(128, 3) (256, 16) None"


def test_tune_set_pins_a_shape(tmp_path, lib):
    """pitn_tune_set stores an entry (and writes it to the cache file)."""
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    code = ("from paper_2511_01465_gb300 import pitn as P; "
            "print(P.pitn_tune_set('small:7:3:22:0:be', 256, 1), P.pitn_tune_get('small:7:3:22:0:be'), "
            "P.pitn_tune_set('x', 0, 1), P.pitn_tune_set('', 1, 1), P.pitn_tune_set('small:1:3:13:1', 100, 1), "
            "P.pitn_tune_set('small:1:3:13:1', 128, 0), P.pitn_tune_set('batch:1:3:13:1', 128, 0), "
            "P.pitn_tune_get('batch:1:3:13:1'))")
    env = dict(os.environ, PITN_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "0 (256, 1) -1 -1 -1 -1 0 (128, 0)"
    assert sorted(cache.read_text().splitlines()) == ["batch:1:3:13:1 128 0", "small:7:3:22:0:be 256 1"]


def test_precision_support_matrix(lib):
    """The reduced-precision scans are accepted exactly where include/pitn.h
    documents them (FP32 delta form and float-float: Lorenz-63, van der Pol,
    oscillator with explicit Euler; van der Pol with RK4; Robertson,
    Dahlquist, van der Pol, logistic with backward Euler or the trapezoidal
    rule; BF16 / TF32 only for Fisher-KPP) and refused on the host
    (PITN_EINVAL, nothing written) everywhere else."""
    from paper_2511_01465_gb300 import pitn as P
    dims = {P.PITN_LORENZ63: 3, P.PITN_VDP: 2, P.PITN_LINEAR_OSC: 2, P.PITN_LOGISTIC: 1,
            P.PITN_DAHLQUIST: 1, P.PITN_ROBERTSON: 3}
    implicit = (P.PITN_STEP_BACKWARD_EULER, P.PITN_STEP_TRAPEZOID)

    def reduced_ok(sys, m):
        return ((sys in (P.PITN_LORENZ63, P.PITN_VDP, P.PITN_LINEAR_OSC) and m == P.PITN_STEP_EULER)
                or (sys == P.PITN_VDP and m == P.PITN_STEP_RK4)
                or (sys in (P.PITN_ROBERTSON, P.PITN_DAHLQUIST, P.PITN_VDP, P.PITN_LOGISTIC) and m in implicit))

    # (an accepted request goes on to device work, which without a GPU fails
    # slowly: one accepted request per step map and reduced precision is run)
    accepted_run = set()
    for sys, d in dims.items():
        p = np.full(P.pitn_num_params(sys), 0.5)
        x0 = np.full(d, 0.5)
        for m in (P.PITN_STEP_EULER, P.PITN_STEP_RK4, P.PITN_STEP_BACKWARD_EULER, P.PITN_STEP_TRAPEZOID):
            for prec in (P.PITN_PREC_MIXED_BF16, P.PITN_PREC_MIXED_FP32, P.PITN_PREC_FP64_FF,
                         P.PITN_PREC_MIXED_TF32):
                if prec in (P.PITN_PREC_MIXED_BF16, P.PITN_PREC_MIXED_TF32):
                    valid = False
                else:
                    valid = reduced_ok(sys, m)
                if valid and (m, prec) in accepted_run:
                    continue
                out = np.full((10, d), 7.0)
                opt = P.make_options(method=m, precision=prec)
                rc, _ = P.pitn_solve_ex(sys, p, x0, 1e-3, 10, d, 1e-10, 5, out, opt)
                if valid:
                    accepted_run.add((m, prec))
                    assert rc != P.PITN_EINVAL, (sys, m, prec, rc)
                else:
                    assert rc == P.PITN_EINVAL and (out == 7.0).all(), (sys, m, prec, rc)
    assert len(accepted_run) == 8


def test_batch_work_before_any_batch_solve(lib):
    """pitn_batch_work reports zeros until a batch solve has run in the
    process, and refuses NULL pointers."""
    import subprocess
    import sys
    code = ("import ctypes; from paper_2511_01465_gb300 import pitn as P; "
            "print(P.pitn_batch_work(), P.lib().pitn_batch_work(None, None))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "(0, 0) -1"
