"""Host logic of bench.py (no GPU): workload specs, the roofline arithmetic of
the JSON line, the stored oracle pass counts and the CPU-baseline leg."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SINGLE = ["vdp", "vdp_mixed", "vdp_ff", "vdp_rk4", "vdp_rk4_ff", "vdp_rk4_mixed", "robertson", "robertson_mixed",
          "robertson_ff", "osc", "lorenz", "lorenz_mixed", "lorenz_ff", "fkpp", "fkpp_mixed", "fkpp_tf32"]


@pytest.mark.parametrize("name", SINGLE + ["batch", "batch_small", "adjoint"])
def test_workload_specs(name):
    spec = bench.workload(name)
    assert spec["kind"] in ("single", "batch", "adjoint")
    assert spec["tol"] > 0 and spec["max_iter"] >= 1 and "desc" in spec
    if spec["kind"] == "single":
        wl = spec["wl"]
        assert wl.N >= 1 and wl.d == len(wl.x0) and wl.h > 0
        assert name in bench.SAMPLE_ITERS


def test_unknown_workload():
    with pytest.raises(SystemExit):
        bench.workload("nope")


@pytest.mark.parametrize("name", SINGLE)
def test_oracle_passes_stored(name):
    # every single-IVP bench workload has the oracle's own pass count stored
    n = bench.oracle_passes(name, -1)
    assert isinstance(n, int) and n >= 1


def _fake_res(iters):
    return SimpleNamespace(iters=iters, status=0, final_res=1e-9)


@pytest.mark.parametrize("name,kern", [("vdp", "newton_small"), ("vdp_rk4", "newton_small"),
                                       ("robertson", "newton_small"), ("vdp_mixed", "newton_small"),
                                       ("fkpp", "fkpp_fold"), ("fkpp_mixed", "fkpp_compose")])
def test_roofline_arithmetic(name, kern):
    spec = bench.workload(name)
    wl = spec["wl"]
    steps, ms = 3, 30.0
    rf = bench.roofline_for(name, spec, wl, _fake_res(10), {kern: (ms, steps)}, steps)
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel"):
        assert k in rf
    assert rf["kernel"] == kern and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-12
    assert rf["bound"] in ("alu", "hbm", "tensor")
    if kern != "newton_small":
        assert rf["traffic"] is None
    # the achieved rate scales inversely with the kernel time
    rf2 = bench.roofline_for(name, spec, wl, _fake_res(10), {kern: (2 * ms, steps)}, steps)
    assert abs(rf2["achieved"] * 2 - rf["achieved"]) <= 1e-9 * rf["achieved"]


def test_cpu_baseline_leg(monkeypatch):
    monkeypatch.setattr(bench, "CPU_SAMPLE_S", 0.05)
    spec = bench.workload("lorenz")
    cb = bench.cpu_baseline(spec, bench.oracle_passes("lorenz", 63), 3)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0 and cb["unit"] == bench.UNIT
    assert "residual evaluations" in cb["sample"]


def test_batch_kernel_name():
    assert bench.batch_kernel_name([128, 0]).startswith("batch_ivp_kernel")
    assert "graph" in bench.batch_kernel_name([256, 32])
    assert "default" in bench.batch_kernel_name(None)


def test_fkpp_tree_counts():
    # 2^15 steps: 512 tiles of 64 make 3.4 waves on 152 SMs; 607 tiles of 54 make 4
    assert bench.fk_tiles(1 << 15) == 607
    assert bench.fk_tiles(65) == 1 and bench.fk_tiles(130) == 3
    # below one wave the tiles stay at 64 steps
    assert bench.fk_tiles(64 * 100 + 1) == 100
    # composes: levels below the root pair their nodes; the root is not composed
    assert bench.fk_composes(1) == 0 and bench.fk_composes(2) == 0
    assert bench.fk_composes(3) == 1       # 3 -> 2 (one compose + a lone copy) -> root
    assert bench.fk_composes(8) == 4 + 2   # 8 -> 4 -> 2 -> root
    assert bench.fk_composes(512) == 256 + 128 + 64 + 32 + 16 + 8 + 4 + 2


def test_reference_arm_batch_line(monkeypatch):
    # the batch reference line carries every contract key, ms_per_step included
    fake = {"value": 2.0e6, "unit": bench.UNIT, "cores": 4, "kind": "oracle", "sample": "fake sample"}
    monkeypatch.setattr(bench, "cpu_baseline_batch_pool", lambda spec: dict(fake))
    args = SimpleNamespace(workload="batch_small", steps=2, warmup=3)
    line = bench.run_reference(args)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] == 2.0e6
    bt = bench.workload("batch_small")["bt"]
    # ms_per_step is the measured wall time of a step (one bounded sample);
    # the whole batch at the sampled rate is reported beside it
    assert 0 < line["ms_per_step"] < 1e3
    assert line["config"]["projected_ms_per_solve"] == pytest.approx(float(bt.N.sum()) / 2.0e6 * 1e3)
    assert line["cpu_baseline"]["cores"] == 4 and line["e2e"]["h2d_bytes_per_step"] == 0


def test_clock_sampler_window():
    """The clock record is that of the samples stamped inside the timed
    region; with none there (a timed region shorter than the sampling
    interval), that of the warm-up and the timed region, marked so."""
    import datetime

    class FakeSmi:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    now = datetime.datetime.now()

    def line(dt, mhz, cap="Not Active"):
        ts = (now + datetime.timedelta(seconds=dt)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.00, 0x0, Not Active, Not Active, Not Active, {cap}"

    cs = bench.ClockSampler("0")
    cs.proc = FakeSmi()
    cs.lines = [line(-1.0, 1500), line(-0.5, 1980, "Active"), "garbage"]
    cs.t_timed = now - datetime.timedelta(seconds=0.2)
    r = cs.stop()
    assert r["samples"] == 2 and r["sm_mhz"] == 1740 and r["reasons"] == ["sw_power_cap"]
    assert r["window"].startswith("warm-up")

    cs = bench.ClockSampler("0")
    cs.proc = FakeSmi()
    cs.lines = [line(-1.0, 1500, "Active"), line(-0.1, 2070), line(-0.05, 2060), line(5.0, 100)]
    cs.t_timed = now - datetime.timedelta(seconds=0.2)
    r = cs.stop()
    assert r == {"sm_mhz": 2065, "sm_max_mhz": 2070, "reasons": [], "samples": 2, "window": "timed region"}



@pytest.mark.parametrize("name", [n for n in SINGLE if not n.startswith("fkpp")])
def test_small_state_roofline_counts(name):
    """Every small-state workload has its per-step FP64 work (SMALL_FLOPS for
    the FP64 kernels, REDUCED_FP64 for the reduced-precision scans) and, while
    the kernel sources are unchanged, its captured DRAM traffic."""
    spec = bench.workload(name)
    if spec.get("precision", 0) in (2, 3):
        ops, flops = bench.REDUCED_FP64[name]
        assert 0 < ops <= flops
    else:
        p1, p3 = bench.SMALL_FLOPS[name]
        assert p1 > 0 and p3 > 0
    t = bench.TRAFFIC.get(name)
    assert t is not None and t[0] > 0


@pytest.mark.parametrize("name", sorted(bench.TWINS))
def test_reduced_precision_twins_match(name):
    """The comparison lines of an FP64 workload solve the same problem to the
    same tolerance and limits, only with the FP32 / float-float scans."""
    base = bench.workload(name)
    for twin, prec in zip(bench.TWINS[name], (2, 3)):
        t = bench.workload(twin)
        assert t["precision"] == prec and base.get("precision", 0) == 0
        for k in ("tol", "max_iter", "guard_B"):
            assert t[k] == base[k]
        assert t.get("method", 0) == base.get("method", 0) and t.get("guess") == base.get("guess")
        assert (t["wl"].system, t["wl"].N, t["wl"].h) == (base["wl"].system, base["wl"].N, base["wl"].h)
