"""The integer-pipe FP64 <-> FP32 conversions used by the mixed-precision
small-state scan agree with the GPU's own conversions: double -> float
rounds to nearest (an exact tie may round away from zero), subnormal
results flush to signed zero; float -> double is exact."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2511_01465_gb300", "csrc")


def test_fpconv_against_hardware(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "fpconv_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "gpu_helpers", "fpconv_check.cu")], check=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    f = out.stdout.split()
    counts = dict(zip(f[0::2], map(int, f[1::2])))
    assert counts["checked"] >= 1 << 24
    assert counts["d2f_bad"] == 0 and counts["d2f_far"] == 0, counts
    assert counts["f2d_bad"] == 0 and counts["f2d_sub_bad"] == 0, counts
