"""Measured FP64 and FP32 FMA rates of the current GPU.

    python -m paper_2511_01465_gb300.peaks

Prints one JSON line: the thread-level FMA rates that pitn_probe_fma_rate
measures (FP64 DFMA and FP32 FFMA; one FMA = 2 flops), the flop rates they
imply, their ratio, and the SM clock sampled by nvidia-smi while the probes
run.  The benchmark takes its ALU roofline denominators from the same probe,
in the same process as the timed solves.
"""
from __future__ import annotations

import json
import subprocess


def sm_clock():
    try:
        out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.sm,clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=10).stdout.strip().splitlines()
        cur, mx = (float(x) for x in out[0].split(","))
        return cur, mx
    except Exception:
        return None, None


def measure():
    import torch
    from . import pitn as P
    torch.cuda.init()
    f64 = P.pitn_probe_fma_rate(0)
    clk0 = sm_clock()
    f32 = P.pitn_probe_fma_rate(1)
    clk1 = sm_clock()
    return {"fp64_fma_per_s": f64, "fp64_tflops": 2 * f64 / 1e12,
            "fp32_fma_per_s": f32, "fp32_tflops": 2 * f32 / 1e12,
            "fp32_over_fp64": f32 / f64,
            "sm_mhz_after_fp64": clk0[0], "sm_mhz_after_fp32": clk1[0], "sm_max_mhz": clk1[1],
            "device": torch.cuda.get_device_name(0)}


def main():
    from . import build
    build.build()
    print(json.dumps(measure()), flush=True)


if __name__ == "__main__":
    main()
