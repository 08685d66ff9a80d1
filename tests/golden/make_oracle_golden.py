"""Writes oracle_full_size.json: CPU-oracle outcomes of the full-size workloads.

Calls only the CPU oracle (``oracle/``) on the seeded inputs of
``paper_2511_01465_gb300.workloads``; the GPU parity tests compare the CUDA
path's iteration counts, statuses, guard indices and residual histories with
these stored values instead of re-running the slow oracle solves.

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2511_01465_gb300 import workloads as W  # noqa: E402

CASES = {
    # name: (workload, tol, max_iter, guard_B)
    "lorenz_8192_plain_tol1e-10_it50": (W.lorenz(), 1e-10, 50, 0.0),
    "lorenz_8192_guard100_tol1e-10_it50": (W.lorenz(), 1e-10, 50, 100.0),
    "lorenz_8192_guard100_tol1e-12_it100": (W.lorenz(), 1e-12, 100, 100.0),
    "vdp_2^22_plain_tol1e-8_it200": (W.vdp(), 1e-8, 200, 0.0),
    "vdp_2^22_guard100_tol1e-12_it400": (W.vdp(), 1e-12, 400, 100.0),
    "osc_2^22_plain_tol1e-8_it10": (W.damped_oscillator(), 1e-8, 10, 0.0),
    "fkpp_d128_2^15_plain_tol1e-8_it50": (W.fkpp(), 1e-8, 50, 0.0),
}


def main():
    out = {"_source": "tests/golden/make_oracle_golden.py (CPU oracle only)"}
    for name, (wl, tol, it, B) in CASES.items():
        t = time.time()
        r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, it, guard_B=B)
        out[name] = dict(system=wl.system, N=wl.N, h=wl.h, tol=tol, max_iter=it, guard_B=B,
                         iters=r["iters"], status=r["status"], guard_index=r["guard_index"],
                         res_history=[float(v) for v in r["res_hist"]])
        print(f"{name}: iters={r['iters']} status={r['status']} ({time.time() - t:.1f}s)", flush=True)
    with open(os.path.join(HERE, "oracle_full_size.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
