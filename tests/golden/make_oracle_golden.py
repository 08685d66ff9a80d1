"""Writes oracle_full_size.json: CPU-oracle outcomes of the full-size workloads.

Calls only the CPU oracle (``oracle/``) on the seeded inputs of
``paper_2511_01465_gb300.workloads``; the GPU parity tests compare the CUDA
path's iteration counts, statuses, guard indices and residual histories with
these stored values instead of re-running the slow oracle solves.

    python tests/golden/make_oracle_golden.py [--missing]

--missing keeps the stored entries and computes only the cases not yet in
the file.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2511_01465_gb300 import workloads as W  # noqa: E402

CASES = {
    # name: (workload, tol, max_iter, guard_B[, step map, constant guess])
    "lorenz_8192_plain_tol1e-10_it50": (W.lorenz(), 1e-10, 50, 0.0),
    "lorenz_8192_guard100_tol1e-10_it50": (W.lorenz(), 1e-10, 50, 100.0),
    "lorenz_8192_guard100_tol1e-12_it100": (W.lorenz(), 1e-12, 100, 100.0),
    "vdp_2^22_plain_tol1e-8_it200": (W.vdp(), 1e-8, 200, 0.0),
    "vdp_2^22_guard100_tol1e-12_it400": (W.vdp(), 1e-12, 400, 100.0),
    "osc_2^22_plain_tol1e-8_it10": (W.damped_oscillator(), 1e-8, 10, 0.0),
    # the bench's tolerance for the guarded van der Pol and Lorenz solves
    "vdp_2^22_guard100_tol1e-8_it400": (W.vdp(), 1e-8, 400, 100.0),
    "lorenz_8192_guard100_tol1e-8_it100": (W.lorenz(), 1e-8, 100, 100.0),
    "fkpp_d128_2^15_plain_tol1e-8_it50": (W.fkpp(), 1e-8, 50, 0.0),
    # backward Euler, the paper's zero guess, Robertson on [0, 500] at h = 1e-4
    "robertson_5e6_be_zeros_tol1e-8_it60": (W.robertson(h=1e-4), 1e-8, 60, 0.0, O.BACKWARD_EULER, 0.0),
    # classical RK4, the paper's ones guess, van der Pol on [0, 10] at h = 1e-5
    "vdp_rk4_1e6_ones_tol1e-8_it50": (W.vdp_paper(h=1e-5), 1e-8, 50, 0.0, O.RK4, 1.0),
}


def main():
    path = os.path.join(HERE, "oracle_full_size.json")
    out = {"_source": "tests/golden/make_oracle_golden.py (CPU oracle only)"}
    if "--missing" in sys.argv[1:] and os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for name, case in CASES.items():
        if name in out:
            continue
        wl, tol, it, B = case[:4]
        method = case[4] if len(case) > 4 else O.EULER
        guess = np.full((wl.N, wl.d), case[5]) if len(case) > 5 else None
        t = time.time()
        r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, it, guard_B=B, guess=guess,
                     method=method)
        out[name] = dict(system=wl.system, N=wl.N, h=wl.h, tol=tol, max_iter=it, guard_B=B,
                         method=method, guess=None if len(case) <= 5 else case[5],
                         iters=r["iters"], status=r["status"], guard_index=r["guard_index"],
                         res_history=[float(v) for v in r["res_hist"]])
        print(f"{name}: iters={r['iters']} status={r['status']} ({time.time() - t:.1f}s)", flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
