"""Writes oracle_rounding_spread.json: the rounding spread of the guarded
full-size workloads, measured on the CPU oracle's rounding variants.

Calls only the CPU oracle (``oracle/``, the oracle itself and its rounding
variants, see ``tests/rounding.py``) on the seeded inputs of
``paper_2511_01465_gb300.workloads``.  For each case it stores the oracle's
Newton count, status, guard index, per-step cuts and residual history, every
variant's count, status and first cut that differs from the oracle's, and
the two figures the GPU parity tests use: ``window`` (the largest count
difference of a variant from the oracle) and ``first_div`` (the first Newton
step at which a variant cut elsewhere).  Under ``ff`` it stores the same three
figures over the FP64 variants and the 48-bit-scan variant ``s48`` together:
the bar of the float-float scan, whose corrections carry 48 significant bits.

    python tests/golden/make_rounding_spread.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CASES = {
    # name: (workload, constructor arguments, tol, max_iter, guard_B)
    "lorenz_8192_guard100_tol1e-10_it50": ("lorenz", {}, 1e-10, 50, 100.0),
    "lorenz_8192_guard100_tol1e-12_it100": ("lorenz", {}, 1e-12, 100, 100.0),
    "lorenz_8192_guard100_tol1e-8_it100": ("lorenz", {}, 1e-8, 100, 100.0),
    "vdp_2^22_guard100_tol1e-12_it400": ("vdp", {}, 1e-12, 400, 100.0),
    "vdp_2^22_guard100_tol1e-8_it400": ("vdp", {}, 1e-8, 400, 100.0),
    # plain Newton that diverges: the index at which the rejected correction overflows
    "vdp_30001_h1e-3_plain_tol1e-10_it60": ("vdp", {"N": 30001, "h": 1e-3}, 1e-10, 60, 0.0),
}


def _one(task):
    name, variant = task
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2511_01465_gb300 import workloads as W
    kind, kw, tol, it, B = CASES[name]
    wl = getattr(W, kind)(**kw)
    t = time.time()
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, tol, it, guard_B=B, variant=variant)
    return name, variant, dict(iters=int(r["iters"]), status=int(r["status"]),
                               guard_index=int(r["guard_index"]), cuts=[int(c) for c in r["cuts"]],
                               res_history=[float(v) for v in r["res_hist"]]), time.time() - t


def main():
    import oracle as O
    sys.path.insert(0, os.path.dirname(HERE))
    from rounding import first_difference, first_res_difference
    variants = [None] + list(O.VARIANTS) + list(O.SCAN_VARIANTS)
    fp64 = list(O.VARIANTS)
    for v in variants:
        O.build(variant=v)
    tasks = [(n, v) for n in CASES for v in variants]
    with mp.get_context("spawn").Pool(min(len(tasks), os.cpu_count() or 4)) as pool:
        results = pool.map(_one, tasks, chunksize=1)
    by = {}
    for name, v, r, dt in results:
        by.setdefault(name, {})[v] = r
        print(f"{name} {v}: iters={r['iters']} status={r['status']} ({dt:.0f} s)", flush=True)
    out = {"_source": "tests/golden/make_rounding_spread.py (CPU oracle and its rounding variants only)"}
    for name, rs in by.items():
        ref = rs[None]
        var = {}
        for v in variants[1:]:
            r = rs[v]
            var[v] = dict(iters=r["iters"], status=r["status"],
                          first_cut_difference=first_difference(ref["cuts"], r["cuts"]),
                          first_res_difference=first_res_difference(r["res_history"], ref["res_history"]))
        kind, kw, tol, it, B = CASES[name]
        rej = 0
        if len(ref["cuts"]) > ref["iters"]:
            rej = max(abs(rs[v]["cuts"][-1] - ref["cuts"][-1]) for v in [None] + fp64)

        def figures(names):
            return dict(window=max([abs(rs[v]["iters"] - ref["iters"]) for v in names] + [0]),
                        first_div=min(var[v]["first_cut_difference"] for v in names),
                        first_res_div=min(var[v]["first_res_difference"] for v in names))
        out[name] = dict(workload=kind, kwargs=kw, tol=tol, max_iter=it, guard_B=B, rejected_cut_window=rej,
                         oracle=ref, variants=var, **figures(fp64), ff=figures(variants[1:]))
    with open(os.path.join(HERE, "oracle_rounding_spread.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
