"""Benchmark of the parallel-in-time Newton solver on one or more GB300s.

One step = one complete Newton solve (every residual evaluation, scan and
update until ||h||_inf <= tol) of the selected workload, inputs resident on
the device.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload vdp|lorenz|osc|fkpp|fkpp_mixed|batch|batch_small|adjoint]
    python bench.py --impl reference ...     # the CPU oracle, timed on the host cores

Multi-GPU (torchrun, one rank per GPU): every rank solves its own replica of
the workload (the single-IVP solve does not shard across GPUs); value is the
total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton-solved time steps/s at residual<=1e-8"
UNIT = "steps/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), \
            d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# FP64 peak of a GB300 (nominal 1.25 TFLOP/s dense FP64, FMA = 2 flops).
FP64_PEAK_TFLOPS = 1.25

# FP64 flops per step per Newton pass executed by the fused small-state
# kernel (residual + compact Jacobian + thread fold + replay + update; FMA
# counted as 2), counted from the kernel source.  The warp/block scan and the
# look-back add a per-thread overhead amortised over C steps, not counted.
FLOPS_PER_STEP = {"vdp": 44.0, "osc": 38.0, "lorenz": 104.0}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload(name):
    from paper_2511_01465_gb300 import workloads as W
    if name == "vdp":
        return dict(kind="single", wl=W.vdp(), tol=1e-8, max_iter=400, guard_B=100.0,
                    desc="van_der_pol mu=1 x0=(2,0) explicit Euler h=1e-4 N=2^22, guarded Newton B=100")
    if name == "osc":
        return dict(kind="single", wl=W.damped_oscillator(), tol=1e-8, max_iter=10, guard_B=0.0,
                    desc="damped oscillator omega=1 zeta=0.05 x0=(2,0) h=1e-4 N=2^22, plain Newton")
    if name == "lorenz":
        return dict(kind="single", wl=W.lorenz(), tol=1e-8, max_iter=100, guard_B=100.0,
                    desc="lorenz63 sigma=10 rho=28 beta=8/3 x0=(1,1,1) h=1e-3 N=8192, guarded Newton B=100")
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2511_01465_gb300 as pk
    from paper_2511_01465_gb300 import pitn as P

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    spec = workload(args.workload)
    wl = spec["wl"]
    stream = torch.cuda.current_stream(dev)
    params = torch.tensor(wl.params, dtype=torch.float64, device=dev)
    x0 = torch.tensor(wl.x0, dtype=torch.float64, device=dev)
    traj = torch.empty((wl.N, wl.d), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    opt = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream)

    def solve_once():
        rc, res = P.pitn_solve_ex(wl.system, params, x0, wl.h, wl.N, wl.d, spec["tol"],
                                  spec["max_iter"], traj, opt)
        P.check(rc, "pitn_solve_ex")
        return rc, res

    for _ in range(args.warmup):
        rc, res = solve_once()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local_rank)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    launches0 = pk.pitn_launch_count()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict the trajectory from L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        rc, res = solve_once()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = pk.pitn_launch_count() - launches0
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = float(sum(times))
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    converged = res.status == P.PITN_OK and res.final_res <= 1e-8
    steps_solved = wl.N if converged else 0
    value = world * steps_solved / (ms_per_step / 1e3)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if True:
        h_params = torch.tensor(wl.params, dtype=torch.float64).pin_memory()
        h_x0 = torch.tensor(wl.x0, dtype=torch.float64).pin_memory()
        h_traj = torch.empty((wl.N, wl.d), dtype=torch.float64).pin_memory()
        hp, hx, ht = h_params.numpy(), h_x0.numpy(), h_traj.numpy()
        opt_h = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream)
        P.pitn_solve_ex(wl.system, hp, hx, wl.h, wl.N, wl.d, spec["tol"], spec["max_iter"], ht, opt_h)
        et = []
        for _ in range(max(1, min(args.steps, 5))):
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rc2, r2 = P.pitn_solve_ex(wl.system, hp, hx, wl.h, wl.N, wl.d, spec["tol"],
                                      spec["max_iter"], ht, opt_h)
            et.append(time.perf_counter() - t0)
        e2e_s = statistics.median(et)
        e2e_ok = r2.status == P.PITN_OK and r2.final_res <= 1e-8
        e2e = {"value": (world * wl.N / e2e_s) if e2e_ok else 0.0, "unit": UNIT,
               "h2d_bytes_per_step": int((wl.d + len(wl.params)) * 8),
               "d2h_bytes_per_step": int(wl.N * wl.d * 8), "ms_per_step": e2e_s * 1e3}

    passes = res.iters + 1
    flops = FLOPS_PER_STEP[args.workload] * wl.N * passes
    achieved_tflops = flops / (ms_per_step / 1e3) / 1e12
    hbm, _, _, src = load_peaks()
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "newton_small_kernel", "peak_source": "nominal GB300 FP64",
                "hbm_frac_of_" + src: (2 * wl.N * wl.d * 8 * passes) / (ms_per_step / 1e3) / 1e9 / hbm}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec["desc"], "N": wl.N, "d": wl.d, "tol": spec["tol"],
                       "max_iter": spec["max_iter"], "newton_updates": res.iters,
                       "status": P.pitn_status_string(res.status), "final_res": res.final_res,
                       "l2": "flushed (512 MiB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}
    return line


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(spec, sample_iters):
    """Times the oracle's Newton solve on the full workload for a bounded number
    of Newton iterations and projects to the full solve's residual count."""
    import oracle as O
    wl = spec["wl"]
    t0 = time.perf_counter()
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, spec["tol"], sample_iters,
                 guard_B=spec["guard_B"])
    dt = time.perf_counter() - t0
    evals = r["iters"] + 1
    return dt / evals, r


def cpu_baseline(spec, full_passes, sample_iters):
    per_eval, r = oracle_sample(spec, sample_iters)
    wl = spec["wl"]
    t_full = per_eval * full_passes
    return {"value": wl.N / t_full, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle Newton on the full workload, first {r['iters'] + 1} residual "
                      f"evaluations ({per_eval * (r['iters'] + 1):.1f} s), projected to the "
                      f"{full_passes} evaluations of the full solve"}


def run_reference(args):
    spec = workload(args.workload)
    wl = spec["wl"]
    import oracle as O
    # number of residual evaluations of the full solve (oracle iteration count)
    full_passes = {"vdp": 157, "osc": 2, "lorenz": 63}.get(args.workload)
    sample_iters = {"vdp": 6, "osc": 1, "lorenz": 62}.get(args.workload, 5)
    for _ in range(args.warmup):
        oracle_sample(spec, 0)
    vals = []
    for _ in range(args.steps):
        per_eval, r = oracle_sample(spec, sample_iters)
        vals.append(wl.N / (per_eval * full_passes))
    v = statistics.median(vals)
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wl.N / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": spec["desc"], "N": wl.N, "d": wl.d, "tol": spec["tol"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"per step: oracle Newton, {sample_iters + 1} residual "
                                       f"evaluations of the full workload, projected to {full_passes}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="vdp")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    # the oracle process pool, if any, must start before the first GPU call
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__ as ge
    ge.build_library_only()
    line = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        full_passes = line["config"]["newton_updates"] + 1
        sample_iters = {"vdp": 6, "osc": 1, "lorenz": 62}.get(args.workload, 5)
        line["cpu_baseline"] = cpu_baseline(workload(args.workload), full_passes, sample_iters)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
