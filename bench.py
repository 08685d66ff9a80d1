"""Benchmark of the parallel-in-time Newton solver on one or more GB300s.

One step = one complete Newton solve (every residual evaluation, scan and
update until ||h||_inf <= tol) of the selected workload, inputs resident on
the device.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload vdp|vdp_mixed|vdp_ff|vdp_rk4|vdp_rk4_ff|vdp_rk4_mixed|lorenz|lorenz_mixed|lorenz_ff|osc|
                                                      robertson|robertson_mixed|robertson_ff|fkpp|fkpp_mixed|fkpp_tf32|batch|batch_small|adjoint]
    python bench.py --impl reference ...     # the CPU oracle, timed on the host cores

Multi-GPU (torchrun, one rank per GPU): every rank solves its own replica of
the workload (the single-IVP solve does not shard across GPUs); value is the
total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
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

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, from an ncu capture of the bench command itself (summaries
# under profiles/), keyed by workload and tagged with a hash of the kernel
# sources they were taken on: a changed kernel reports traffic null.
SMALL_SRC = ["newton_small.cuh", "newton_small.cu", "newton_small_mixed.cuh", "newton_fused.cuh",
             "newton_fused_mixed.cuh", "newton_implicit.cu", "systems.cuh", "fpconv.cuh", "ffarith.cuh",
             "scan_policy.cuh",
             "common.cuh"]
TRAFFIC = {
    # workload: (bytes per launch of the timed solve, kernel-source hash)
    "vdp": (28936841472 + 24172120576, "66a389d6a17f759c"),  # 147 passes, newton_small_kernel<VanDerPol>
    "vdp_ff": (25473908736 + 27281655552, "66a389d6a17f759c"),  # 151 passes, newton_fused_mixed_kernel<VanDerPol, ScanFF>
    "vdp_mixed": (18092340736 + 15309869824, "66a389d6a17f759c"),  # 137 passes, newton_fused_mixed_kernel<VanDerPol, ScanF32>
    "lorenz": (158208 + 45312, "66a389d6a17f759c"),  # 64 passes, newton_small_kernel<Lorenz63>
    "lorenz_ff": (224512 + 34304, "66a389d6a17f759c"),  # 62 passes, newton_small_mixed_kernel<Lorenz63, ScanFF>
    "lorenz_mixed": (99840 + 25088, "66a389d6a17f759c"),  # 52 passes, newton_small_mixed_kernel<Lorenz63, ScanF32>
    "vdp_rk4": (31176192 + 345217536, "66a389d6a17f759c"),  # 8 passes, newton_fused_kernel<RK4Map<VdpRhs>>
    "vdp_rk4_ff": (44198144 + 338967808, "66a389d6a17f759c"),  # 8 passes, newton_fused_mixed_kernel<RK4Map<VdpRhs>, ScanFF>
    "vdp_rk4_mixed": (16180480 + 20744192, "66a389d6a17f759c"),  # 8 passes, newton_fused_mixed_kernel<RK4Map<VdpRhs>, ScanF32>
    "robertson": (13365496320 + 13725852672, "66a389d6a17f759c"),  # 22 passes, newton_fused_kernel<BackwardEulerMap<RobertsonRhs>>
    "robertson_mixed": (8638719488 + 8672999168, "66a389d6a17f759c"),  # 23 passes, newton_fused_mixed_kernel<BackwardEulerMap<RobertsonRhs>, ScanF32>
    "robertson_ff": (13365422592 + 13701216512, "66a389d6a17f759c"),  # 22 passes, newton_fused_mixed_kernel<BackwardEulerMap<RobertsonRhs>, ScanFF>
    "osc": (102232576 + 197507840, "66a389d6a17f759c"),  # 2 passes, newton_small_kernel<LinearOsc>
}


def kernel_src_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2511_01465_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(name):
    t = TRAFFIC.get(name)
    if not t or t[1] != kernel_src_hash(SMALL_SRC):
        return None
    return t[0]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), \
            d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ALU peaks.  Measured in the bench process itself by the library's
# register-only FMA probe (pitn_probe_fma_rate: FP64 DFMA and FP32 FFMA
# issue rates, FMA = 2 flops); profiles/fp64_peak.md records one such
# measurement (0.525 T DFMA/s, 39.0 T FFMA/s at 2070 MHz).  The figures
# below are what the unit counts and clocks give, used only until the
# probe has run: FP64 nominal 1.25 TFLOP/s; FP32 152 SMs x 128 lanes x 2 x
# 2.07 GHz = 80.5 TFLOP/s.
PEAKS = {"fp64_tflops": 1.25, "fp32_tflops": 152 * 128 * 2 * 2.07e9 / 1e12, "source": "unit counts"}


def measure_alu_peaks():
    from paper_2511_01465_gb300 import pitn as P
    PEAKS["fp64_tflops"] = 2 * P.pitn_probe_fma_rate(0) / 1e12
    PEAKS["fp32_tflops"] = 2 * P.pitn_probe_fma_rate(1) / 1e12
    PEAKS["source"] = "measured in this run (pitn_probe_fma_rate)"
    return dict(PEAKS)


def fp64_peak():
    return PEAKS["fp64_tflops"]


def fp32_peak():
    return PEAKS["fp32_tflops"]


# Algorithmic bytes per step and Newton pass of the small-state solves: the
# state read once and written once (2 d doubles); everything else (the
# scan's scratch, a second read) is implementation traffic.
def small_alg_bytes(d):
    return 16 * d

# FP64 flops per step executed by the small-state kernel, counted from its
# source (FMA = 2): phase 1 (residual, compact Jacobian, thread fold) runs on
# every residual evaluation, phase 3 (replay, update) once per Newton update.
SMALL_FLOPS = {"vdp": (34.0, 9.0), "osc": (26.0, 9.0), "lorenz": (76.0, 19.0),
               "vdp_mixed": (34.0, 9.0), "lorenz_mixed": (76.0, 19.0),
               "vdp_ff": (34.0, 9.0),
               # backward Euler Robertson: f 8, Jf 9, I - h Jf 12, h_n 9, 3x3 inverse 42
               # (one division counted as 1), M^-1 h_n 18, dense fold 72; replay 18 + update 3
               "robertson": (170.0, 21.0),
               # RK4 van der Pol (fused kernel): four stages with their Jacobian chain
               # (8 + 3 x 24), weighted sums for phi and dphi/dx (20 + 34), fold 20;
               # replay 8 + update 2
               "vdp_rk4": (154.0, 10.0)}
# FP64 instructions per step (phase 1, phase 3) of the three-phase kernel,
# as counted by ncu (DADD + DFMA + DMUL thread instructions at 1 and 11 passes;
# equal to the count of the source)
FP64_OPS = {"vdp": (20.0, 6.0)}
# FP64 work per step and pass of the reduced-precision scans (fused kernel,
# one pass per Newton iteration): the van der Pol residual (7 instructions,
# 11 flops) and the update (FP32 scan: 2 DADD; float-float: 4 DADD)
REDUCED_FP64 = {"vdp_mixed": (9.0, 13.0), "vdp_ff": (11.0, 15.0), "lorenz_mixed": (13.0, 20.0),
                "lorenz_ff": (20.0, 23.0),
                # RK4 van der Pol, float-float Jacobian chain: the FP64 residual (four
                # right-hand sides 4 x 3, stage states 6, weighted sums 8, residual 4,
                # h/2 1) and the update (4 DADD)
                "vdp_rk4_ff": (35.0, 57.0),
                # the same residual with the FP32 scan's update (2 DADD)
                "vdp_rk4_mixed": (33.0, 55.0),
                # backward Euler Robertson: f, Jf, I - h Jf, h_n, the 3 x 3 inverse
                # (one division counted as 1 flop), M^-1 h_n, S's diagonal and the
                # update: 104 flops from the source; 74.8 FP64 instructions per step
                # and pass as counted by ncu (DFMA + DMUL + DADD thread instructions)
                "robertson_mixed": (74.8, 104.0),
                # the same FP64 work with the float-float update instead of S's
                # diagonal and the FP32 update: 69.8 FP64 instructions per step and
                # pass as counted by ncu
                "robertson_ff": (69.8, 104.0)}
# Fisher-KPP (d padded to 128): per step, fold of the dense column block
# (4 flops per entry in the working precision) + FP64 residual/diagonal and
# vector fold; per compose 2*128^3.
FK_FOLD_REAL_FLOPS = 128 * 128 * 4
FK_FOLD_F64_FLOPS = 128 * (15 + 5)
FK_COMPOSE_FLOPS = 2 * 128 ** 3


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
    if name == "vdp_rk4":
        return dict(kind="single", wl=W.vdp_paper(h=1e-5), tol=1e-8, max_iter=50, guard_B=0.0, method=1,
                    guess=1.0,
                    desc="van_der_pol mu=1 x0=(0,1) on [0,10], classical RK4 h=1e-5 N=1e6, plain Newton "
                         "from the ones guess (Sec. 4.1)")
    if name == "vdp_rk4_ff":
        return dict(kind="single", wl=W.vdp_paper(h=1e-5), tol=1e-8, max_iter=50, guard_B=0.0, method=1,
                    guess=1.0, precision=3,
                    desc="van_der_pol mu=1 x0=(0,1) on [0,10], classical RK4 h=1e-5 N=1e6, plain Newton "
                         "from the ones guess (Sec. 4.1), Jacobian chain and scan in double-FP32 "
                         "(float-float), FP64 residual and update")
    if name == "vdp_rk4_mixed":
        return dict(kind="single", wl=W.vdp_paper(h=1e-5), tol=1e-8, max_iter=50, guard_B=0.0, method=1,
                    guess=1.0, precision=2,
                    desc="van_der_pol mu=1 x0=(0,1) on [0,10], classical RK4 h=1e-5 N=1e6, plain Newton "
                         "from the ones guess (Sec. 4.1), Jacobian chain and scan in FP32 delta form "
                         "(inexact Newton), FP64 residual and update")
    if name == "vdp_mixed":
        return dict(kind="single", wl=W.vdp(), tol=1e-8, max_iter=400, guard_B=100.0, precision=2,
                    desc="van_der_pol mu=1 x0=(2,0) explicit Euler h=1e-4 N=2^22, guarded Newton B=100, "
                         "scan in FP32 delta form (inexact Newton), FP64 residual and update")
    if name == "vdp_ff":
        return dict(kind="single", wl=W.vdp(), tol=1e-8, max_iter=400, guard_B=100.0, precision=3,
                    desc="van_der_pol mu=1 x0=(2,0) explicit Euler h=1e-4 N=2^22, guarded Newton B=100, "
                         "scan in double-FP32 (float-float), FP64 residual and update")
    if name == "lorenz_ff":
        return dict(kind="single", wl=W.lorenz(), tol=1e-8, max_iter=100, guard_B=100.0, precision=3,
                    desc="lorenz63 N=8192 h=1e-3, guarded Newton B=100, scan in double-FP32 (float-float)")
    if name == "lorenz_mixed":
        return dict(kind="single", wl=W.lorenz(), tol=1e-8, max_iter=100, guard_B=100.0, precision=2,
                    desc="lorenz63 N=8192 h=1e-3, guarded Newton B=100, scan in FP32 delta form")
    if name == "robertson":
        return dict(kind="single", wl=W.robertson(h=1e-4), tol=1e-8, max_iter=60, guard_B=0.0, method=2,
                    guess=0.0,
                    desc="robertson k=(0.04,3e7,1e4) y0=(1,0,0) on [0,500], backward Euler h=1e-4 N=5e6, "
                         "plain Newton from the zero guess (Sec. 4.2), preconditioned residual")
    if name == "robertson_mixed":
        return dict(kind="single", wl=W.robertson(h=1e-4), tol=1e-8, max_iter=60, guard_B=0.0, method=2,
                    precision=2, guess=0.0,
                    desc="robertson k=(0.04,3e7,1e4) y0=(1,0,0) on [0,500], backward Euler h=1e-4 N=5e6, "
                         "plain Newton from the zero guess (Sec. 4.2), preconditioned residual; scan in FP32 "
                         "delta form (inexact Newton), FP64 residual, inverse and update")
    if name == "robertson_ff":
        return dict(kind="single", wl=W.robertson(h=1e-4), tol=1e-8, max_iter=60, guard_B=0.0, method=2,
                    precision=3, guess=0.0,
                    desc="robertson k=(0.04,3e7,1e4) y0=(1,0,0) on [0,500], backward Euler h=1e-4 N=5e6, "
                         "plain Newton from the zero guess (Sec. 4.2), preconditioned residual; scan in "
                         "double-FP32 (float-float), FP64 residual, inverse and update")
    if name == "fkpp":
        return dict(kind="single", wl=W.fkpp(), tol=1e-8, max_iter=50, guard_B=0.0, precision=0,
                    desc="fisher_kpp MOL d=128 D=1e-3 h=5e-5 N=2^15, plain Newton, FP64 scan")
    if name == "fkpp_mixed":
        return dict(kind="single", wl=W.fkpp(), tol=1e-8, max_iter=50, guard_B=0.0, precision=1,
                    desc="fisher_kpp MOL d=128 D=1e-3 h=5e-5 N=2^15, plain Newton, BF16 tensor-core "
                         "composes (FP32 accumulate), FP64 residual and update")
    if name == "fkpp_tf32":
        return dict(kind="single", wl=W.fkpp(), tol=1e-8, max_iter=50, guard_B=0.0, precision=4,
                    desc="fisher_kpp MOL d=128 D=1e-3 h=5e-5 N=2^15, plain Newton, TF32 tensor-core "
                         "composes (FP32 accumulate), FP64 residual and update")
    if name == "batch":
        return dict(kind="batch", bt=W.lorenz_batch(), tol=1e-8, max_iter=50, guard_B=100.0,
                    desc="4096 lorenz63 IVPs (seed 0; sigma~U[8,12], rho~U[20,35], beta~U[2,3], "
                         "x0~N(0,25I)), h=1e-3, N_i~U{2^10..2^16}, guarded Newton B=100, max_iter 50")
    if name == "batch_small":
        return dict(kind="batch", bt=W.lorenz_batch(n_max=1 << 13), tol=1e-8, max_iter=100, guard_B=100.0,
                    desc="4096 lorenz63 IVPs (seed 0), h=1e-3, N_i~U{2^10..2^13}, guarded Newton B=100, "
                         "max_iter 100")
    if name == "adjoint":
        return dict(kind="adjoint", bt=W.vdp_adjoint_batch(), tol=1e-10, max_iter=200, guard_B=100.0,
                    desc="256 van_der_pol IVPs (seed 0; mu~U[0.5,2], x0~U[-2,2]^2), h=1e-3, N=2^14: "
                         "batched Newton forward (guarded B=100, tol 1e-10) + adjoint reverse scan "
                         "(checkpoint every 1024 steps), loss sum ||x_N - (1,0)||^2")
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling every 200 ms from before the warm-up steps to the
    end of the timed region.  The median SM clock and the throttle reasons
    are those of the samples stamped inside the timed region; a timed region
    shorter than the sampling interval may hold none, and then the samples
    of the warm-up steps and the timed region are reported, marked so."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None
        self.t_timed = None

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

    def timed(self):
        """Marks the start of the timed region."""
        self.t_timed = datetime.datetime.now()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        t_end = datetime.datetime.now()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        run, timed = [], []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
                smp = (float(f[2]), float(f[3]), {n for n, v in zip(names, f[6:10]) if v.lower() == "active"})
            except ValueError:
                continue
            if ts > t_end:
                continue
            run.append(smp)
            if self.t_timed is not None and ts >= self.t_timed:
                timed.append(smp)
        use = timed or run
        if not use:
            return None
        return {"sm_mhz": statistics.median(x[0] for x in use), "sm_max_mhz": max(x[1] for x in use),
                "reasons": sorted(set().union(*(x[2] for x in use))), "samples": len(use),
                "window": "timed region" if timed else
                          "warm-up and timed region (no sample fell inside the shorter timed region)"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def gpu_uuid(dev, local_rank):
    """The nvidia-smi id of a torch device (its UUID; the local rank if the
    UUID is not available)."""
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return str(local_rank)


def batch_kernel_name(shape):
    """The batch solver's timed kernel for a (threads per CTA, steps per
    thread) launch shape: steps per thread 0 is the per-IVP path."""
    if shape is None:
        return "batch solve (untuned default launch shape)"
    if shape[1] == 0:
        return f"batch_ivp_kernel (persistent {shape[0]}-thread CTAs, one IVP each, longest first)"
    return "batch solve graph (conditional while loop over fold, decide, replay, end)"


def run_ours_batch(args, rank, world, local_rank, spec):
    import torch
    import paper_2511_01465_gb300 as pk
    from paper_2511_01465_gb300 import pitn as P

    from paper_2511_01465_gb300 import dist as D

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    bt_full = spec["bt"]
    # independent IVPs: each rank solves its contiguous share, no data-path collective
    bt, _ = D.shard_batch(bt_full, rank, world)
    stream = torch.cuda.current_stream(dev)
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=dev)
    params, x0, h, N = t(bt.params), t(bt.x0), t(bt.h), t(bt.N, torch.int64)
    M, d = int(bt.N.sum()), bt.d
    traj = torch.empty((M, d), dtype=torch.float64, device=dev)
    offs = torch.empty(bt.B + 1, dtype=torch.int64, device=dev)
    iters = torch.empty(bt.B, dtype=torch.int32, device=dev)
    status = torch.empty(bt.B, dtype=torch.int32, device=dev)
    res = torch.empty(bt.B, dtype=torch.float64, device=dev)
    opt = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream)

    def solve_once():
        rc = P.pitn_solve_batch(bt.system, bt.B, params, x0, h, N, d, spec["tol"], spec["max_iter"],
                                traj, offs, iters, status, res, opt)
        P.check(rc, "pitn_solve_batch")

    clocks = ClockSampler(gpu_uuid(dev, local_rank))
    clocks.start()
    P.pitn_tune_enable(not args.no_tune)
    for _ in range(args.warmup):
        solve_once()
    P.pitn_tune_enable(False)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks.timed()
    launches0 = pk.pitn_launch_count()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solve_once()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = pk.pitn_launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    # per-iteration device times from separate, instrumented solves
    nk = min(args.steps, 3)
    P.pitn_timing_reset()
    P.pitn_timing_enable(True)
    for _ in range(nk):
        solve_once()
    torch.cuda.synchronize(dev)
    P.pitn_timing_enable(False)
    kms, kl = P.pitn_timing_get("batch")
    st_h, it_h, res_h = status.cpu().numpy(), iters.cpu().numpy(), res.cpu().numpy()
    ok = (st_h == P.PITN_OK) & (res_h <= spec["tol"])
    solved, total_ms = D.aggregate(int(bt.N[ok].sum()), float(sum(times)))
    ms_per_step = total_ms / args.steps
    value = solved / (ms_per_step / 1e3)
    # FP64 flops of the steps actually evaluated and replayed (counted by the
    # kernels, pitn_batch_work), per step as counted from the kernel source
    p1, p3 = SMALL_FLOPS["lorenz"]
    n_ev, n_rep = P.pitn_batch_work()
    flops = float(n_ev * p1 + n_rep * p3)
    achieved = flops / (kms / 1e3 / nk) / 1e12 if kms > 0 else 0.0
    shape = P.pitn_tune_get(f"batch:{bt.system}:{d}:{M.bit_length() - 1}:{1 if spec['guard_B'] > 0 else 0}")
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak(), "unit": "TFLOP/s",
                "frac": achieved / fp64_peak(), "traffic": None,
                "kernel": batch_kernel_name(shape),
                "kernel_launches_per_step": kl / nk, "kernel_ms_per_launch": kms / max(kl, 1),
                "steps_evaluated": n_ev, "steps_replayed": n_rep,
                "note": f"FP64 flops of the steps evaluated ({p1:g} each) and replayed ({p3:g} each), "
                        "counted by the kernels (a guard's fill region is folded by powering one "
                        "element); peak = measured DFMA rate x 2"}
    # the same IVPs solved one at a time by the single-IVP GPU solver (a sample)
    single = None
    if rank == 0:
        n_s = min(64, bt.B)
        so = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream)
        tr1 = torch.empty((int(bt.N[:n_s].max()), d), dtype=torch.float64, device=dev)
        ps = [t(bt.params[b]) for b in range(n_s)]
        xs = [t(bt.x0[b]) for b in range(n_s)]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        solved1 = 0
        for b in range(n_s):
            rc1, r1 = P.pitn_solve_ex(bt.system, ps[b], xs[b], float(bt.h[b]), int(bt.N[b]), d, spec["tol"],
                                      spec["max_iter"], tr1, so)
            if r1.status == P.PITN_OK and r1.final_res <= spec["tol"]:
                solved1 += int(bt.N[b])
        torch.cuda.synchronize(dev)
        dt1 = time.perf_counter() - t0
        single = {"value": solved1 / dt1, "unit": UNIT,
                  "sample": f"first {n_s} IVPs, one pitn_solve_ex call each ({dt1 * 1e3:.1f} ms)"}
    # ---- end to end through the C ABI with pinned host buffers ----
    pin = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt).pin_memory()
    hp, hx, hh, hN = (pin(bt.params).numpy(), pin(bt.x0).numpy(), pin(bt.h).numpy(),
                      pin(bt.N, torch.int64).numpy())
    htraj = torch.empty((M, d), dtype=torch.float64).pin_memory().numpy()
    hoffs = torch.empty(bt.B + 1, dtype=torch.int64).pin_memory().numpy()
    hit = torch.empty(bt.B, dtype=torch.int32).pin_memory().numpy()
    hst = torch.empty(bt.B, dtype=torch.int32).pin_memory().numpy()
    hres = torch.empty(bt.B, dtype=torch.float64).pin_memory().numpy()

    def solve_host():
        P.check(P.pitn_solve_batch(bt.system, bt.B, hp, hx, hh, hN, d, spec["tol"], spec["max_iter"],
                                   htraj, hoffs, hit, hst, hres, opt), "pitn_solve_batch")

    solve_host()
    et = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        solve_host()
        et.append(time.perf_counter() - t0)
    e2e_s = statistics.median(et)
    ok_h = (hst == P.PITN_OK) & (hres <= spec["tol"])
    solved_e, e2e_max = D.aggregate(int(bt.N[ok_h].sum()), e2e_s)
    e2e = {"value": solved_e / e2e_max, "unit": UNIT,
           "h2d_bytes_per_step": int(hp.nbytes + hx.nbytes + hh.nbytes + hN.nbytes),
           "d2h_bytes_per_step": int(htraj.nbytes + hoffs.nbytes + hit.nbytes + hst.nbytes + hres.nbytes),
           "ms_per_step": e2e_max * 1e3}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "single_ivp_gpu_solver": single,
            "config": {"workload": spec["desc"], "B": bt.B, "sum_N": M, "d": d, "tol": spec["tol"],
                       "max_iter": spec["max_iter"], "converged_ivps": int(ok.sum()),
                       "converged_steps": int(solved), "not_converged_ivps": int((st_h == 1).sum()),
                       "nonfinite_ivps": int((st_h == 2).sum()),
                       "mean_newton_updates": float(it_h.mean()),
                       "step_ms": [round(x, 3) for x in times],
                       "l2": "inputs (>3 GB per trajectory buffer) larger than L2",
                       "launch_shape": shape,
                       "parallelism": f"IVP shards x{world}"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}
    if world == 1 and not args.no_companions:
        # the same batch with the reduced-precision scans (per-IVP path), timed
        # the same way; only the steps of IVPs that reach the FP64 tolerance count
        line["mixed"] = {}
        for key, prec in (("fp32_scan", P.PITN_PREC_MIXED_FP32), ("float_float_scan", P.PITN_PREC_FP64_FF)):
            mo = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream, precision=prec)

            def solve_mixed():
                P.check(P.pitn_solve_batch(bt.system, bt.B, params, x0, h, N, d, spec["tol"], spec["max_iter"],
                                           traj, offs, iters, status, res, mo), "pitn_solve_batch")

            P.pitn_tune_enable(not args.no_tune)
            for _ in range(args.warmup):
                solve_mixed()
            P.pitn_tune_enable(False)
            mt = []
            for _ in range(args.steps):
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                solve_mixed()
                e1.record(stream)
                e1.synchronize()
                mt.append(e0.elapsed_time(e1))
            st_m, it_m, res_m = status.cpu().numpy(), iters.cpu().numpy(), res.cpu().numpy()
            ok_m = (st_m == P.PITN_OK) & (res_m <= spec["tol"])
            ms_m = float(sum(mt)) / len(mt)
            v_m = float(bt.N[ok_m].sum()) / (ms_m / 1e3)
            line["mixed"][key] = {"value": v_m, "unit": UNIT, "ms_per_step": ms_m,
                                  "vs_fp64": v_m / value if value > 0 else None,
                                  "converged_ivps": int(ok_m.sum()), "converged_steps": int(bt.N[ok_m].sum()),
                                  "mean_newton_updates": float(it_m.mean()),
                                  "steps_evaluated": P.pitn_batch_work()[0],
                                  "launch_shape": P.pitn_tune_get(
                                      f"batch:{bt.system}:{d}:{M.bit_length() - 1}:"
                                      f"{1 if spec['guard_B'] > 0 else 0}:{'f32' if prec == 2 else 'ff'}")}
    return line


def run_ours_adjoint(args, rank, world, local_rank, spec):
    import torch
    import paper_2511_01465_gb300 as pk
    from paper_2511_01465_gb300 import pitn as P

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    bt = spec["bt"]
    stream = torch.cuda.current_stream(dev)
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=dev)
    params, x0, h, N = t(bt.params), t(bt.x0), t(bt.h), t(bt.N, torch.int64)
    M, d = int(bt.N.sum()), bt.d
    traj = torch.empty((M, d), dtype=torch.float64, device=dev)
    offs = torch.empty(bt.B + 1, dtype=torch.int64, device=dev)
    iters = torch.empty(bt.B, dtype=torch.int32, device=dev)
    status = torch.empty(bt.B, dtype=torch.int32, device=dev)
    res = torch.empty(bt.B, dtype=torch.float64, device=dev)
    gx0 = torch.empty((bt.B, d), dtype=torch.float64, device=dev)
    gp = torch.empty((bt.B, bt.params.shape[1]), dtype=torch.float64, device=dev)
    target = t([1.0, 0.0])
    opt = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream)

    def step():
        rc = P.pitn_solve_batch(bt.system, bt.B, params, x0, h, N, d, spec["tol"], spec["max_iter"],
                                traj, offs, iters, status, res, opt)
        P.check(rc, "pitn_solve_batch")
        last = offs[1:] - 1
        gN = (2.0 * (traj[last] - target)).contiguous()
        P.check(P.pitn_backward(bt.system, bt.B, params, x0, h, N, d, traj, None, gN, 1024, gx0, gp, opt),
                "pitn_backward")

    clocks = ClockSampler(gpu_uuid(dev, local_rank))
    clocks.start()
    P.pitn_tune_enable(not args.no_tune)
    for _ in range(args.warmup):
        step()
    P.pitn_tune_enable(False)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks.timed()
    launches0 = pk.pitn_launch_count()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = pk.pitn_launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    # forward / adjoint device times from separate, instrumented steps
    nk = min(args.steps, 3)
    P.pitn_timing_reset()
    P.pitn_timing_enable(True)
    for _ in range(nk):
        step()
    torch.cuda.synchronize(dev)
    P.pitn_timing_enable(False)

    # ---- end to end through the C ABI with pinned host buffers: forward solve,
    # loss gradient on the host, adjoint ----
    pin = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt).pin_memory()
    hp, hx, hh, hN = (pin(bt.params).numpy(), pin(bt.x0).numpy(), pin(bt.h).numpy(),
                      pin(bt.N, torch.int64).numpy())
    htraj = torch.empty((M, d), dtype=torch.float64).pin_memory().numpy()
    hoffs = torch.empty(bt.B + 1, dtype=torch.int64).pin_memory().numpy()
    hit = torch.empty(bt.B, dtype=torch.int32).pin_memory().numpy()
    hst = torch.empty(bt.B, dtype=torch.int32).pin_memory().numpy()
    hres = torch.empty(bt.B, dtype=torch.float64).pin_memory().numpy()
    hgN = torch.empty((bt.B, d), dtype=torch.float64).pin_memory().numpy()
    hgx0 = torch.empty((bt.B, d), dtype=torch.float64).pin_memory().numpy()
    hgp = torch.empty((bt.B, bt.params.shape[1]), dtype=torch.float64).pin_memory().numpy()

    def step_host():
        P.check(P.pitn_solve_batch(bt.system, bt.B, hp, hx, hh, hN, d, spec["tol"], spec["max_iter"],
                                   htraj, hoffs, hit, hst, hres, opt), "pitn_solve_batch")
        hgN[:] = 2.0 * (htraj[hoffs[1:] - 1] - np.array([1.0, 0.0]))
        P.check(P.pitn_backward(bt.system, bt.B, hp, hx, hh, hN, d, htraj, None, hgN, 1024, hgx0, hgp, opt),
                "pitn_backward")

    step_host()
    et = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        step_host()
        et.append(time.perf_counter() - t0)
    e2e_s = statistics.median(et)
    e2e = {"value": float(bt.N[hst == P.PITN_OK].sum()) / e2e_s * world, "unit": UNIT,
           "h2d_bytes_per_step": int(2 * (hp.nbytes + hx.nbytes + hh.nbytes + hN.nbytes) + htraj.nbytes
                                     + hgN.nbytes),
           "d2h_bytes_per_step": int(htraj.nbytes + hoffs.nbytes + hit.nbytes + hst.nbytes + hres.nbytes
                                     + hgx0.nbytes + hgp.nbytes),
           "ms_per_step": e2e_s * 1e3}
    fwd_ms, fwd_n = P.pitn_timing_get("batch")
    adj_ms, adj_n = P.pitn_timing_get("adjoint")
    ms_per_step = float(sum(times)) / args.steps
    st_h, it_h = status.cpu().numpy(), iters.cpu().numpy()
    ok = st_h == P.PITN_OK
    value = float(bt.N[ok].sum()) / (ms_per_step / 1e3)
    p1, p3 = SMALL_FLOPS["vdp"]
    n_ev, n_rep = P.pitn_batch_work()   # of the last forward solve
    flops = float(n_ev * p1 + n_rep * p3)
    ach = flops / (fwd_ms / 1e3 / nk) / 1e12 if fwd_ms > 0 else 0.0
    shape = P.pitn_tune_get(f"batch:{bt.system}:{d}:{M.bit_length() - 1}:{1 if spec['guard_B'] > 0 else 0}")
    roofline = {"bound": "alu", "achieved": ach, "peak": fp64_peak(), "unit": "TFLOP/s",
                "frac": ach / fp64_peak(), "traffic": None,
                "kernel": "forward solve: " + batch_kernel_name(shape),
                "kernel_launches_per_step": fwd_n / nk, "kernel_ms_per_launch": fwd_ms / max(fwd_n, 1),
                "steps_evaluated": n_ev, "steps_replayed": n_rep,
                "note": "FP64 flops of the forward solve's steps evaluated and replayed (counted by "
                        "the kernels), per step counted from the kernel source; peak = measured DFMA "
                        "rate x 2"}
    mixed = None
    if world == 1 and not args.no_companions:
        # the same step with the forward solve's scan in FP32 or float-float (the
        # adjoint stays FP64); the gradients against the FP64 step's
        gp_ref, gx_ref = gp.clone(), gx0.clone()
        mixed = {}
        for key, prec in (("fp32_scan", P.PITN_PREC_MIXED_FP32), ("float_float_scan", P.PITN_PREC_FP64_FF)):
            mo = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream, precision=prec)

            def step_m():
                P.check(P.pitn_solve_batch(bt.system, bt.B, params, x0, h, N, d, spec["tol"], spec["max_iter"],
                                           traj, offs, iters, status, res, mo), "pitn_solve_batch")
                gNm = (2.0 * (traj[offs[1:] - 1] - target)).contiguous()
                P.check(P.pitn_backward(bt.system, bt.B, params, x0, h, N, d, traj, None, gNm, 1024, gx0, gp,
                                        opt), "pitn_backward")

            P.pitn_tune_enable(not args.no_tune)
            for _ in range(args.warmup):
                step_m()
            P.pitn_tune_enable(False)
            mt = []
            for _ in range(args.steps):
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step_m()
                e1.record(stream)
                e1.synchronize()
                mt.append(e0.elapsed_time(e1))
            ok_m = status.cpu().numpy() == P.PITN_OK
            ms_m = float(sum(mt)) / len(mt)
            v_m = float(bt.N[ok_m].sum()) / (ms_m / 1e3)
            rel = lambda a, b: float((a - b).abs().max() / b.abs().max())
            mixed[key] = {"value": v_m, "unit": UNIT, "ms_per_step": ms_m,
                          "vs_fp64": v_m / value if value > 0 else None, "converged_ivps": int(ok_m.sum()),
                          "grad_params_rel_diff": rel(gp, gp_ref), "grad_x0_rel_diff": rel(gx0, gx_ref)}
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "mixed": mixed,
            "config": {"workload": spec["desc"], "B": bt.B, "sum_N": M, "d": d, "tol": spec["tol"],
                       "converged_ivps": int(ok.sum()), "mean_newton_updates": float(it_h.mean()),
                       "forward_ms_per_step": fwd_ms / nk, "launch_shape": shape,
                       "adjoint_ms_per_step": adj_ms / nk,
                       "step_ms": [round(x, 3) for x in times], "parallelism": f"replicas x{world}"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}


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
    prec = spec.get("precision", 0)
    method = spec.get("method", 0)
    guess = None
    if "guess" in spec:  # constant initial guess, copied into the trajectory by every solve
        guess = torch.full((wl.N, wl.d), spec["guess"], dtype=torch.float64, device=dev)
    opt = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream, precision=prec, guess=guess,
                         method=method)

    def solve_once():
        rc, res = P.pitn_solve_ex(wl.system, params, x0, wl.h, wl.N, wl.d, spec["tol"],
                                  spec["max_iter"], traj, opt)
        P.check(rc, "pitn_solve_ex")
        return rc, res

    clocks = ClockSampler(gpu_uuid(dev, local_rank))
    clocks.start()
    P.pitn_tune_enable(not args.no_tune)  # the first warm-up solve picks the launch shape
    for _ in range(args.warmup):
        rc, res = solve_once()
    P.pitn_tune_enable(False)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)

    clocks.timed()
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
    # per-kernel device times from separate solves: the library's event pairs
    # around each launch would add to the timed steps of many-launch solves
    nk = min(args.steps, 3)
    P.pitn_timing_reset()
    P.pitn_timing_enable(True)
    for _ in range(nk):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        solve_once()
    torch.cuda.synchronize(dev)
    P.pitn_timing_enable(False)
    ktimes = {k: P.pitn_timing_get(k) for k in
              ("newton_small", "fkpp_residual", "fkpp_fold", "fkpp_compose", "fkpp_down", "fkpp_replay")}
    ktimes = {k: v for k, v in ktimes.items() if v[1] > 0}
    total_ms = float(sum(times))
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    converged = res.status == P.PITN_OK and res.final_res <= spec["tol"]
    steps_solved = wl.N if converged else 0
    value = world * steps_solved / (ms_per_step / 1e3)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if True:
        h_params = torch.tensor(wl.params, dtype=torch.float64).pin_memory()
        h_x0 = torch.tensor(wl.x0, dtype=torch.float64).pin_memory()
        h_traj = torch.empty((wl.N, wl.d), dtype=torch.float64).pin_memory()
        hp, hx, ht = h_params.numpy(), h_x0.numpy(), h_traj.numpy()
        h_guess = None
        if guess is not None:
            h_guess = torch.full((wl.N, wl.d), spec["guess"], dtype=torch.float64).pin_memory().numpy()
        opt_h = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream, precision=prec,
                               guess=h_guess, method=method)
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
        e2e_ok = r2.status == P.PITN_OK and r2.final_res <= spec["tol"]
        e2e = {"value": (world * wl.N / e2e_s) if e2e_ok else 0.0, "unit": UNIT,
               "h2d_bytes_per_step": int((wl.d + len(wl.params)) * 8 +
                                         (wl.N * wl.d * 8 if h_guess is not None else 0)),
               "d2h_bytes_per_step": int(wl.N * wl.d * 8), "ms_per_step": e2e_s * 1e3}

    roofline = roofline_for(args.workload, spec, wl, res, ktimes, nk)
    tkey = (f"small:{wl.system}:{wl.d}:{wl.N.bit_length() - 1}:{1 if spec['guard_B'] > 0 else 0}"
            f"{ {1: ':rk4', 2: ':be', 3: ':tr'}.get(method, '')}{ {2: ':f32', 3: ':ff'}.get(prec, '')}")
    launch_shape = P.pitn_tune_get(tkey)   # (threads per CTA, CTAs per SM), + min steps per thread
    if launch_shape is not None:
        cm = P.pitn_tune_get(tkey + ":c")
        launch_shape = list(launch_shape) + ([cm[0]] if cm is not None else [])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec["desc"], "N": wl.N, "d": wl.d, "tol": spec["tol"],
                       "max_iter": spec["max_iter"], "newton_updates": res.iters,
                       "status": P.pitn_status_string(res.status), "final_res": res.final_res,
                       "l2": "flushed (512 MiB write) between timed steps",
                       "step_ms": [round(t, 3) for t in times],
                       "launch_shape": launch_shape,
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "kernel_ms_per_step": {k: v[0] / nk for k, v in ktimes.items()}}
    if args.workload in TWINS and not args.no_companions and world == 1:
        # the metric's comparison: reduced-precision scans (and, on the default
        # line, batching) against the plain FP64 solver, same tolerance, timed
        # after the FP64 line (on one GPU: with several, the replicas' line
        # carries no comparison)
        f32, ffw = TWINS[args.workload]
        line["mixed"] = {
            "fp32_scan": companion_single(args, f32, dev, stream, flush, value, traj),
            "float_float_scan": companion_single(args, ffw, dev, stream, flush, value, traj),
        }
        if args.workload == "vdp":
            line["batched"] = companion_batched(args, dev, stream)
    return line


# FP64 workloads and their FP32-scan and float-float twins (same problem,
# tolerance and iteration limit)
TWINS = {"vdp": ("vdp_mixed", "vdp_ff"), "lorenz": ("lorenz_mixed", "lorenz_ff"),
         "vdp_rk4": ("vdp_rk4_mixed", "vdp_rk4_ff"), "robertson": ("robertson_mixed", "robertson_ff")}


def companion_single(args, name, dev, stream, flush, ref_value, ref_traj):
    """The same metric for another precision of the same workload (same
    tolerance, same timing rules), with its ratio to the FP64 line's value
    and its largest difference from the FP64 solve's trajectory."""
    import torch
    from paper_2511_01465_gb300 import pitn as P
    spec = workload(name)
    wl = spec["wl"]
    params = torch.tensor(wl.params, dtype=torch.float64, device=dev)
    x0 = torch.tensor(wl.x0, dtype=torch.float64, device=dev)
    traj = torch.empty((wl.N, wl.d), dtype=torch.float64, device=dev)
    guess = None
    if "guess" in spec:  # constant initial guess, copied into the trajectory by every solve
        guess = torch.full((wl.N, wl.d), spec["guess"], dtype=torch.float64, device=dev)
    opt = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream, precision=spec["precision"],
                         guess=guess, method=spec.get("method", 0))

    def solve_once():
        rc, res = P.pitn_solve_ex(wl.system, params, x0, wl.h, wl.N, wl.d, spec["tol"], spec["max_iter"],
                                  traj, opt)
        P.check(rc, "pitn_solve_ex")
        return res

    P.pitn_tune_enable(not args.no_tune)
    for _ in range(args.warmup):
        res = solve_once()
    P.pitn_tune_enable(False)
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        res = solve_once()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(sum(times)) / args.steps
    ok = res.status == P.PITN_OK and res.final_res <= spec["tol"]
    value = (wl.N if ok else 0) / (ms / 1e3)
    diff = float((traj - ref_traj).abs().max() / ref_traj.abs().max())
    return {"workload": spec["desc"], "value": value, "unit": UNIT, "ms_per_step": ms,
            "newton_updates": res.iters, "status": P.pitn_status_string(res.status), "final_res": res.final_res,
            "ratio_vs_fp64": value / ref_value if ref_value > 0 else None,
            "max_rel_diff_vs_fp64_solve": diff}


def companion_batched(args, dev, stream):
    """Batching against the plain solver: the 4096-IVP Lorenz batch
    (lengths 2^10..2^13) in one batched solve, against its first 64 IVPs
    solved one pitn_solve_ex call at a time, both at tol 1e-8."""
    import torch
    from paper_2511_01465_gb300 import pitn as P
    spec = workload("batch_small")
    bt = spec["bt"]
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device=dev)
    params, x0, h, N = t(bt.params), t(bt.x0), t(bt.h), t(bt.N, torch.int64)
    M, d = int(bt.N.sum()), bt.d
    traj = torch.empty((M, d), dtype=torch.float64, device=dev)
    offs = torch.empty(bt.B + 1, dtype=torch.int64, device=dev)
    iters = torch.empty(bt.B, dtype=torch.int32, device=dev)
    status = torch.empty(bt.B, dtype=torch.int32, device=dev)
    res = torch.empty(bt.B, dtype=torch.float64, device=dev)
    opt = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream)

    def solve_once():
        P.check(P.pitn_solve_batch(bt.system, bt.B, params, x0, h, N, d, spec["tol"], spec["max_iter"],
                                   traj, offs, iters, status, res, opt), "pitn_solve_batch")

    P.pitn_tune_enable(not args.no_tune)
    solve_once()
    P.pitn_tune_enable(False)
    solve_once()
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solve_once()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    st_h, res_h = status.cpu().numpy(), res.cpu().numpy()
    ok = (st_h == P.PITN_OK) & (res_h <= spec["tol"])
    batched = float(bt.N[ok].sum()) / (ms / 1e3)
    n_s = 64
    so = P.make_options(guard_B=spec["guard_B"], stream=stream.cuda_stream)
    tr1 = torch.empty((int(bt.N[:n_s].max()), d), dtype=torch.float64, device=dev)
    ps = [t(bt.params[b]) for b in range(n_s)]
    xs = [t(bt.x0[b]) for b in range(n_s)]
    P.pitn_solve_ex(bt.system, ps[0], xs[0], float(bt.h[0]), int(bt.N[0]), d, spec["tol"], spec["max_iter"],
                    tr1, so)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    solved1 = 0
    for b in range(n_s):
        _, r1 = P.pitn_solve_ex(bt.system, ps[b], xs[b], float(bt.h[b]), int(bt.N[b]), d, spec["tol"],
                                spec["max_iter"], tr1, so)
        if r1.status == P.PITN_OK and r1.final_res <= spec["tol"]:
            solved1 += int(bt.N[b])
    torch.cuda.synchronize(dev)
    one = solved1 / (time.perf_counter() - t0)
    return {"workload": spec["desc"], "value": batched, "unit": UNIT, "ms_per_step": ms,
            "converged_ivps": int(ok.sum()),
            "one_at_a_time": {"value": one, "unit": UNIT,
                              "sample": f"first {n_s} IVPs, one pitn_solve_ex call each (host clock)"},
            "ratio_vs_one_at_a_time": batched / one if one > 0 else None}


def fk_tiles(N, sms=152, per_sm=1):
    """Tiles of the FKPP scan, as the library picks them: 64 steps, shortened
    once there is a full wave so that the count is a whole number of waves of
    the fold (one 1024-thread FP32 or 512-thread FP64 CTA per SM)."""
    ts = 64
    t0 = (N - 1 + 63) // 64
    slots = sms * per_sm
    if t0 >= slots:
        tw = (t0 + slots - 1) // slots * slots
        ts = (N - 1 + tw - 1) // tw
    return max(1, (N - 1 + ts - 1) // ts)


def fk_composes(T):
    """Dense composes of one up-sweep over T tiles: every level below the root
    pairs its nodes (a lone last node is copied); the root is not composed."""
    n, total = T, 0
    while n > 2:
        total += n // 2
        n = (n + 1) // 2
    return total


def roofline_for(name, spec, wl, res, ktimes, steps):
    """Roofline of the kernel family with the largest device time."""
    kern = max(ktimes, key=lambda k: ktimes[k][0])
    extra = {}
    ms, launches = ktimes[kern]
    passes = res.iters + 1
    per_step_s = ms / 1e3 / steps
    if kern == "newton_small":
        # FP64-pipe bound (ncu: the FP64 pipe is the busiest unit of every
        # small-state kernel); flops counted from the source (FMA = 2) against
        # the measured DFMA rate, the FP64 instruction issue (DADD, DMUL, DFMA
        # one slot each) as the pipe's fraction, and the algorithmic bytes
        # (state read and written once per pass) against the measured copy
        # bandwidth
        hbm, _, _, src = load_peaks()
        if name in REDUCED_FP64:
            ops, fl = REDUCED_FP64[name]
            flops = wl.N * fl * passes
            fp64_ops = wl.N * ops * passes
            note = ("FP64 work of the reduced-precision scan: residual and update per step and pass "
                    f"({ops:g} instructions, {fl:g} flops); the scan itself runs on the FP32 pipe")
        else:
            p1, p3 = SMALL_FLOPS[name]
            flops = wl.N * (p1 * passes + p3 * res.iters)
            o = FP64_OPS.get(name)
            fp64_ops = wl.N * (o[0] * passes + o[1] * res.iters) if o else None
            note = "FP64 flops per step counted from the kernel source (phase 1 every pass, phase 3 per update)"
        achieved = flops / per_step_s / 1e12
        alg = wl.N * small_alg_bytes(wl.d) * passes
        out = {"bound": "alu", "achieved": achieved, "peak": fp64_peak(), "unit": "TFLOP/s",
               "frac": achieved / fp64_peak(), "traffic": traffic_for(name), "kernel": kern,
               "kernel_launches_per_step": launches / steps, "kernel_ms_per_launch": ms / max(launches, 1),
               "peak_source": PEAKS["source"] + " (DFMA rate x 2)",
               "hbm_achieved_gbs": alg / per_step_s / 1e9, "hbm_peak_gbs": hbm,
               "hbm_frac": alg / per_step_s / 1e9 / hbm,
               "hbm_note": f"algorithmic bytes {small_alg_bytes(wl.d)} B per step and pass (x read and written "
                           f"once) against the {src} copy bandwidth",
               "note": note}
        if fp64_ops:
            out["fp64_pipe_frac"] = fp64_ops / per_step_s / (fp64_peak() / 2 * 1e12)
        return out
    elif kern == "fkpp_residual":
        flops = wl.N * passes * 128 * 15
        peak, bound, unit = fp64_peak(), "alu", "TFLOP/s"
        note = "FP64 residual flops (15 per entry); peak = measured DFMA rate x 2"
    elif kern == "fkpp_fold":
        # the scan runs once per Newton update (a converged pass stops after its residual)
        mixed = spec.get("precision", 0) in (1, 4)
        flops = wl.N * res.iters * FK_FOLD_REAL_FLOPS
        peak = fp32_peak() if mixed else fp64_peak()
        bound, unit = "alu", "TFLOP/s"
        note = ("dense fold flops in " + ("FP32" if mixed else "FP64") +
                "; peak = measured " + ("FFMA" if mixed else "DFMA") + " rate x 2")
    elif kern == "fkpp_compose":
        mixed = spec.get("precision", 0) in (1, 4)
        flops = fk_composes(fk_tiles(wl.N)) * FK_COMPOSE_FLOPS * res.iters
        if mixed and spec.get("precision") == 4:
            _, bf16, _, src = load_peaks()
            peak, bound, unit = bf16 * 1.1 / 2.25, "tensor", "TFLOP/s"
            note = (f"TF32 tensor-core composes; peak = {src} cuBLAS bf16 burst x 1.1/2.25 "
                    "(nominal dense TF32 / BF16)")
        elif mixed:
            _, bf16, _, src = load_peaks()
            peak, bound, unit = bf16, "tensor", "TFLOP/s"
            note = f"BF16 tensor-core composes; peak = {src} cuBLAS bf16 burst"
        else:
            peak, bound, unit = fp64_peak(), "alu", "TFLOP/s"
            note = "FP64 CUDA-core composes; peak = measured DFMA rate x 2"
    else:
        hbm, _, _, src = load_peaks()
        flops = None
        peak, bound, unit = hbm, "hbm", "GB/s"
        note = "memory-bound helper"
    achieved = (flops / per_step_s / 1e12) if flops is not None else 0.0
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic_for(name) if kern == "newton_small" else None,
            **extra, "kernel": kern,
            "kernel_launches_per_step": launches / steps,
            "kernel_ms_per_launch": ms / max(launches, 1), "note": note}


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(spec, sample_iters):
    """Times the oracle's Newton solve on the full workload for a bounded number
    of Newton iterations and projects to the full solve's residual count."""
    import oracle as O
    wl = spec["wl"]
    guess = np.full((wl.N, wl.d), spec["guess"]) if "guess" in spec else None
    t0 = time.perf_counter()
    r = O.newton(wl.system, wl.params, wl.x0, wl.h, wl.N, spec["tol"], sample_iters,
                 guard_B=spec["guard_B"], guess=guess, method=spec.get("method", O.EULER))
    dt = time.perf_counter() - t0
    evals = r["iters"] + 1
    return dt / evals, r


def oracle_passes(name, fallback):
    """Residual evaluations the oracle's own full solve needs (stored by
    tests/golden/make_oracle_golden.py, which runs only the oracle)."""
    key = {"vdp": "vdp_2^22_guard100_tol1e-8_it400", "osc": "osc_2^22_plain_tol1e-8_it10",
           "vdp_mixed": "vdp_2^22_guard100_tol1e-8_it400", "vdp_ff": "vdp_2^22_guard100_tol1e-8_it400",
           "lorenz_mixed": "lorenz_8192_guard100_tol1e-8_it100", "lorenz_ff": "lorenz_8192_guard100_tol1e-8_it100",
           "lorenz": "lorenz_8192_guard100_tol1e-8_it100",
           "fkpp": "fkpp_d128_2^15_plain_tol1e-8_it50", "fkpp_mixed": "fkpp_d128_2^15_plain_tol1e-8_it50",
           "fkpp_tf32": "fkpp_d128_2^15_plain_tol1e-8_it50",
           "robertson": "robertson_5e6_be_zeros_tol1e-8_it60", "robertson_mixed": "robertson_5e6_be_zeros_tol1e-8_it60",
           "robertson_ff": "robertson_5e6_be_zeros_tol1e-8_it60",
           "vdp_rk4": "vdp_rk4_1e6_ones_tol1e-8_it50",
           "vdp_rk4_ff": "vdp_rk4_1e6_ones_tol1e-8_it50", "vdp_rk4_mixed": "vdp_rk4_1e6_ones_tol1e-8_it50"}
    p = os.path.join(ROOT, "tests", "golden", "oracle_full_size.json")
    try:
        with open(p) as f:
            return json.load(f)[key[name]]["iters"] + 1
    except (OSError, KeyError, ValueError):
        return fallback


CPU_SAMPLE_S = 10.0   # the oracle samples repeat until at least this much CPU time


def cpu_baseline(spec, full_passes, sample_iters):
    wl = spec["wl"]
    total, evals, reps = 0.0, 0, 0
    while total < CPU_SAMPLE_S:
        per_eval, r = oracle_sample(spec, sample_iters)
        total += per_eval * (r["iters"] + 1)
        evals += r["iters"] + 1
        reps += 1
    per_eval = total / evals
    t_full = per_eval * full_passes
    return {"value": wl.N / t_full, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle Newton on the full workload, first {r['iters'] + 1} residual "
                      f"evaluations, {reps} time(s) ({total:.1f} s), projected to the "
                      f"{full_passes} evaluations of the full solve"}


# Newton iterations of the oracle timed per baseline sample (bounded CPU time)
SAMPLE_ITERS = {"vdp": 6, "osc": 1, "lorenz": 62, "fkpp": 3, "fkpp_mixed": 3, "fkpp_tf32": 3, "vdp_mixed": 6, "vdp_ff": 6, "lorenz_ff": 62,
                "lorenz_mixed": 62, "robertson": 9, "robertson_mixed": 9, "robertson_ff": 9, "vdp_rk4": 7, "vdp_rk4_ff": 7,
                "vdp_rk4_mixed": 7}


def cpu_baseline_batch(spec, n_ivps=96):
    """The oracle solving the first n_ivps IVPs of the batch one after another."""
    import oracle as O
    bt = spec["bt"]
    t0 = time.perf_counter()
    solved = 0
    for b in list(range(n_ivps)) * 8:
        if b == 0 and time.perf_counter() - t0 >= CPU_SAMPLE_S:
            break
        r = O.newton(bt.system, bt.params[b], bt.x0[b], bt.h[b], bt.N[b], spec["tol"], spec["max_iter"],
                     guard_B=spec["guard_B"])
        if spec["kind"] == "adjoint":
            O.adjoint(bt.system, bt.params[b], bt.x0[b], bt.h[b], r["traj"],
                      grad_xN=2.0 * (r["traj"][-1] - [1.0, 0.0]))
        if r["status"] == O.OK:
            solved += int(bt.N[b])
    dt = time.perf_counter() - t0
    return {"value": solved / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle Newton{' + adjoint' if spec['kind'] == 'adjoint' else ''} on the first "
                      f"{n_ivps} IVPs of the batch, one after another, repeated to {CPU_SAMPLE_S:g} s "
                      f"or 8 times ({dt:.1f} s)"}


def _oracle_ivp(a):
    """One IVP of a batch through the oracle (a pool worker)."""
    import oracle as O
    system, p, x0, h, N, tol, max_iter, guard_B, adj = a
    r = O.newton(system, p, x0, h, N, tol, max_iter, guard_B=guard_B)
    if adj:
        O.adjoint(system, p, x0, h, r["traj"], grad_xN=2.0 * (r["traj"][-1] - [1.0, 0.0]))
    return int(N) if r["status"] == O.OK else 0


def cpu_baseline_batch_pool(spec, per_core=256):
    """The oracle on every host core, one IVP per task (the batch is a set of
    independent IVPs): the first per_core x cores IVPs of the batch (all of
    them on a 16-core host: about 20 s for the 4096-IVP Lorenz batch)."""
    import multiprocessing as mp
    bt = spec["bt"]
    cores = max(1, min(len(os.sched_getaffinity(0)), 64))
    n = min(bt.B, per_core * cores)
    tasks = [(bt.system, bt.params[b], bt.x0[b], float(bt.h[b]), int(bt.N[b]), spec["tol"],
              spec["max_iter"], spec["guard_B"], spec["kind"] == "adjoint") for b in range(n)]
    with mp.get_context("spawn").Pool(cores) as pool:   # spawn: safe after CUDA initialisation
        pool.map(_oracle_ivp, tasks[:cores], chunksize=1)  # warm the workers (imports, library load)
        solved, dt, reps = 0, 0.0, 0
        while dt < CPU_SAMPLE_S:
            t0 = time.perf_counter()
            solved += sum(pool.map(_oracle_ivp, tasks, chunksize=1))
            dt += time.perf_counter() - t0
            reps += 1
    return {"value": solved / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle Newton{' + adjoint' if spec['kind'] == 'adjoint' else ''} on the first "
                      f"{n} IVPs of the batch, one IVP per task on {cores} host cores, {reps} time(s) "
                      f"({dt:.1f} s)"}


def run_reference(args):
    spec = workload(args.workload)
    if spec["kind"] != "single":
        runs, walls = [], []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            runs.append(cpu_baseline_batch_pool(spec))
            walls.append(time.perf_counter() - t0)
        v = statistics.median(r["value"] for r in runs)
        cb = runs[-1]
        bt = spec["bt"]
        # a step is one bounded sample of the batch (its wall time); value is
        # the sampled rate of solved steps
        return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": spec["desc"], "B": bt.B,
                           "step": "one bounded sample of the batch: " + cb["sample"],
                           "projected_ms_per_solve": float(bt.N.sum()) / v * 1e3 if v > 0 else None},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                 "sample": cb["sample"]},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    wl = spec["wl"]
    import oracle as O
    # number of residual evaluations of the oracle's full solve
    full_passes = oracle_passes(args.workload, 2)
    sample_iters = SAMPLE_ITERS.get(args.workload, 5)
    for _ in range(args.warmup):
        oracle_sample(spec, 0)
    vals, walls = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        per_eval, r = oracle_sample(spec, sample_iters)
        walls.append(time.perf_counter() - t0)
        vals.append(wl.N / (per_eval * full_passes))
    v = statistics.median(vals)
    # a step is a bounded sample of the full workload (its wall time is
    # ms_per_step); value projects the sampled time per residual evaluation
    # to the oracle's own full solve
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": spec["desc"], "N": wl.N, "d": wl.d, "tol": spec["tol"],
                       "step": f"oracle Newton on the full workload, {sample_iters + 1} residual evaluations "
                               f"and {sample_iters} Newton steps",
                       "oracle_residual_evaluations_full_solve": full_passes,
                       "projected_ms_per_solve": wl.N / v * 1e3},
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
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--no-companions", action="store_true",
                    help="vdp: skip the FP32-scan, float-float and batched comparison lines")
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
    torch.cuda.set_device(local_rank)
    peaks = measure_alu_peaks()
    spec0 = workload(args.workload)
    if spec0["kind"] == "batch":
        line = run_ours_batch(args, rank, world, local_rank, spec0)
    elif spec0["kind"] == "adjoint":
        line = run_ours_adjoint(args, rank, world, local_rank, spec0)
    else:
        line = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and spec0["kind"] in ("batch", "adjoint"):
        line["cpu_baseline"] = cpu_baseline_batch_pool(spec0)
        line["cpu_baseline_1core"] = cpu_baseline_batch(spec0)
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        full_passes = oracle_passes(args.workload, line["config"]["newton_updates"] + 1)
        line["cpu_baseline"] = cpu_baseline(workload(args.workload), full_passes,
                                            SAMPLE_ITERS.get(args.workload, 5))
    line["alu_peaks"] = peaks
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
