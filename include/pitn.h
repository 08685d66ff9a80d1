/*
 * pitn.h -- C ABI of the parallel-in-time Newton ODE solver (arXiv 2511.01465)
 * for NVIDIA GB300 (sm_103a).
 *
 * Problem (Sec. 2.1, eq. 2.1):  dx/dt = f(x), x(t0) = x0, discretised by the
 * explicit Euler one-step map phi(x) = x + h f(x) (eq. 2.2) on N steps.
 * The solver finds xi = [x_1 .. x_N] with h(xi) = 0, where
 *     h_n = x_n - phi(x_{n-1}),  n = 1..N                       (eq. 3.8)
 * by Newton's method (eqs. 3.10-3.11).  Each Newton step solves the affine
 * recursion  dx_1 = -h_1,  dx_n = J_{n-1} dx_{n-1} - h_n  (eq. 3.13), with
 * J = dphi/dx, as a parallel prefix scan over the affine elements
 * (J_n, -h_{n+1}) combined by (A2,b2) o (A1,b1) = (A2 A1, A2 b1 + b2)
 * (eq. 3.3; element 1 is the earlier one).  The solve stops when
 * ||h(xi)||_inf <= tol (Sec. 4), when a residual entry is not finite, or
 * after max_iter Newton updates.
 *
 * Conventions shared by every entry point
 *   - Arrays are FP64 (int64/int32 where stated), contiguous, row-major.
 *     A pointer may be device memory of the current CUDA device or host
 *     memory (pageable or pinned); the library detects which with
 *     cudaPointerGetAttributes and stages host arrays through device memory.
 *     All array arguments of one call should live on the same side.  Device
 *     memory of a GPU other than the current one is refused (PITN_EINVAL).
 *   - Ownership: the caller owns every array.  The library never frees or
 *     keeps a pointer after the call returns.  Scratch memory comes from a
 *     per-device cache that grows on demand; pitn_release_workspace frees it.
 *   - Streams: work runs on opt->stream (pitn_solve_ex etc.) or on the
 *     legacy default stream.  Every call blocks until its results are
 *     available on the host (it must read the device status word).
 *   - Errors: every call returns a pitn_status.  Argument errors are detected
 *     on the host before any device work and leave all outputs untouched.
 *     Nothing is thrown across the ABI.
 *   - Counting: `iters` is the number of Newton updates applied; the paper's
 *     K (number of residual evaluations) is iters + 1.
 */
#ifndef PITN_H
#define PITN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes.  Non-negative codes describe a completed solve. */
typedef enum {
    PITN_OK = 0,              /* ||h||_inf <= tol reached */
    PITN_NOT_CONVERGED = 1,   /* max_iter updates applied, tolerance not met */
    PITN_NONFINITE = 2,       /* a residual entry, or (plain Newton) a Newton
                                 correction, was NaN/Inf; the trajectory holds
                                 the last iterate whose residual was finite */
    PITN_EINVAL = -1,         /* bad argument (nothing was written) */
    PITN_ENOMEM = -2,         /* device or host allocation failed */
    PITN_ECUDA = -3,          /* a CUDA runtime call failed */
    PITN_ETIMEOUT = -4,       /* an in-kernel wait exceeded its time limit */
    PITN_EUNSUPPORTED = -5    /* valid request this build does not implement */
} pitn_status;

/* ODE systems (right-hand sides f; parameters in this order). */
enum {
    PITN_LORENZ63 = 1,   /* d = 3; params {sigma, rho, beta}:
                            f = (sigma(y-x), x(rho-z)-y, xy-beta z) */
    PITN_VDP = 2,        /* d = 2; params {mu}; state (x, dx/dt):
                            f = (v, mu(1-x^2)v - x)  (Sec. 4.1, van der Pol) */
    PITN_LINEAR_OSC = 3, /* d = 2; params {omega, zeta}; state (x, dx/dt):
                            f = (v, -omega^2 x - 2 zeta omega v) (affine) */
    PITN_FKPP = 4,       /* d >= 3 interior nodes of [0,1], spacing 1/(d+1),
                            zero Dirichlet ends; params {D}:
                            f_i = D (u_{i-1} - 2u_i + u_{i+1})/dx^2 + u_i(1-u_i) */
    PITN_LOGISTIC = 5,   /* d = 1; params {r, K}: f = r P (1 - P/K)  (Sec. 4.1) */
    PITN_DAHLQUIST = 6,  /* d = 1; params {lambda}: f = lambda y  (Sec. 4.2) */
    PITN_ROBERTSON = 7   /* d = 3; params {k1, k2, k3}: f = (-k1 y1 + k3 y2 y3,
                            k1 y1 - k2 y2^2 - k3 y2 y3, k2 y2^2)  (Sec. 4.2, stiff) */
};

/* One-step maps (Sec. 2.1). */
enum {
    PITN_STEP_EULER = 0,  /* explicit Euler, eq. 2.2: every system in pitn_solve_ex;
                             LORENZ63 / VDP / LINEAR_OSC in the batched, adjoint and
                             no-allocation entry points */
    PITN_STEP_RK4 = 1,    /* classical Runge-Kutta, eq. 2.3; pitn_solve_ex only, for
                             PITN_VDP and PITN_LOGISTIC (the paper's explicit tests) */
    PITN_STEP_BACKWARD_EULER = 2, /* implicit Euler, eq. 2.5, with the implicit Newton
                             step of Sec. 3.4 (eqs. 3.14-3.19); pitn_solve_ex only, for
                             PITN_DAHLQUIST, PITN_ROBERTSON, PITN_VDP, PITN_LOGISTIC.
                             The residual an implicit rule reports, stops on and returns
                             in final_res / res_history is the preconditioned one,
                             ||(I - dg/dx_n)^{-1} h_n||_inf (h_n of eq. 3.15). */
    PITN_STEP_TRAPEZOID = 3 /* trapezoidal rule, g = (h/2)(f(x_{n-1}) + f(x_n))
                             (Sec. 3.4); same entry point, systems and residual as
                             PITN_STEP_BACKWARD_EULER */
};

/* Arithmetic of the Newton step (the residual and the update are always FP64). */
enum {
    PITN_PREC_FP64 = 0,        /* every operation in FP64 */
    PITN_PREC_MIXED_BF16 = 1,  /* PITN_FKPP with d >= 64: dense composes of the
                                  scan on tensor cores (BF16 operands, FP32
                                  accumulation) in the delta form A = J - I,
                                  tile folds and replay in FP32; residual,
                                  stopping test and update in FP64.  An
                                  inexact Newton step */
    PITN_PREC_MIXED_FP32 = 2,  /* d <= 3 (LORENZ63, VDP, LINEAR_OSC) with explicit
                                  Euler, VDP with RK4 (not in the paper; the
                                  stage chain rule of S in FP32 from the FP64
                                  stage states), and the implicit rules (backward
                                  Euler, trapezoidal; ROBERTSON, DAHLQUIST, VDP,
                                  LOGISTIC; S = J - I from the FP64 element):
                                  the scan's elements in FP32
                                  delta form (I + S, c); an inexact Newton step */
    PITN_PREC_FP64_FF = 3,     /* d <= 3 (VDP, LINEAR_OSC, LORENZ63) with explicit
                                  Euler, VDP with RK4, and the implicit rules
                                  (backward Euler, trapezoidal; ROBERTSON,
                                  DAHLQUIST, VDP, LOGISTIC; the FP64 element
                                  split into pairs) (not in the paper): the
                                  scan (Jacobians -- for RK4 the stage chain rule --,
                                  folds, carries, replay) in double-FP32 "float-float"
                                  arithmetic, ~2^-47 relative, on the FP32 pipe;
                                  residual, stopping test and update in FP64.  An
                                  inexact Newton step whose error is ~64x FP64
                                  rounding: it reaches the FP64 root at FP64
                                  accuracy.  Its range is the float range: a
                                  correction beyond 3.4e38 counts as not finite
                                  (FP64: 1.8e308) */
    PITN_PREC_MIXED_TF32 = 4   /* PITN_FKPP with d >= 64: as PITN_PREC_MIXED_BF16
                                  with TF32 operands (tcgen05 kind::tf32: the FP32
                                  aggregates as they stand, 10 mantissa bits) */
};

/* Per-solve outcome. */
typedef struct {
    int32_t iters;        /* Newton updates applied (paper K - 1) */
    int32_t status;       /* PITN_OK / PITN_NOT_CONVERGED / PITN_NONFINITE */
    double final_res;     /* ||h(xi)||_inf of the returned trajectory */
    int64_t guard_index;  /* guard cut q of the last update, N if none */
} pitn_result;

/* Options for the _ex entry points; a zero-initialised struct (or NULL)
 * selects the defaults shown. */
typedef struct {
    int32_t precision;      /* PITN_PREC_*; default FP64 */
    int32_t tile_elems;     /* elements per thread of the scan; 0 = autotuned */
    double guard_B;         /* <= 0: the paper's plain Newton (default).
                               > 0: divergence guard (not in the paper): after
                               each Newton step, q = first step index whose
                               correction has an entry that is not finite or
                               exceeds guard_B in magnitude; steps before q
                               are updated, steps from q on are set to the
                               last updated state (x0 if q = 0). */
    const double* guess;    /* NULL: constant guess x_n = x0; else [N][d] */
    void* stream;           /* cudaStream_t; NULL = legacy default stream */
    double* res_history;    /* NULL or host array of max_iter + 1 doubles:
                               ||h||_inf at every residual evaluation */
    int32_t method;         /* PITN_STEP_*; default explicit Euler */
    int64_t* cut_history;   /* NULL or host array of max_iter + 1 int64 (not in the
                               paper): entry k receives the guard cut q of
                               Newton step k, N when nothing was cut, for every
                               step computed -- the `iters` accepted steps and,
                               when a plain solve ends NONFINITE on a
                               correction, the rejected last one; the
                               remaining entries receive -1 */
} pitn_options;

/*
 * Solve one IVP by the paper's plain Newton method in FP64.
 *   system_id  PITN_LORENZ63 / PITN_VDP / PITN_LINEAR_OSC / PITN_FKPP / PITN_LOGISTIC /
 *              PITN_DAHLQUIST / PITN_ROBERTSON
 *   params     system parameters (see the enum), host or device
 *   x0         initial value x_0, [d]
 *   h          step size (finite, > 0)
 *   N          number of steps (>= 1); the trajectory has N states x_1..x_N
 *   d          state dimension; must match the system
 *   tol        stop when ||h(xi)||_inf <= tol (finite, >= 0)
 *   max_iter   maximum Newton updates (>= 0; 0 evaluates the residual only)
 *   traj_out   [N][d] output x_1..x_N
 * Returns the solve status (PITN_OK / PITN_NOT_CONVERGED / PITN_NONFINITE)
 * or a negative error code.
 */
int pitn_solve(int system_id, const double* params, const double* x0, double h, int64_t N, int d,
               double tol, int max_iter, double* traj_out);

/* pitn_solve with options (NULL = defaults) and an optional result record. */
int pitn_solve_ex(int system_id, const double* params, const double* x0, double h, int64_t N,
                  int d, double tol, int max_iter, double* traj_out, const pitn_options* opt,
                  pitn_result* result);

/*
 * Solve B independent IVPs of one system and uneven lengths N[b] in one call
 * (not in the paper: its experiments run one IVP at a time).  Each IVP runs
 * its own Newton iteration (Sec. 3) with its own stopping test; an IVP that
 * has stopped is frozen (neither its trajectory nor its count changes), and
 * the solve ends when every IVP has stopped or max_iter is reached.  Two
 * device paths compute the same iteration: one segmented scan over all IVPs
 * per Newton iteration, or one CTA per IVP running that IVP's whole loop
 * (IVPs taken longest first).  The autotuner, or with it off the lengths
 * (the per-IVP path when no IVP is longer than one CTA's share of the
 * steps), choose; tile_elems > 0 forces the segmented path with that many
 * steps per thread.
 *   params     [B][P], x0 [B][d], h [B], N [B] (each >= 1)
 *   traj_out   [sum N][d]: IVP b occupies rows offsets[b] .. offsets[b+1]-1
 *   offsets_out [B+1]: exclusive prefix sum of N (int64)
 *   iters_out, status_out [B] (int32); res_out [B] (nullable) final norms
 *   opt        guard_B, stream and tile_elems are honoured; method must be
 *              explicit Euler; guess and res_history must be NULL.
 *              precision PITN_PREC_FP64, or PITN_PREC_MIXED_FP32 /
 *              PITN_PREC_FP64_FF (the scans of pitn_solve_ex, on the per-IVP
 *              path only: tile_elems must then be 0, and a pinned segmented
 *              shape returns PITN_EUNSUPPORTED).
 * Returns PITN_OK when every IVP converged, PITN_NOT_CONVERGED when one did
 * not (see status_out), or a negative error code.
 */
int pitn_solve_batch(int system_id, int64_t B, const double* params, const double* x0,
                     const double* h, const int64_t* N, int d, double tol, int max_iter,
                     double* traj_out, int64_t* offsets_out, int32_t* iters_out,
                     int32_t* status_out, double* res_out, const pitn_options* opt);

/*
 * Gradients of a loss L(x_1..x_N) of converged trajectories with respect to
 * x0 and the parameters, for B IVPs laid out as in pitn_solve_batch (not in
 * the paper; the transposed, reverse-time form of the recursion of eq. 3.13):
 *   lambda_N = G_N,  lambda_n = J_n^T lambda_{n+1} + G_n,
 *   dL/dx0 = J_0^T lambda_1,  dL/dp = sum_n (dphi/dp(x_n))^T lambda_{n+1},
 * with G_n = grad_traj row n-1 (nullable) plus grad_xN on G_N (nullable).
 * The reverse recursion runs as an affine scan over (J^T, G); the scan keeps
 * one checkpoint (block product and block offset) per ckpt_every steps
 * (0 = 1024) and recomputes J_n from traj.
 *   traj       [sum N][d] forward trajectories (x_1..x_N per IVP)
 *   grad_x0_out [B][d], grad_params_out [B][P]
 */
int pitn_backward(int system_id, int64_t B, const double* params, const double* x0,
                  const double* h, const int64_t* N, int d, const double* traj,
                  const double* grad_traj, const double* grad_xN, int ckpt_every,
                  double* grad_x0_out, double* grad_params_out, const pitn_options* opt);

/*
 * The combine of eq. 3.3 for dense elements in the delta form A = I + S, as
 * used by the mixed-precision scan (Sec. 3.1; the delta form is not in the
 * paper):
 *   (I + S2, b2) o (I + S1, b1) = (I + S, b),  S = S2 + S1 + S2 S1,  b = b2 + b1 + S2 b1
 * for n independent pairs of 128 x 128 FP32 matrices stored column-major
 * (S[col][row]), element 2 the later one.  S2 S1 runs on the tensor cores
 * with BF16 operands and FP32 accumulation; sums and b in FP32.  All pointers
 * are device memory (matrices 16-byte aligned), n matrices / vectors each,
 * packed; stream may be NULL.  Returns PITN_OK or a negative error code.
 */
int pitn_affine_combine_delta(int64_t n, const float* S2, const float* b2, const float* S1,
                              const float* b1, float* S, float* b, void* stream);

/* The same combine with TF32 operands (tcgen05.mma kind::tf32, FP32
 * accumulation): the FP32 inputs are the operands as they stand, of which
 * the tensor core uses the TF32 part; the vector part uses the FP32 rows of
 * S2.  Same arguments, layouts and return codes. */
int pitn_affine_combine_delta_tf32(int64_t n, const float* S2, const float* b2, const float* S1,
                                   const float* b1, float* S, float* b, void* stream);

/* Number of parameters of a system, or -1 for an unknown id. */
int pitn_num_params(int system_id);

/* Static description of a code. */
const char* pitn_status_string(int code);

/* Frees the cached scratch memory of the current device.  Not to be called
 * while a solve is running on another host thread. */
int pitn_release_workspace(void);

/* Number of kernel launches the library issued since the process started
 * (all devices, all entry points). */
int64_t pitn_launch_count(void);

/* Work of the most recent pitn_solve_batch in this process (instrumentation
 * for throughput figures): the steps whose residual and Jacobian were
 * evaluated and folded, and the steps whose Newton step was replayed,
 * summed over its IVPs and passes, as the kernels count them (on both
 * paths a thread's share of a guard's fill region costs one evaluation, and
 * a thread's replay of an IVP ends at its first cut).  Both 0 before the
 * first batch solve.  Returns PITN_EINVAL for a NULL pointer. */
int pitn_batch_work(int64_t* evaluated, int64_t* replayed);

/*
 * Allocation-free solve for the small-state systems (PITN_LORENZ63, PITN_VDP,
 * PITN_LINEAR_OSC).  The paper has no counterpart: this is a deployment aid.
 *
 * Some callers cannot call cudaMalloc once they are running: a real-time
 * control loop whose time budget cannot absorb cudaMalloc's implicit device
 * synchronisation, or a host application whose own allocator has reserved
 * the device memory.  This entry point allocates nothing.  Its scratch is one
 * fixed file-scope __device__ array (about 8 MB, held on every GPU that
 * loads the library until the process exits), sized for at most
 * PITN_NOALLOC_MAX_STEPS steps and PITN_NOALLOC_MAX_ITER Newton updates;
 * larger requests return PITN_EINVAL.
 *   traj_out  [N][d] DEVICE memory (nothing can be staged for a host array);
 *   params, x0 host or device memory; guard_B as in pitn_options (<= 0 plain);
 *   result    nullable; runs on the legacy default stream and blocks until
 *             the result is on the host.
 * The first call on a device looks up the array's device address (a
 * one-time set-up per device); make that first call before any stream
 * capture on the device.  Every call shares the array and finds it holding
 * the previous call's contents; each call clears what must start at zero.
 * Calls that overlapped on the GPU would race on the array, so the entry
 * point holds a process-wide lock until its results are back on the host.
 * Results equal pitn_solve_ex's for the same arguments when no tuned or
 * pinned launch shape exists for the configuration (see pitn_tune_set):
 * this entry point always takes the default launch shape, and a different
 * shape associates the scan differently (last bits, and the iteration count
 * of a borderline solve, may then differ).  params, x0 and traj_out must not
 * be another GPU's memory (PITN_EINVAL).
 */
#define PITN_NOALLOC_MAX_STEPS 65536
#define PITN_NOALLOC_MAX_ITER 1024
int pitn_solve_noalloc(int system_id, const double* params, const double* x0, double h, int64_t N,
                       int d, double tol, int max_iter, double guard_B, double* traj_out,
                       pitn_result* result);

/*
 * Time-sharded solve of one IVP over several GPUs (not in the paper, which
 * runs on one GPU; the split is the paper's own scan split at the level of
 * devices).  A shard owns the contiguous steps [s, s + n) of one IVP of
 * PITN_LORENZ63, PITN_VDP or PITN_LINEAR_OSC (explicit Euler, FP64).  Per
 * Newton iteration a driver exchanges, between the shards, the state before
 * each shard (halo), the shard aggregates ((d^2 + d) doubles each, eq. 3.3),
 * the largest residual and the first guard cut; the shard-local work runs in
 * these calls:
 *   pitn_shard_create   a plan for n local steps (owns its device scratch);
 *                       guard_B as in pitn_options; stream nullable
 *   pitn_shard_pass     x_prev [d]: the state before the shard (x0 for the
 *                       shard holding step 0; the guard's fill state for a
 *                       shard wholly beyond the cut); holds_first: the shard
 *                       holds step 0 (its first element is (0, -r_0),
 *                       eq. 3.4); X [n][d]: the current iterate, whose states
 *                       from q_local on are read as the state before them
 *                       (lazy guard fill); writes the shard aggregate
 *                       agg_out [d^2 + d] (matrix row-major, then vector) and
 *                       the bit pattern of max |r| (eq. 3.8) to res_bits_out
 *                       [1] (non-negative doubles order like their bits; NaN
 *                       above +inf, so the driver reduces them as integers)
 *   pitn_shard_carry    the incoming correction of shard r: aggs [r][d^2 + d]
 *                       (the aggregates of shards 0 .. r-1 in order) composed
 *                       from the zero correction; z_out [d]
 *   pitn_shard_update   the replay of eq. 3.13 from z_in [d] over the elements
 *                       of the last pass, the next iterate into Xn [n][d], and
 *                       the local index of the first correction that is not
 *                       finite or exceeds guard_B, or n, into cut_out [1]
 *                       (int64)
 *   pitn_shard_finalize the iterate with its lazy fill written out: out [n][d]
 *   pitn_shard_destroy  frees the plan
 * Every array is device memory of the current device; each call blocks
 * until its outputs are written.  paper_2511_01465_gb300/timeshard.py is the
 * driver (torch.distributed, or shards emulated on one GPU).  Returns
 * PITN_OK, PITN_EINVAL (bad argument, update without a pass), PITN_ENOMEM or
 * PITN_ECUDA.
 */
typedef struct pitn_shard pitn_shard;
int pitn_shard_create(int system_id, const double* params, double h, int64_t n, int d, double guard_B,
                      void* stream, pitn_shard** out);
int pitn_shard_pass(pitn_shard* s, const double* x_prev, int holds_first, const double* X, int64_t q_local,
                    double* agg_out, int64_t* res_bits_out);
int pitn_shard_carry(pitn_shard* s, int64_t r, const double* aggs, double* z_out);
int pitn_shard_update(pitn_shard* s, const double* z_in, double* Xn, int64_t* cut_out);
int pitn_shard_finalize(pitn_shard* s, const double* X, const double* x_prev, int64_t q_local, double* out);
int pitn_shard_destroy(pitn_shard* s);

/*
 * Measured FMA issue rate of the current device (not in the paper; the
 * benchmark's ALU roofline denominators): kind 0 = FP64 (DFMA), 1 = FP32
 * (FFMA).  A register-only kernel runs 8 independent FMA chains per thread on
 * 8 blocks of 256 threads per SM; the best of three timed launches (after one
 * untimed) gives *fma_per_s, thread-level FMAs per second (one FMA = 2 flops).
 * Returns PITN_OK, PITN_EINVAL (unknown kind, NULL output) or PITN_ECUDA.
 */
int pitn_probe_fma_rate(int kind, double* fma_per_s);

/*
 * Failure injection for tests of the error paths (not in the paper).  Each
 * call changes one process-wide setting; PITN_DEBUG_RESET restores them all.
 *   PITN_DEBUG_FAIL_ALLOCS   value = n >= 0: the next n growths of the
 *                            scratch cache fail as if cudaMalloc had, so the
 *                            calls that need them return PITN_ENOMEM
 *   PITN_DEBUG_GRID_WAIT_NS  value ns (<= 0: the default 2 s): how long a
 *                            grid barrier of a cooperative kernel waits for
 *                            the other CTAs before the kernel gives up and
 *                            the call returns PITN_ETIMEOUT
 *   PITN_DEBUG_LOAD_POLLS    value polls (< 0: default 2^26): how long the
 *                            tensor-core compose waits on its bulk copies
 *   PITN_DEBUG_MMA_POLLS     value polls (< 0: default 2^26): how long it
 *                            waits on the tensor-core product
 * A compose whose wait gave up waits again with the default limit for the
 * copies or the product already in flight, so that it reads no TMEM and
 * frees neither TMEM nor shared memory under an asynchronous operation; only
 * if that wait also ends without completion does the CTA leave its TMEM
 * allocated.  Either way the call returns PITN_ETIMEOUT and the device stays
 * usable.  The settings apply to launches that start after the call.
 * Returns PITN_OK or PITN_EINVAL.
 */
enum {
    PITN_DEBUG_RESET = 0,
    PITN_DEBUG_FAIL_ALLOCS = 1,
    PITN_DEBUG_GRID_WAIT_NS = 2,
    PITN_DEBUG_LOAD_POLLS = 3,
    PITN_DEBUG_MMA_POLLS = 4
};
int pitn_debug_inject(int what, int64_t value);

/*
 * Launch-shape autotuner (not in the paper).  While enabled, the first solve
 * of a configuration class -- (entry point, system, d, floor(log2 size),
 * guard on/off) -- times each candidate launch shape (threads per CTA and
 * CTAs per SM for pitn_solve; threads per CTA and steps per thread for
 * pitn_solve_batch, where 0 steps per thread is the per-IVP path) on the
 * call's own inputs, keeps the fastest in a process-wide cache, and then
 * returns the result computed with it; later solves of that class use the
 * cached shape.  With the environment
 * variable PITN_TUNE_CACHE naming a file, the cache is loaded from and saved
 * to that file.  A user guess is saved and put back around the trials.
 * Different shapes associate the scan differently, so results may differ in
 * the last bits.  Keys: "small:<system>:<d>:<floor log2 N>:<guarded 0/1>"
 * plus ":rk4", ":be" or ":tr" for the RK4, backward Euler and trapezoidal
 * maps and ":f32" / ":ff" for PITN_PREC_MIXED_FP32 / PITN_PREC_FP64_FF
 * (e.g. "small:2:2:22:1"), and "batch:<system>:<d>:<floor log2 of the total
 * steps>:<guarded>", with the same ":f32" / ":ff".
 * pitn_tune_get reads one entry; pitn_tune_set pins one (a: threads per
 * CTA, a multiple of 32 up to 1024; b > 0, or b = 0 in a batch key for the
 * per-IVP path; else PITN_EINVAL.  A shape that does not fit the device
 * makes the solve return PITN_EUNSUPPORTED or PITN_ECUDA), so that a
 * deployment can fix its launch shapes without tuning. */
int pitn_tune_enable(int on);
int pitn_tune_clear(void);
int pitn_tune_get(const char* key, int* a, int* b);
int pitn_tune_set(const char* key, int a, int b);

/* Per-kernel timing (tracing).  While enabled, every kernel launch of the
 * library is bracketed by CUDA events on its stream; pitn_timing_get returns
 * the summed device time and launch count of one kernel family since the
 * last reset (names: "newton_small", "fkpp_residual", "fkpp_fold", "fkpp_compose",
 * "fkpp_replay", "batch", "adjoint").  Timing adds two event
 * records per launch; it is off by default. */
int pitn_timing_enable(int on);
int pitn_timing_reset(void);
int pitn_timing_get(const char* kernel, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* PITN_H */
