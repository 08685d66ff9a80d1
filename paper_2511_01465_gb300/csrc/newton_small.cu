// newton_small.cu -- the whole Newton solve for small state dimension
// (d = 1, 2, 3) in ONE persistent cooperative kernel.
//
// Thread g of the grid owns a contiguous range of steps.  Per Newton
// iteration the three-phase kernel (newton_small.cuh) runs:
//   1. phase 1: loads x_{k-1}, x_k (lazy fill of the guard, see below),
//      evaluates the residual r_k = x_{k+1} - phi(x_k) (eq. 3.8) and the
//      compact Jacobian J_k = dphi/dx(x_k), stores both to scratch, keeps
//      ||r||_inf (an integer max of the bit patterns) and folds its affine
//      elements (J_k, -r_k) (eq. 3.4; element 0 has matrix 0) into a thread
//      aggregate with the operator of eq. 3.3, as two interleaved chains;
//   2. scans the thread aggregates: Kogge-Stone over the warp with shuffles,
//      then over the warps through shared memory, and writes the CTA
//      aggregate to its slot of a global array;
//   3. grid barrier: every CTA's aggregate and the iteration's ||r||_inf are
//      visible; every CTA takes the same stop/continue decision;
//   4. every CTA scans the CTA aggregates in one fixed order to find its own
//      incoming correction vector (only the vector part is needed: every
//      prefix that starts at element 0 has matrix 0).  The order does not
//      depend on timing, so results are reproducible run to run;
//   5. phase 3: replays its steps from the incoming vector,
//      dx_{k+1} = J_k dx_k - r_k (eq. 3.13), with J_k and r_k read back from
//      scratch, and writes x_k + dx_k into the other trajectory buffer,
//      recording the first index whose correction is not finite or exceeds
//      the guard bound;
//   6. grid barrier: the iteration's guard index is visible to all CTAs.
// Every CTA writes its aggregate slot before the first barrier of each
// iteration, so the aggregate array never needs clearing between solves.
// The guard's fill (states from q on set to state q-1) is never written
// during the loop: the next pass reads x_k for k >= q as x_{q-1}.
//
// The decision order per iteration is the oracle's: non-finite residual ->
// NONFINITE; ||r|| <= tol -> OK; max_iter updates -> NOT_CONVERGED; plain
// Newton with a non-finite correction -> NONFINITE (iterate kept); otherwise
// accept the step.
#include "newton_small.cuh"


namespace pitn_host {

// Launch shape: about `cmin` steps per thread at least, as many CTAs as the
// device holds at once (cooperative launch), blocks of 32..256 threads.
void small_default_config(int d, long long N, int* block, int* C) {
    (void)d;
    const int sms = props().multiProcessorCount;
    const long long cmin = 4;
    long long threads = (N + cmin - 1) / cmin;
    long long b = (threads + sms - 1) / sms;
    b = ((b + 31) / 32) * 32;
    b = std::max(32LL, std::min(256LL, b));
    *block = (int)b;
    *C = (int)cmin;
}

// The kernel instantiation for a system, step map and precision.  Explicit
// maps are instantiated here; the implicit (backward Euler) ones and the
// stiff test systems live in newton_implicit.cu.
int select_small_kernel(int system_id, int method, int precision, pitn::SmallKernel* K) {
    using namespace pitn;
    if (precision == PITN_PREC_FP64_FF && (method == PITN_STEP_BACKWARD_EULER || method == PITN_STEP_TRAPEZOID))
        return select_implicit_kernel(system_id, method, precision, K);
    if (precision == PITN_PREC_FP64_FF) {
        // the float-float scan runs fused, like the FP32 one: its FP64 work
        // is the residual and the update
        if (method == PITN_STEP_RK4) {
            // the RK4 map's stage chain rule in float-float, its residual in FP64
            if (system_id != PITN_VDP) return PITN_EUNSUPPORTED;
            *K = small_kernel_of<RK4Map<VdpRhs>, kVarFusedFF>();
            return PITN_OK;
        }
        if (method != PITN_STEP_EULER) return PITN_EUNSUPPORTED;
        switch (system_id) {
        case PITN_VDP: *K = small_kernel_of<VanDerPol, kVarFusedFF>(); return PITN_OK;
        case PITN_LINEAR_OSC: *K = small_kernel_of<LinearOsc, kVarFusedFF>(); return PITN_OK;
        // d = 3 keeps the three-phase structure, as its FP32 twin (registers)
        case PITN_LORENZ63: *K = small_kernel_of<Lorenz63, kVarMixedFF>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (precision == PITN_PREC_MIXED_FP32 && method == PITN_STEP_RK4) {
        // the RK4 map's stage chain rule in FP32 (delta form), its residual in FP64
        if (system_id != PITN_VDP) return PITN_EUNSUPPORTED;
        *K = small_kernel_of<RK4Map<VdpRhs>, kVarFusedMixed>();
        return PITN_OK;
    }
    if (precision == PITN_PREC_MIXED_FP32 && (method == PITN_STEP_BACKWARD_EULER || method == PITN_STEP_TRAPEZOID))
        return select_implicit_kernel(system_id, method, precision, K);
    if (precision == PITN_PREC_MIXED_FP32) {
        // the d = 2 FP32-scan solves run fused: their FP64 work (residual,
        // update) is light enough that one pass per iteration beats two (van
        // der Pol N = 2^22: 21.5 -> 17.0 ms); Lorenz (177 registers fused)
        // keeps the three-phase kernel (N = 8192: 1.14 vs 1.22 ms)
        if (method != PITN_STEP_EULER) return PITN_EUNSUPPORTED;
        switch (system_id) {
        case PITN_LORENZ63: *K = small_kernel_of<Lorenz63, kVarMixed>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<VanDerPol, kVarFusedMixed>(); return PITN_OK;
        case PITN_LINEAR_OSC: *K = small_kernel_of<LinearOsc, kVarFusedMixed>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    // Maps with a costly element (RK4 stages, implicit solves) take the fused
    // kernel, whose single pass overlaps the element's FP64 work with the
    // update's memory traffic; the cheap explicit Euler elements run faster
    // in the three-phase kernel (measured on van der Pol, N = 2^22).
    if (method == PITN_STEP_RK4) {
        switch (system_id) {
        case PITN_VDP: *K = small_kernel_of<RK4Map<VdpRhs>, kVarFused>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<RK4Map<LogisticRhs>, kVarFused>(); return PITN_OK;
        default: return PITN_EUNSUPPORTED;
        }
    }
    if (method == PITN_STEP_EULER) {
        switch (system_id) {
        case PITN_LORENZ63: *K = small_kernel_of<Lorenz63, kVarPlain>(); return PITN_OK;
        case PITN_VDP: *K = small_kernel_of<VanDerPol, kVarPlain>(); return PITN_OK;
        case PITN_LINEAR_OSC: *K = small_kernel_of<LinearOsc, kVarPlain>(); return PITN_OK;
        case PITN_LOGISTIC: *K = small_kernel_of<EulerMap<LogisticRhs>, kVarPlain>(); return PITN_OK;
        default: break;
        }
    }
    return select_implicit_kernel(system_id, method, precision, K);
}

// One solve with an explicit launch shape: `block` threads per CTA, at most
// `per_sm_cap` co-resident CTAs per SM (cooperative launch) and at least
// `cmin` steps per thread (which bounds the grid of a short trajectory;
// the caller's tile_elems overrides it).
int small_launch(int system_id, const SolveIO& io, double h, int64_t N, int d, double tol,
                 int max_iter, const pitn_options& o, cudaStream_t st, SolveOutcome* out, int block,
                 int per_sm_cap, int cmin) {
    using namespace pitn;
    if (o.tile_elems > 0) cmin = o.tile_elems;
    pitn::SmallKernel K{};
    int rc = select_small_kernel(system_id, o.method, o.precision, &K);
    if (rc != PITN_OK) return rc;
    int per_sm = K.per_sm(block);
    const int W = K.W;
    if (per_sm < 1) return PITN_EUNSUPPORTED;  // shape does not fit on an SM
    per_sm = std::min(per_sm, per_sm_cap);
    const long long max_grid = (long long)per_sm * props().multiProcessorCount;
    const long long want = (N + (long long)block * cmin - 1) / ((long long)block * cmin);
    const int grid = (int)std::max(1LL, std::min(max_grid, want));
    const long long chunk = (N + (long long)grid * block - 1) / ((long long)grid * block);
    const int E = d * d + d;
    // a thread's regular steps per iteration are at most ceil(N / threads) (the
    // weighted partition gives a regular step a quarter of a thread's share)
    const long long nthr = (long long)grid * block;
    const long long lcap = (N + nthr - 1) / nthr + 1;

    double* X1 = (double*)workspace((size_t)N * d * sizeof(double), kSlotX1);
    double* scratch = (double*)workspace((size_t)lcap * nthr * W * sizeof(double), kSlotAux);
    // control block: agg | res_bits | qenc | bar | err | record
    size_t off_agg = 0;
    size_t off_res = off_agg + (size_t)grid * E * sizeof(double);
    size_t off_q = off_res + sizeof(unsigned long long) * (size_t)(max_iter + 1);
    size_t off_bar = (off_q + sizeof(unsigned long long) * (size_t)(max_iter + 1) + 15) & ~(size_t)15;
    size_t off_err = off_bar + 16;
    size_t off_rec = off_err + 16;
    size_t total = off_rec + sizeof(SolveRecord);
    char* ctrl = (char*)workspace(total, kSlotCtrl);
    // host mirror: err | record | history | cut codes
    size_t hbytes = 16 + sizeof(SolveRecord) + 2 * sizeof(double) * (size_t)(max_iter + 1);
    char* hbuf = (char*)pinned(hbytes);
    if (!X1 || !scratch || !ctrl || !hbuf) return PITN_ENOMEM;

    SmallArgs a{};
    a.x0 = io.x0_dev;
    a.X0 = io.traj_dev;
    a.X1 = X1;
    a.out = io.traj_dev;
    a.scratch = scratch;
    a.lcap = lcap;
    a.agg = (double*)(ctrl + off_agg);
    a.N = N;
    a.chunk = chunk;
    a.h = h;
    a.tol = tol;
    a.guarded = (o.guard_B > 0.0 && std::isfinite(o.guard_B)) ? 1 : 0;
    {
        const double cap = a.guarded ? o.guard_B : DBL_MAX;
        std::memcpy(&a.cap_bits, &cap, sizeof(cap));
    }
    a.max_iter = max_iter;
    a.q_init = io.have_guess ? N : 0;
    for (int i = 0; i < 4; ++i) a.params[i] = io.params[i];
    a.res_bits = (unsigned long long*)(ctrl + off_res);
    a.qenc = (unsigned long long*)(ctrl + off_q);
    a.bar = (unsigned*)(ctrl + off_bar);
    a.err = (int*)(ctrl + off_err);
    a.rec = (SolveRecord*)(ctrl + off_rec);
    a.wait_ns = wait_limits().grid_ns;

    if (cudaMemsetAsync(ctrl, 0, total, st) != cudaSuccess) return PITN_ECUDA;
    if (K.consts) K.consts(io.params, h, a.fc, a.dc);
    cudaError_t e = K.launch(a, grid, block, st);
    if (e != cudaSuccess) { cudaGetLastError(); return PITN_ECUDA; }
    int* h_err = (int*)hbuf;
    SolveRecord* h_rec = (SolveRecord*)(hbuf + 16);
    unsigned long long* h_hist = (unsigned long long*)(hbuf + 16 + sizeof(SolveRecord));
    unsigned long long* h_q = h_hist + (max_iter + 1);
    // the residual history and the cut codes are adjacent in the control block
    if (cudaMemcpyAsync(h_err, ctrl + off_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_rec, ctrl + off_rec, sizeof(SolveRecord), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_hist, ctrl + off_res, sizeof(unsigned long long) * (max_iter + 1),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_q, ctrl + off_q, sizeof(unsigned long long) * (max_iter + 1),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PITN_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return PITN_ECUDA; }
    if (*h_err != 0) return *h_err;
    out->iters = h_rec->iters;
    out->status = h_rec->status;
    out->final_res = h_rec->final_res;
    out->guard_index = h_rec->guard_index;
    out->history.resize(out->iters + 1);
    for (int k = 0; k <= out->iters; ++k) {
        long long b = (long long)h_hist[k];
        double v;
        std::memcpy(&v, &b, sizeof(v));
        out->history[k] = v;
    }
    // cut of every computed Newton step (the code is ~q, 0 when nothing was
    // cut); a step at index iters was computed only if it was rejected, which
    // a plain solve does on a cut (a non-finite correction)
    out->cuts.clear();
    for (int k = 0; k < out->iters; ++k) out->cuts.push_back(h_q[k] ? (long long)~h_q[k] : (long long)N);
    if (out->iters <= max_iter && h_q[out->iters]) out->cuts.push_back((long long)~h_q[out->iters]);
    return PITN_OK;
}

// Launch shapes the autotuner tries (threads per CTA, CTAs per SM).
// (Shapes beyond a kernel's occupancy are capped by it; repeats are skipped.)
static const int kSmallShapes[][2] = {{128, 1}, {128, 2}, {128, 3}, {128, 4}, {128, 6}, {128, 8},
                                      {256, 1}, {256, 2}, {256, 3}, {256, 4}};

int small_solve_full(int system_id, const SolveIO& io, double h, int64_t N, int d, double tol,
                     int max_iter, const pitn_options& o, cudaStream_t st, SolveOutcome* out) {
    int block = 0, cmin = 0;
    small_default_config(d, N, &block, &cmin);
    int cap = 2;
    const bool guarded = o.guard_B > 0.0 && std::isfinite(o.guard_B);
    char key[96];
    std::snprintf(key, sizeof(key), "small:%d:%d:%d:%d%s%s", system_id, d, tune_bucket(N), guarded ? 1 : 0,
                  o.method == PITN_STEP_RK4 ? ":rk4"
                  : o.method == PITN_STEP_BACKWARD_EULER ? ":be"
                  : o.method == PITN_STEP_TRAPEZOID ? ":tr" : "",
                  o.precision == PITN_PREC_MIXED_FP32 ? ":f32" : o.precision == PITN_PREC_FP64_FF ? ":ff" : "");
    char ckey[104];
    std::snprintf(ckey, sizeof(ckey), "%s:c", key);   // steps-per-thread floor of the shape
    int tb = 0, tc = 0;
    if (tune_lookup(key, &tb, &tc)) {
        block = tb;
        cap = tc;
        int c2 = 0, unused = 0;
        if (tune_lookup(ckey, &c2, &unused) && c2 > 0) cmin = c2;
    } else if (tune_enabled()) {
        // time every shape on this very solve; the cost per Newton pass decides.
        // A caller's guess lives in the trajectory buffer, which every trial
        // overwrites: keep a copy and put it back before each trial and the
        // final solve.
        const size_t gbytes = (size_t)N * d * sizeof(double);
        double* saved = nullptr;
        if (io.have_guess) {
            saved = (double*)workspace(gbytes, kSlotAux2);
            if (!saved) return PITN_ENOMEM;
            if (cudaMemcpyAsync(saved, io.traj_dev, gbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return PITN_ECUDA;
        }
        pitn::SmallKernel K{};
        int rk = select_small_kernel(system_id, o.method, o.precision, &K);
        if (rk != PITN_OK) return rk;
        // a short trajectory fills the GPU only with few steps per thread, and
        // there the floor decides the grid: try 1, 2 and 4 steps as well
        const bool short_n = N < 2LL * 256 * 4 * props().multiProcessorCount;
        const int cmins_short[] = {1, 2, 4}, cmins_long[] = {4};
        const int* cmins = short_n ? cmins_short : cmins_long;
        const int ncm = short_n ? 3 : 1;
        // the trials solve the same problem from the same start: the whole
        // solve's time decides (the FP32-scan solve, an inexact Newton method,
        // needs a number of iterations that depends on the shape)
        // one untimed solve first: a kernel's first launch also loads its code
        // (lazy module loading), which must not count against the first shape
        for (const auto& shp : kSmallShapes) {
            if (std::min(K.per_sm(shp[0]), shp[1]) < 1) continue;
            SolveOutcome tmp;
            (void)small_launch(system_id, io, h, N, d, tol, max_iter, o, st, &tmp, shp[0], shp[1], cmins[0]);
            if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
            break;
        }
        double best = 1e300;
        int tried[3 * sizeof(kSmallShapes) / sizeof(kSmallShapes[0])][3];
        int ntried = 0;
        for (int ci = 0; ci < ncm; ++ci) {
            for (const auto& shp : kSmallShapes) {
                const int eff = std::min(K.per_sm(shp[0]), shp[1]);  // CTAs per SM this shape gets
                if (eff < 1) continue;
                bool seen = false;
                for (int i = 0; i < ntried; ++i)
                    seen |= tried[i][0] == shp[0] && tried[i][1] == eff && tried[i][2] == cmins[ci];
                if (seen) continue;
                tried[ntried][0] = shp[0];
                tried[ntried][1] = eff;
                tried[ntried][2] = cmins[ci];
                ++ntried;
                if (saved && cudaMemcpyAsync(io.traj_dev, saved, gbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    return PITN_ECUDA;
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
                SolveOutcome tmp;
                const int rc = small_launch(system_id, io, h, N, d, tol, max_iter, o, st, &tmp, shp[0], shp[1],
                                            cmins[ci]);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (rc != PITN_OK) continue;
                if (ms < best) {
                    best = ms;
                    block = shp[0];
                    cap = shp[1];
                    cmin = cmins[ci];
                }
            }
        }
        tune_store(key, block, cap);
        tune_store(ckey, cmin, 0);
        if (saved && cudaMemcpyAsync(io.traj_dev, saved, gbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return PITN_ECUDA;
    }
    return small_launch(system_id, io, h, N, d, tol, max_iter, o, st, out, block, cap, cmin);
}

}  // namespace pitn_host

// ---------------------------------------------------------------------------
// Allocation-free variant of the small-state solve.
//
// Some callers must not allocate device memory once they are running: a
// real-time control loop (the optimal-control use the method targets) whose
// time budget cannot absorb cudaMalloc's implicit device synchronisation, or
// a host application whose own allocator has reserved the device memory, so
// that a cudaMalloc from this library would fail or fragment its pool.  This
// entry point keeps all of its scratch in one file-scope __device__ array of
// fixed size instead of the library's growing workspace cache.  Every GPU that
// loads the library holds that array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr long long kNaMaxSteps = 1LL << 16;  // N limit
constexpr int kNaMaxIter = 1024;              // max_iter limit
constexpr int kNaMaxCtas = 1024;              // CTA aggregates
constexpr size_t kNaX1 = 0;                                            // [N][3]
constexpr size_t kNaScratch = kNaX1 + (size_t)kNaMaxSteps * 3;         // [6][lcap][threads]
constexpr size_t kNaScratchDoubles = (size_t)kNaMaxSteps * 6 * 2;      // >= 6 (N + 2 threads)
// CTA aggregates: never cleared, since every CTA writes its own slot before
// the grid barrier after which any CTA reads it
constexpr size_t kNaAgg = kNaScratch + kNaScratchDoubles;               // [CTAs][12]
constexpr size_t kNaRes = kNaAgg + (size_t)kNaMaxCtas * 12;            // [iter+1] bits
constexpr size_t kNaQ = kNaRes + (size_t)(kNaMaxIter + 1);             // [iter+1] bits
constexpr size_t kNaCtl = kNaQ + (size_t)(kNaMaxIter + 1);             // bar, err, record, x0
constexpr size_t kNaDoubles = kNaCtl + 32;

}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

namespace {
std::mutex g_na_mu;
double* g_na_addr[256] = {};  // device address of the array, per device ordinal
}  // namespace

extern "C" int pitn_solve_noalloc(int system_id, const double* params, const double* x0, double h,
                                  int64_t N, int d, double tol, int max_iter, double guard_B,
                                  double* traj_out, pitn_result* result) {
    using namespace pitn;
    using namespace pitn_host;
    if (system_id != PITN_LORENZ63 && system_id != PITN_VDP && system_id != PITN_LINEAR_OSC)
        return PITN_EINVAL;
    if (!system_dim_ok(system_id, d) || !params || !x0 || !traj_out) return PITN_EINVAL;
    if (N < 1 || N > kNaMaxSteps || max_iter < 0 || max_iter > kNaMaxIter) return PITN_EINVAL;
    if (!std::isfinite(h) || !(h > 0.0) || !std::isfinite(tol) || !(tol >= 0.0) || std::isnan(guard_B))
        return PITN_EINVAL;
    if (!is_device_ptr(traj_out)) return PITN_EINVAL;  // nowhere to stage a host trajectory
    // the kernel runs on the current device: another GPU's memory is refused
    if (any_foreign({params, x0, traj_out})) return PITN_EINVAL;

    std::lock_guard<std::mutex> lk(g_na_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PITN_ECUDA;
    if (!g_na_addr[dev]) {
        // one-time set-up on this device: the host-side name of the array is
        // not a device address, so ask the runtime for the real one
        double* ptr = nullptr;
        if (cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return PITN_ECUDA;
        }
        g_na_addr[dev] = ptr;
    }
    double* base = g_na_addr[dev];

    double hp[4] = {0.0, 0.0, 0.0, 0.0};
    const int P = num_params(system_id);
    if (is_device_ptr(params)) {
        if (cudaMemcpy(hp, params, sizeof(double) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
            return PITN_ECUDA;
    } else {
        for (int i = 0; i < P; ++i) hp[i] = params[i];
    }

    // launch shape: the same rule as the workspace-backed solve, capped by
    // the number of CTA aggregates the array holds
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PITN_ECUDA;
    const long long cmin = 4;
    long long b = ((N + cmin - 1) / cmin + sms - 1) / sms;
    b = std::max(32LL, std::min(256LL, ((b + 31) / 32) * 32));
    const int block = (int)b;
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    // Lorenz-63's kernel takes the CTA-wide scan buffer, as in the workspace-backed solve
    const size_t dyn = (system_id == PITN_LORENZ63) ? CtaScanLayout<3>::kBytes : 0;
    if (dyn > 0 && cudaFuncSetAttribute((const void*)newton_small_kernel<Lorenz63>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return PITN_ECUDA;
    switch (system_id) {
    case PITN_LORENZ63:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_small_kernel<Lorenz63>, block, dyn);
        break;
    case PITN_VDP:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_small_kernel<VanDerPol>, block, 0);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_small_kernel<LinearOsc>, block, 0);
        break;
    }
    if (e != cudaSuccess || per_sm < 1) return PITN_ECUDA;
    per_sm = std::min(per_sm, 2);
    const long long want = (N + (long long)block * cmin - 1) / ((long long)block * cmin);
    const int grid = (int)std::max(1LL, std::min<long long>({(long long)per_sm * sms, want, (long long)kNaMaxCtas}));
    const long long chunk = (N + (long long)grid * block - 1) / ((long long)grid * block);

    cudaStream_t st = 0;
    char* ctl = (char*)(base + kNaCtl);
    SmallArgs a{};
    double* x0_dev = (double*)(ctl + 128);
    const cudaMemcpyKind k0 = is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(x0_dev, x0, sizeof(double) * d, k0, st) != cudaSuccess) return PITN_ECUDA;
    // everything that must start at zero: per-iteration reductions, barrier, error, record
    if (cudaMemsetAsync(base + kNaRes, 0, sizeof(double) * (kNaCtl - kNaRes) + 128, st) != cudaSuccess)
        return PITN_ECUDA;
    a.x0 = x0_dev;
    a.X0 = traj_out;
    a.X1 = base + kNaX1;
    a.out = traj_out;
    a.scratch = base + kNaScratch;
    {
        const long long nthr = (long long)grid * block;
        a.lcap = (N + nthr - 1) / nthr + 1;
        if ((size_t)(a.lcap * nthr * 6) > kNaScratchDoubles) return PITN_EINVAL;  // cannot happen: N/cmin + block threads
    }
    a.agg = base + kNaAgg;
    a.N = N;
    a.chunk = chunk;
    a.h = h;
    a.tol = tol;
    a.guarded = (guard_B > 0.0 && std::isfinite(guard_B)) ? 1 : 0;
    {
        const double cap = a.guarded ? guard_B : DBL_MAX;
        std::memcpy(&a.cap_bits, &cap, sizeof(cap));
    }
    a.max_iter = max_iter;
    a.q_init = 0;
    for (int i = 0; i < 4; ++i) a.params[i] = hp[i];
    a.res_bits = (unsigned long long*)(base + kNaRes);
    a.qenc = (unsigned long long*)(base + kNaQ);
    a.bar = (unsigned*)ctl;
    a.err = (int*)(ctl + 16);
    a.rec = (SolveRecord*)(ctl + 32);
    a.wait_ns = wait_limits().grid_ns;
    a.cta_scan = dyn > 0 ? 1 : 0;
    void* args[] = {(void*)&a};
    const void* kern = (system_id == PITN_LORENZ63) ? (const void*)newton_small_kernel<Lorenz63>
                       : (system_id == PITN_VDP)    ? (const void*)newton_small_kernel<VanDerPol>
                                                    : (const void*)newton_small_kernel<LinearOsc>;
    if (cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(block), args, dyn, st) != cudaSuccess) {
        cudaGetLastError();
        return PITN_ECUDA;
    }
    count_launch(1);
    SolveRecord rec{};
    int err = 0;
    if (cudaMemcpy(&err, ctl + 16, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&rec, ctl + 32, sizeof(SolveRecord), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PITN_ECUDA;
    if (err != 0) return err;
    if (result) {
        result->iters = rec.iters;
        result->status = rec.status;
        result->final_res = rec.final_res;
        result->guard_index = rec.guard_index;
    }
    return rec.status;
}
