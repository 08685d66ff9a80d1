// newton_small.cuh -- the persistent small-state Newton kernel and its launch
// helpers, shared by the translation units that instantiate it for the
// explicit maps (newton_small.cu) and the implicit ones (newton_implicit.cu).
// The algorithm is described at the top of newton_small.cu.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cfloat>

#include "common.cuh"
#include "solver.h"
#include "systems.cuh"

namespace pitn {

struct SolveRecord {
    int iters;
    int status;
    double final_res;
    long long guard_index;
};

struct SmallArgs {
    const double* x0;   // [D] device
    double* X0;         // trajectory buffer 0 [N][D]
    double* X1;         // trajectory buffer 1 [N][D]
    double* out;        // destination of the final iterate
    double* scratch;    // [JN + D][lcap][threads]: compact Jacobian and residual of every
                        // regular step, component-major and interleaved over the threads so
                        // that a warp's accesses to step i of its chunks are coalesced
    long long lcap;     // upper bound on a thread's regular steps per iteration
    double* agg;        // [gridDim][D*D + D]: CTA aggregates
    long long N;
    long long chunk;    // consecutive steps per thread
    double h, tol;
    unsigned long long cap_bits;  // |dx| bits above this are cut (guard bound or DBL_MAX)
    int guarded;
    int max_iter;
    long long q_init;   // 0: constant guess x0 (buffer contents ignored); N: buffer 0 holds the guess
    double params[4];
    unsigned long long* res_bits;  // [max_iter + 1]  ||r||_inf bits per iteration
    unsigned long long* qenc;      // [max_iter + 1]  max of ~q (0 = no cut)
    unsigned* bar;                 // [2] grid barrier
    int* err;
    SolveRecord* rec;
    int stage_rows;                // > 0: rows of the next iterate leave through shared-memory
                                   // tiles and bulk copies (dynamic smem sized by stage_bytes)
    int cta_scan;                  // d = 3 three-phase kernel: 1 when the launch gave it the
                                   // CTA-wide scan buffer (dynamic smem, CtaScanLayout<3>::kBytes)
    unsigned long long wait_ns;    // grid-barrier wait limit (0: the default)
    // system constants precomputed on the host for the float-float scan
    // (kernel parameters live in the constant bank, so the compiler reloads
    // them instead of recomputing them with FP64 instructions inside the loop)
    float fc[16];
    double dc[4];
};

constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

template <int D>
__device__ __forceinline__ void mat_identity(double* P) {
#pragma unroll
    for (int i = 0; i < D * D; ++i) P[i] = (i % (D + 1) == 0) ? 1.0 : 0.0;
}

// (P, c) <- (P2, c2) o (P1, c1) = (P2 P1, P2 c1 + c2)   (eq. 3.3, 2 = later)
template <int D>
__device__ __forceinline__ void compose(const double* P2, const double* c2, const double* P1,
                                        const double* c1, double* P, double* c) {
    double tP[D * D], tc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double s = P2[i * D] * P1[j];
#pragma unroll
            for (int l = 1; l < D; ++l) s = fma(P2[i * D + l], P1[l * D + j], s);
            tP[i * D + j] = s;
        }
        double s = c2[i];
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(P2[i * D + l], c1[l], s);
        tc[i] = s;
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) P[i] = tP[i];
#pragma unroll
    for (int i = 0; i < D; ++i) c[i] = tc[i];
}

// o = P v + c
template <int D>
__device__ __forceinline__ void apply(const double* P, const double* c, const double* v, double* o) {
    double t[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        double s = c[i];
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(P[i * D + l], v[l], s);
        t[i] = s;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) o[i] = t[i];
}

// x_k of the current iterate with the guard's lazy fill.  L1-cacheable
// loads (ld.global.ca, never the non-coherent read-only path: the buffers
// alternate roles between iterations): every state read in a phase was
// written before the grid barrier that opens it, and the barrier's gpu-scope
// acquire orders the loads after those writes; a thread's consecutive steps
// then share L1 sectors instead of each going to L2.
template <int D>
__device__ __forceinline__ void load_state(const double* __restrict__ X, const double* __restrict__ x0,
                                           long long k, long long q, double* o) {
    const double* src;
    if (k < 0) src = x0;
    else if (k < q) src = X + k * D;
    else if (q > 0) src = X + (q - 1) * D;
    else src = x0;
#pragma unroll
    for (int i = 0; i < D; ++i) o[i] = __ldca(src + i);
}

constexpr int kMaxWarps = 8;  // BLOCK <= 256

// ---------------------------------------------------------------------------
// Staged stores of the next iterate (rows of 2 doubles).  A thread's rows are
// contiguous in the trajectory, but a warp's row-by-row stores land in 32
// different lines; instead each thread collects kStageT consecutive rows in a
// private shared-memory tile and sends the tile with one bulk copy (TMA, an
// async-proxy write of one contiguous 16 B-aligned span).  Two tiles per
// chain alternate, so a tile is refilled only after its copy has read it.
// ---------------------------------------------------------------------------
constexpr int kStageT = 4;                   // rows per tile
constexpr int kStageSeg = kStageT * 2 + 2;   // doubles per tile slot (+16 B: bank spread)

__host__ __device__ constexpr size_t stage_bytes(int block) {
    return (size_t)2 * 2 * block * kStageSeg * sizeof(double);
}

__device__ __forceinline__ void bulk_store_rows(double* gdst, const double* ssrc, unsigned bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(ssrc);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :: "l"(gdst), "r"(s), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

struct RowStage {
    double* seg;      // this thread's first slot; slot (c, s) at seg + (c * 2 + s) * stride
    int stride;       // doubles between slots (blockDim * kStageSeg)
    int n[2], slot[2];
    long long start[2];
    __device__ __forceinline__ void init(double* smem) {
        stride = blockDim.x * kStageSeg;
        seg = smem + (size_t)threadIdx.x * kStageSeg;
        n[0] = n[1] = 0;
        slot[0] = slot[1] = 0;
        start[0] = start[1] = 0;
    }
    __device__ __forceinline__ double* tile(int c) { return seg + (size_t)(c * 2 + slot[c]) * stride; }
    __device__ __forceinline__ void flush(int c, double* X) {
        if (n[c] == 0) return;
        bulk_store_rows(X + start[c] * 2, tile(c), (unsigned)(n[c] * 16));
        slot[c] ^= 1;
        n[c] = 0;
    }
    // row k (2 doubles) of chain c; rows of one chain arrive in increasing order
    __device__ __forceinline__ void put(int c, long long k, double v0, double v1, double* X) {
        if (n[c] > 0 && k != start[c] + n[c]) flush(c, X);
        if (n[c] == 0) {
            // the slot's previous copy is at least two groups old
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            start[c] = k;
        }
        double2* t = reinterpret_cast<double2*>(tile(c)) + n[c];
        *t = make_double2(v0, v1);
        if (++n[c] == kStageT) flush(c, X);
    }
    // all tiles written to global memory and ordered before later generic accesses
    __device__ __forceinline__ void finish(double* X) {
        flush(0, X);
        flush(1, X);
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
};

// Inclusive Kogge-Stone scan of (P, c) across the warp (later lanes on the left).
template <int D>
__device__ __forceinline__ void warp_scan(double* P, double* c, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        double uP[D * D], uc[D];
#pragma unroll
        for (int j = 0; j < D * D; ++j) uP[j] = __shfl_up_sync(0xffffffffu, P[j], off);
#pragma unroll
        for (int j = 0; j < D; ++j) uc[j] = __shfl_up_sync(0xffffffffu, c[j], off);
        if (lane >= off) compose<D>(P, c, uP, uc, P, c);
    }
}

// CTA-wide inclusive Kogge-Stone scan (eq. 3.3) of n <= kCtaScanMax elements
// held in shared memory, for d = 3.  A warp's FP64 instruction holds its
// sub-partition's FP64 unit for ~70 cycles on this part, so a level of a
// scan that one warp runs alone (36 FP64 instructions for a 3 x 3 compose)
// takes ~2.7 k cycles while the CTA's other sub-partitions idle.  Here each
// level's composes are dealt out to all threads one output at a time
// (element l, output o), so every sub-partition's FP64 unit shares the
// level.  Each output is computed in compose<D>'s order: the results are
// those of the warp scan.  buf holds two halves of kCtaScanMax elements of
// EP doubles (E padded to an odd count: 8-byte accesses of consecutive
// elements without bank conflicts); the elements start in the first half,
// and the returned pointer is the half that holds the result.
constexpr int kCtaScanMax = 128;
template <int D>
struct CtaScanLayout {
    static constexpr int E = D * D + D;
    static constexpr int EP = E | 1;
    static constexpr size_t kBytes = 2 * (size_t)kCtaScanMax * EP * sizeof(double);
};

// output o of compose<D>(A, B) (A the later element), in compose<D>'s order
template <int D>
__device__ __forceinline__ double compose_out(const double* A, const double* B, int o) {
    double v;
    if (o < D * D) {
        const int i = o / D, j = o - i * D;
        v = A[i * D] * B[j];
#pragma unroll
        for (int k = 1; k < D; ++k) v = fma(A[i * D + k], B[k * D + j], v);
    } else {
        const int i = o - D * D;
        v = A[D * D + i];
#pragma unroll
        for (int k = 0; k < D; ++k) v = fma(A[i * D + k], B[D * D + k], v);
    }
    return v;
}

template <int D>
__device__ __forceinline__ double* cta_scan(double* buf, int n) {
    constexpr int E = CtaScanLayout<D>::E, EP = CtaScanLayout<D>::EP;
    double* src = buf;
    double* dst = buf + kCtaScanMax * EP;
    for (int off = 1; off < n; off <<= 1) {
        for (int item = threadIdx.x; item < n * E; item += blockDim.x) {
            const int l = item / E, o = item - l * E;
            dst[l * EP + o] = (l >= off) ? compose_out<D>(src + l * EP, src + (l - off) * EP, o) : src[l * EP + o];
        }
        __syncthreads();
        double* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Exclusive block scan of per-thread elements.  On return (eP, ec) is the
// lane-exclusive prefix within the warp, s_wex[warp] the warp-exclusive
// prefix, and s_tot the block total.  All in a fixed order.
// (d = 3 with a scan buffer: the scan over the warps runs CTA-wide, see
// cta_scan, with the same results.)
// live_warps: warps from live_warps on hold identities only and skip their
// warp scan (which would leave the identities unchanged).
template <int D>
__device__ __forceinline__ void block_scan(double* P, double* c, double* eP, double* ec,
                                           double (*s_wex)[D * D + D], double* s_tot,
                                           double* scan_buf = nullptr, int live_warps = kMaxWarps) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (warp < live_warps) warp_scan<D>(P, c, lane);
#pragma unroll
    for (int j = 0; j < D * D; ++j) eP[j] = __shfl_up_sync(0xffffffffu, P[j], 1);
#pragma unroll
    for (int j = 0; j < D; ++j) ec[j] = __shfl_up_sync(0xffffffffu, c[j], 1);
    if (lane == 0) {
        mat_identity<D>(eP);
#pragma unroll
        for (int j = 0; j < D; ++j) ec[j] = 0.0;
    }
    __syncthreads();  // s_wex may still be read from a previous use
    if (D == 3 && scan_buf != nullptr) {   // (the launchers pass a buffer for d = 3 only)
        constexpr int E = D * D + D, EP = CtaScanLayout<D>::EP;
        if (lane == 31) {
#pragma unroll
            for (int j = 0; j < D * D; ++j) scan_buf[warp * EP + j] = P[j];
#pragma unroll
            for (int j = 0; j < D; ++j) scan_buf[warp * EP + D * D + j] = c[j];
        }
        __syncthreads();
        const double* inc = cta_scan<D>(scan_buf, nwarps);
        // warp-exclusive prefixes (identity for warp 0) and the block total
        for (int item = threadIdx.x; item < nwarps * E; item += blockDim.x) {
            const int w = item / E, o = item - w * E;
            s_wex[w][o] = (w > 0) ? inc[(w - 1) * EP + o] : ((o < D * D && o % (D + 1) == 0) ? 1.0 : 0.0);
        }
        if (threadIdx.x < E) s_tot[threadIdx.x] = inc[(nwarps - 1) * EP + threadIdx.x];
        __syncthreads();
        return;
    }
    if (lane == 31) {
#pragma unroll
        for (int j = 0; j < D * D; ++j) s_wex[warp][j] = P[j];
#pragma unroll
        for (int j = 0; j < D; ++j) s_wex[warp][D * D + j] = c[j];
    }
    __syncthreads();
    if (warp == 0) {
        double wP[D * D], wc[D];
        if (lane < nwarps) {
#pragma unroll
            for (int j = 0; j < D * D; ++j) wP[j] = s_wex[lane][j];
#pragma unroll
            for (int j = 0; j < D; ++j) wc[j] = s_wex[lane][D * D + j];
        } else {
            mat_identity<D>(wP);
#pragma unroll
            for (int j = 0; j < D; ++j) wc[j] = 0.0;
        }
#pragma unroll
        for (int off = 1; off < kMaxWarps; off <<= 1) {
            if (off >= nwarps) break;   // lanes from nwarps on hold identities
            double uP[D * D], uc[D];
#pragma unroll
            for (int j = 0; j < D * D; ++j) uP[j] = __shfl_up_sync(0xffffffffu, wP[j], off);
#pragma unroll
            for (int j = 0; j < D; ++j) uc[j] = __shfl_up_sync(0xffffffffu, wc[j], off);
            if (lane >= off) compose<D>(wP, wc, uP, uc, wP, wc);
        }
        double xP[D * D], xc[D];
#pragma unroll
        for (int j = 0; j < D * D; ++j) xP[j] = __shfl_up_sync(0xffffffffu, wP[j], 1);
#pragma unroll
        for (int j = 0; j < D; ++j) xc[j] = __shfl_up_sync(0xffffffffu, wc[j], 1);
        __syncwarp();
        if (lane < nwarps) {
            if (lane == 0) {
                mat_identity<D>(xP);
#pragma unroll
                for (int j = 0; j < D; ++j) xc[j] = 0.0;
            }
#pragma unroll
            for (int j = 0; j < D * D; ++j) s_wex[lane][j] = xP[j];
#pragma unroll
            for (int j = 0; j < D; ++j) s_wex[lane][D * D + j] = xc[j];
        }
        if (lane == nwarps - 1) {
#pragma unroll
            for (int j = 0; j < D * D; ++j) s_tot[j] = wP[j];
#pragma unroll
            for (int j = 0; j < D; ++j) s_tot[D * D + j] = wc[j];
        }
    }
    __syncthreads();
}

// Incoming correction vector of this CTA for small grids: the vector part of
// the composition of the CTA aggregates 0 .. b-1, in a fixed order, computed
// by warp 0 alone (the other warps wait at the closing barrier).  Lane l folds
// aggregates [l m, (l+1) m), m = ceil(G / 32); a warp scan gives each lane the
// prefix before its group, whose vector part is its whole effect on the zero
// initial correction (every prefix from aggregate 0 has matrix 0, eq. 3.4);
// the lane holding aggregate b - 1 applies its group's aggregates up to b - 1
// to that vector.  With few aggregates this avoids the CTA-wide scan; with
// many, the lanes' serial folds make it slower than the CTA-wide one.
template <int D>
__device__ __forceinline__ void cta_incoming(const double* __restrict__ agg, unsigned G, double* s_zin) {
    constexpr int E = D * D + D;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned m = (G + 31) / 32;
        double gP[D * D], gc[D];
        mat_identity<D>(gP);
#pragma unroll
        for (int j = 0; j < D; ++j) gc[j] = 0.0;
        for (unsigned i = lane * m; i < min(G, (lane + 1) * m); ++i) {
            double sP[D * D], sc[D];
#pragma unroll
            for (int j = 0; j < D * D; ++j) sP[j] = __ldcg(agg + (size_t)i * E + j);
#pragma unroll
            for (int j = 0; j < D; ++j) sc[j] = __ldcg(agg + (size_t)i * E + D * D + j);
            compose<D>(sP, sc, gP, gc, gP, gc);
        }
        warp_scan<D>(gP, gc, lane);
        double v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = __shfl_up_sync(0xffffffffu, gc[j], 1);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < D; ++j) v[j] = 0.0;
        }
        if (blockIdx.x > 0 && (unsigned)lane == (blockIdx.x - 1) / m) {
            for (unsigned i = lane * m; i <= blockIdx.x - 1; ++i) {
                double sP[D * D], sc[D], t[D];
#pragma unroll
                for (int j = 0; j < D * D; ++j) sP[j] = __ldcg(agg + (size_t)i * E + j);
#pragma unroll
                for (int j = 0; j < D; ++j) sc[j] = __ldcg(agg + (size_t)i * E + D * D + j);
                apply<D>(sP, sc, v, t);
#pragma unroll
                for (int j = 0; j < D; ++j) v[j] = t[j];
            }
#pragma unroll
            for (int j = 0; j < D; ++j) s_zin[j] = v[j];
        }
        if (blockIdx.x == 0 && lane == 0) {
#pragma unroll
            for (int j = 0; j < D; ++j) s_zin[j] = 0.0;
        }
    }
    __syncthreads();
}

// cta_incoming with its composes dealt out to the whole CTA (d = 3, G <= 64),
// in the same order and so with the same results: each group's fold onto the
// identity, aggregate by aggregate; the Kogge-Stone scan of the group
// aggregates (cta_scan); then the owner of aggregate b - 1 (one thread)
// applies its group's aggregates up to b - 1 to the group's incoming vector.
// buf (CtaScanLayout<D>) holds the group aggregates in rows [0, 32) of its
// halves and the CTA aggregates, read once through L2, in rows [64, 128) of
// its first half.
template <int D>
__device__ __forceinline__ void cta_incoming_wide(const double* __restrict__ agg, unsigned G, double* s_zin,
                                                  double* buf) {
    constexpr int E = D * D + D, EP = CtaScanLayout<D>::EP;
    const unsigned m = (G + 31) / 32;
    const int ng = (int)((G + m - 1) / m);   // groups that hold aggregates
    double* g = buf;                          // group aggregates (first half, rows [0, ng))
    double* t = buf + kCtaScanMax * EP;       // second half: the folds' other buffer
    double* A = buf + 64 * EP;                // the CTA aggregates (first half, rows [64, 64 + G))
    for (int item = threadIdx.x; item < (int)G * E; item += blockDim.x) {
        const int l = item / E, o = item - l * E;
        A[l * EP + o] = __ldcg(agg + (size_t)l * E + o);
    }
    for (int item = threadIdx.x; item < ng * E; item += blockDim.x) {
        const int o = item % E;
        g[(item / E) * EP + o] = (o < D * D && o % (D + 1) == 0) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (unsigned r = 0; r < m; ++r) {
        // g_l <- aggregate (l m + r) o g_l, for every group that has one
        for (int item = threadIdx.x; item < ng * E; item += blockDim.x) {
            const int l = item / E, o = item - l * E;
            const unsigned i = (unsigned)l * m + r;
            t[l * EP + o] = (i < G) ? compose_out<D>(A + i * EP, g + l * EP, o) : g[l * EP + o];
        }
        __syncthreads();
        for (int item = threadIdx.x; item < ng * E; item += blockDim.x) {
            const int l = item / E, o = item - l * E;
            g[l * EP + o] = t[l * EP + o];
        }
        __syncthreads();
    }
    const double* inc = cta_scan<D>(buf, ng);
    if (threadIdx.x == 0) {
        double v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = 0.0;
        if (blockIdx.x > 0) {
            const unsigned lo = (blockIdx.x - 1) / m;   // the group that holds aggregate b - 1
            if (lo > 0) {
#pragma unroll
                for (int j = 0; j < D; ++j) v[j] = inc[(lo - 1) * EP + D * D + j];
            }
            for (unsigned i = lo * m; i <= blockIdx.x - 1; ++i) {
                double tv[D];
                apply<D>(A + i * EP, A + i * EP + D * D, v, tv);
#pragma unroll
                for (int j = 0; j < D; ++j) v[j] = tv[j];
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) s_zin[j] = v[j];
    }
    __syncthreads();
}

// Deterministic three-phase Newton kernel (persistent, cooperative launch).
// Thread g owns steps [g*chunk, (g+1)*chunk).  Per Newton iteration:
//   phase 1: residuals + compact Jacobians (stored to scratch), thread fold,
//            block scan, CTA aggregate to global;   grid barrier;
//   decision on ||r||_inf (identical in every CTA);
//   scan of the CTA aggregates in a fixed order (every CTA derives its own
//   incoming prefix the same way), replay of the thread's steps from its
//   incoming vector, update into the other buffer, first guard cut;
//   grid barrier.
template <class Sys>
__global__ void __launch_bounds__(256) newton_small_kernel(SmallArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D, W = JN + D;
    Sys sys;
    sys.init(a.params, a.h);

    __shared__ double s_wex[kMaxWarps][E];
    __shared__ double s_tot[E];
    __shared__ double s_g[kMaxWarps][E];
    __shared__ double s_gtot[E];
    __shared__ double s_zin[D];
    // row-stage tiles (D == 2, stage_rows > 0); the CTA-wide scan buffer (D == 3, cta_scan)
    extern __shared__ __align__(16) double s_dyn[];
    double* const scan_buf = (D == 3 && a.cta_scan) ? s_dyn : nullptr;

    const int lane = threadIdx.x & 31;
    const long long N = a.N;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const unsigned G = gridDim.x;
    double* __restrict__ scr = a.scratch;

    int cur = 0;
    long long q = a.q_init;
    long long last_cut = N;
    int it = 0, status = PITN_NOT_CONVERGED;
    double final_res = 0.0;

    for (;;) {
        const double* __restrict__ Xc = cur ? a.X1 : a.X0;
        double* __restrict__ Xn = cur ? a.X0 : a.X1;
        // ---- phase 1: residual, Jacobian, fold -------------------------------
        // Elements from sfill on lie in the guard's fill region: all their
        // states equal x_{q-1}, so every one of them is the same element
        // (J(x_{q-1}), -r_f); a thread folds its share of them by binary
        // powering instead of one by one.
        const long long sfill = (q < N) ? (q > 1 ? q : 1LL) : N;
        // Work partition of this iteration: a regular element costs about four
        // times a fill element (phase 1 + phase 3 against phase 3 only), so the
        // steps are split over all threads by that weight; every thread derives
        // its contiguous range [k0, k1) from (N, sfill) alone.
        long long k0, k1;
        {
            const long long wreg = 4 * sfill;
            const long long wtot = wreg + (N - sfill);
            const long long per = (wtot + nthreads - 1) / nthreads;
            const long long w0 = gt * per, w1 = w0 + per;
            k0 = (w0 <= wreg) ? (w0 + 3) / 4 : sfill + (w0 - wreg);
            k1 = (w1 <= wreg) ? (w1 + 3) / 4 : sfill + (w1 - wreg);
            k0 = min(N, k0);
            k1 = min(N, k1);
        }
        const long long kreg = min(k1, max(k0, sfill));  // regular elements: [k0, kreg)
        // scratch slot of component j of this thread's i-th regular element
        // slot of component j of step i: (j lcap + i) threads + gt, written so
        // that a step costs one multiply and the components fixed offsets
        const long long cstride = a.lcap * nthreads;
        auto sidx = [&](long long i, int j) -> long long { return i * nthreads + gt + j * cstride; };
        // The regular part is folded as two interleaved halves A = [k0, km) and
        // B = [km, kreg): two independent FP64 dependency chains per thread.
        unsigned long long my_res = 0ull;
        const long long Lr = kreg - k0;
        const long long LA = (Lr + 1) / 2, LB = Lr - LA, km = k0 + LA;
        double PA[D * D], cA[D], PB[D * D], cB[D], xpA[D], xpB[D];
        mat_identity<D>(PA);
        mat_identity<D>(PB);
#pragma unroll
        for (int j = 0; j < D; ++j) { cA[j] = 0.0; cB[j] = 0.0; }
        if (LA > 0) load_state<D>(Xc, a.x0, k0 - 1, q, xpA);
        if (LB > 0) load_state<D>(Xc, a.x0, km - 1, q, xpB);
        auto fold_step = [&](long long k, double* xp, double* P, double* c) {
            double x[D], r[D], jv[JN];
            load_state<D>(Xc, a.x0, k, q, x);
            sys.eval(xp, x, r, jv);
#pragma unroll
            for (int j = 0; j < JN; ++j) scr[sidx(k - k0, j)] = jv[j];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                scr[sidx(k - k0, JN + j)] = r[j];
                const unsigned long long b = abs_bits(r[j]);
                my_res = b > my_res ? b : my_res;
            }
            if (k == 0) {  // a_0 = (0, -r_0), eq. 3.4
#pragma unroll
                for (int j = 0; j < D * D; ++j) P[j] = 0.0;
#pragma unroll
                for (int j = 0; j < D; ++j) c[j] = -r[j];
            } else {
                double tP[D * D], tc[D];
                sys.jmul(jv, P, tP);
                sys.jvec_sub(jv, c, r, tc);
#pragma unroll
                for (int j = 0; j < D * D; ++j) P[j] = tP[j];
#pragma unroll
                for (int j = 0; j < D; ++j) c[j] = tc[j];
            }
#pragma unroll
            for (int j = 0; j < D; ++j) xp[j] = x[j];
        };
        for (long long i = 0; i < LA; ++i) {
            fold_step(k0 + i, xpA, PA, cA);
            if (i < LB) fold_step(km + i, xpB, PB, cB);
        }
        double P[D * D], c[D];
        compose<D>(PB, cB, PA, cA, P, c);
        if (kreg < k1) {
            double xf[D], rf[D], jvf[JN], EP[D * D], Ec[D], RP[D * D], Rc[D];
            load_state<D>(Xc, a.x0, q - 1, q, xf);
            sys.eval(xf, xf, rf, jvf);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const unsigned long long b = abs_bits(rf[j]);
                my_res = b > my_res ? b : my_res;
                Ec[j] = -rf[j];
                Rc[j] = 0.0;
            }
            sys.jfull(jvf, EP);
            mat_identity<D>(RP);
            for (long long e = k1 - kreg;;) {
                if (e & 1) compose<D>(EP, Ec, RP, Rc, RP, Rc);
                e >>= 1;
                if (!e) break;
                compose<D>(EP, Ec, EP, Ec, EP, Ec);
            }
            compose<D>(RP, Rc, P, c, P, c);
        }
        double eP[D * D], ec[D];
        block_scan<D>(P, c, eP, ec, s_wex, s_tot, scan_buf);
        if (threadIdx.x < E) a.agg[(size_t)blockIdx.x * E + threadIdx.x] = s_tot[threadIdx.x];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_res, off);
            my_res = o > my_res ? o : my_res;
        }
        if (lane == 0 && my_res) atomicMax(a.res_bits + it, my_res);
        if (!grid_barrier(a.bar, a.bar + 1, G, a.err, a.wait_ns)) return;

        // ---- decision --------------------------------------------------------
        const unsigned long long rb = __ldcg(a.res_bits + it);
        const double res = __longlong_as_double((long long)rb);
        final_res = res;
        if (rb >= kInfBits) { status = PITN_NONFINITE; break; }
        if (res <= a.tol) { status = PITN_OK; break; }
        if (it == a.max_iter) { status = PITN_NOT_CONVERGED; break; }

        // ---- incoming prefix of this CTA: fixed-order scan of the aggregates ----
        // (a grid of at most 64 CTAs: warp 0 alone, its serial part stays short;
        // larger grids: every thread takes a share and the CTA scans)
        if (G <= 64 && scan_buf != nullptr) {
            cta_incoming_wide<D>(a.agg, G, s_zin, scan_buf);   // d = 3: dealt out to the CTA
        } else if (G <= 64) {
            cta_incoming<D>(a.agg, G, s_zin);
        } else {
            const unsigned m = (G + blockDim.x - 1) / blockDim.x;   // aggregates per thread
            // only aggregates 0 .. b-1 reach CTA b's prefix: later groups stay
            // the identity and warps holding none of them skip their scan
            // (the prefixes this CTA reads are the same)
            const unsigned need = blockIdx.x;
            const int live_warps = (int)(((need + m - 1) / m + 31) / 32);
            double gP[D * D], gc[D];
            mat_identity<D>(gP);
#pragma unroll
            for (int j = 0; j < D; ++j) gc[j] = 0.0;
            for (unsigned i = threadIdx.x * m; i < min(need, (threadIdx.x + 1) * m); ++i) {
                double sP[D * D], sc[D];
#pragma unroll
                for (int j = 0; j < D * D; ++j) sP[j] = __ldcg(a.agg + (size_t)i * E + j);
#pragma unroll
                for (int j = 0; j < D; ++j) sc[j] = __ldcg(a.agg + (size_t)i * E + D * D + j);
                compose<D>(sP, sc, gP, gc, gP, gc);
            }
            double xP[D * D], xc[D];
            block_scan<D>(gP, gc, xP, xc, s_g, s_gtot, scan_buf, live_warps);
            // CTA b needs the prefix through aggregate b-1, held by thread (b-1)/m:
            // its exclusive prefix (warp part, then lane part) applied to the zero
            // vector -- every prefix from aggregate 0 has matrix 0 -- then the
            // aggregates it owns up to b-1, in order.
            if (blockIdx.x > 0 && threadIdx.x == (blockIdx.x - 1) / m) {
                double v[D], t[D], zero[D];
#pragma unroll
                for (int j = 0; j < D; ++j) zero[j] = 0.0;
                apply<D>(s_g[threadIdx.x >> 5], s_g[threadIdx.x >> 5] + D * D, zero, t);
                apply<D>(xP, xc, t, v);
                for (unsigned i = threadIdx.x * m; i <= blockIdx.x - 1; ++i) {
                    double sP[D * D], sc[D];
#pragma unroll
                    for (int j = 0; j < D * D; ++j) sP[j] = __ldcg(a.agg + (size_t)i * E + j);
#pragma unroll
                    for (int j = 0; j < D; ++j) sc[j] = __ldcg(a.agg + (size_t)i * E + D * D + j);
                    apply<D>(sP, sc, v, t);
#pragma unroll
                    for (int j = 0; j < D; ++j) v[j] = t[j];
                }
#pragma unroll
                for (int j = 0; j < D; ++j) s_zin[j] = v[j];
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
                for (int j = 0; j < D; ++j) s_zin[j] = 0.0;
            }
            __syncthreads();
        }

        // ---- phase 3: replay + update ------------------------------------------
        // A thread stops at its first cut index: every later state of its
        // chunk lies beyond the iteration's cut and is never read again.
        unsigned long long my_q = 0ull;
        {
            double zw[D], zA[D], zB[D];
            apply<D>(s_wex[threadIdx.x >> 5], s_wex[threadIdx.x >> 5] + D * D, s_zin, zw);
            apply<D>(eP, ec, zw, zA);
            apply<D>(PA, cA, zA, zB);  // state entering half B
            bool foundA = false, foundB = false;
            long long firstA = 0, firstB = 0;
            const bool staged = (D == 2) && a.stage_rows > 0;
            RowStage stg;
            if (staged) stg.init(s_dyn);
            // x_{k+1} = x + dx of chain c into the other buffer
            auto put_row = [&](int c, long long k, const double* v) {
                if constexpr (D == 2) {
                    if (staged) { stg.put(c, k, v[0], v[1], Xn); return; }
                }
#pragma unroll
                for (int j = 0; j < D; ++j) Xn[k * D + j] = v[j];
            };
            auto replay_step = [&](int c, long long k, double* z) -> bool {
                double jv[JN], r[D], x[D];
#pragma unroll
                for (int j = 0; j < JN; ++j) jv[j] = scr[sidx(k - k0, j)];   // this thread's phase-1 writes
#pragma unroll
                for (int j = 0; j < D; ++j) r[j] = scr[sidx(k - k0, JN + j)];
                load_state<D>(Xc, a.x0, k, q, x);
                if (k == 0) {
#pragma unroll
                    for (int j = 0; j < D; ++j) z[j] = -r[j];
                } else {
                    double tz[D];
                    sys.jvec_sub(jv, z, r, tz);
#pragma unroll
                    for (int j = 0; j < D; ++j) z[j] = tz[j];
                }
                unsigned long long zb = 0ull;
                double xn[D];
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    xn[j] = x[j] + z[j];
                    const unsigned long long b = abs_bits(z[j]);
                    zb = b > zb ? b : zb;
                }
                put_row(c, k, xn);
                return zb > a.cap_bits;
            };
            for (long long i = 0; i < LA && !foundA; ++i) {
                if (replay_step(0, k0 + i, zA)) { foundA = true; firstA = k0 + i; }
                if (i < LB && !foundB && replay_step(1, km + i, zB)) { foundB = true; firstB = km + i; }
            }
            bool found = foundA || foundB;
            if (found) my_q = ~(unsigned long long)(foundA ? firstA : firstB);
            double z[D];
#pragma unroll
            for (int j = 0; j < D; ++j) z[j] = (LB > 0) ? zB[j] : zA[j];
            if (!found && kreg < k1) {
                double xf[D], rf[D], jvf[JN];
                load_state<D>(Xc, a.x0, q - 1, q, xf);
                sys.eval(xf, xf, rf, jvf);
                for (long long k = kreg; k < k1; ++k) {
                    double tz[D];
                    sys.jvec_sub(jvf, z, rf, tz);
                    unsigned long long zb = 0ull;
                    double xn[D];
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        z[j] = tz[j];
                        xn[j] = xf[j] + z[j];
                        const unsigned long long b = abs_bits(z[j]);
                        zb = b > zb ? b : zb;
                    }
                    put_row(1, k, xn);
                    if (zb > a.cap_bits) {
                        my_q = ~(unsigned long long)k;
                        break;
                    }
                }
            }
            if (staged) stg.finish(Xn);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_q, off);
            my_q = o > my_q ? o : my_q;
        }
        if (lane == 0 && my_q) atomicMax(a.qenc + it, my_q);
        if (!grid_barrier(a.bar, a.bar + 1, G, a.err, a.wait_ns)) return;
        const unsigned long long qe = __ldcg(a.qenc + it);
        const long long cut = qe ? (long long)(~qe) : N;
        if (!a.guarded && cut < N) { status = PITN_NONFINITE; break; }
        cur ^= 1;
        q = a.guarded ? cut : N;
        last_cut = cut;
        ++it;
    }

    // ---- write the final iterate (with its fill) to the destination ---------
    const double* Xc = cur ? a.X1 : a.X0;
    const bool same = (Xc == a.out);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = gt; k < N; k += stride) {
        if (same && k < q) continue;
        double v[D];
        load_state<D>(Xc, a.x0, k, q, v);
#pragma unroll
        for (int j = 0; j < D; ++j) a.out[k * D + j] = v[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.rec->iters = it;
        a.rec->status = status;
        a.rec->final_res = final_res;
        a.rec->guard_index = last_cut;
    }
}

}  // namespace pitn

#include "newton_small_mixed.cuh"
#include "newton_fused.cuh"
#include "newton_fused_mixed.cuh"

namespace pitn {

// Kernel variants behind a SmallKernel: the three-phase FP64 kernel, its
// reduced-precision twins (FP32 delta form, float-float), and the fused FP64
// and reduced-precision kernels.
enum SmallVariant { kVarPlain = 0, kVarMixed = 1, kVarFused = 2, kVarFusedMixed = 3, kVarFusedFF = 4,
                    kVarMixedFF = 5 };

// Dynamic shared memory of a launch: the row-stage tiles for d = 2; the
// CTA-wide scan buffer of the three-phase FP64 kernel for d = 3.
template <class Sys, int VAR>
static size_t small_dyn_smem(int block) {
    if constexpr (Sys::D == 2) return stage_bytes(block);
    else if constexpr (Sys::D == 3 && VAR == kVarPlain) return CtaScanLayout<3>::kBytes;
    else return 0;
}

template <class Sys, int VAR>
static const void* small_kernel_ptr() {
    if constexpr (VAR == kVarMixed) return (const void*)newton_small_mixed_kernel<Sys, ScanF32>;
    else if constexpr (VAR == kVarMixedFF) return (const void*)newton_small_mixed_kernel<Sys, ScanFF>;
    else if constexpr (VAR == kVarFused) return (const void*)newton_fused_kernel<Sys>;
    else if constexpr (VAR == kVarFusedMixed) return (const void*)newton_fused_mixed_kernel<Sys, ScanF32>;
    else if constexpr (VAR == kVarFusedFF) return (const void*)newton_fused_mixed_kernel<Sys, ScanFF>;
    else return (const void*)newton_small_kernel<Sys>;
}

template <class Sys, int VAR = kVarPlain>
static cudaError_t launch_small(SmallArgs& a, int grid, int block, cudaStream_t st) {
    const void* kern = small_kernel_ptr<Sys, VAR>();
    const size_t dyn = small_dyn_smem<Sys, VAR>(block);
    if (dyn > 0 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return cudaErrorInvalidValue;
    // bulk copies need 16 B-aligned rows in both trajectory buffers
    const bool aligned = ((reinterpret_cast<uintptr_t>(a.X0) | reinterpret_cast<uintptr_t>(a.X1)) & 15) == 0;
    a.stage_rows = (Sys::D == 2 && dyn > 0 && aligned) ? kStageT : 0;
    a.cta_scan = (Sys::D == 3 && dyn > 0) ? 1 : 0;
    void* args[] = {(void*)&a};
    auto tok = pitn_host::timed_begin("newton_small", st);
    cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(block), args, dyn, st);
    pitn_host::timed_end(tok, st);
    pitn_host::count_launch(1);
    return e;
}

template <class Sys, int VAR = kVarPlain>
static int max_blocks_per_sm(int block) {
    const void* kern = small_kernel_ptr<Sys, VAR>();
    const size_t dyn = small_dyn_smem<Sys, VAR>(block);
    if (dyn > 0 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, dyn) != cudaSuccess) return 0;
    return per_sm;
}

// One instantiation of the kernel as the host sees it: its launcher, its
// occupancy query and the scratch doubles it keeps per step (compact
// Jacobian and residual, JN + D).
struct SmallKernel {
    cudaError_t (*launch)(SmallArgs&, int, int, cudaStream_t);
    int (*per_sm)(int);
    int W;
    void (*consts)(const double* p, double h, float* fc, double* dc);  // nullable
};

template <class Sys, int VAR = kVarPlain>
static SmallKernel small_kernel_of() {
    SmallKernel k{&launch_small<Sys, VAR>, &max_blocks_per_sm<Sys, VAR>, Sys::JN + Sys::D, nullptr};
    if constexpr (VAR == kVarFusedFF || VAR == kVarMixedFF) k.consts = &Sys::ff_consts;
    return k;
}

}  // namespace pitn

namespace pitn_host {
// Instantiations for the backward Euler map and for the stiff test systems
// (newton_implicit.cu); PITN_EUNSUPPORTED for combinations not built.
int select_implicit_kernel(int system_id, int method, int precision, pitn::SmallKernel* K);
}  // namespace pitn_host
