// fkpp.cu -- Newton solve for the Fisher-KPP method-of-lines systems
// (d >= 3 interior nodes, d <= 128), FP64 or mixed precision.
//
// The step map is phi(u) = u + h f(u) with f_i = D (u_{i-1} - 2u_i + u_{i+1})/dx^2
// + u_i (1 - u_i), so the Jacobian of every leaf element is tridiagonal:
//   J_k = I + S_k,  S_k = h (D L/dx^2 + diag(1 - 2 u_k)),
// diagonal a_i = 1 + h (1 - 2 u_i) - 2 o and off-diagonals o = h D / dx^2.
// One Newton pass is a host loop of launches on one stream:
//   A0. residual: fk_residual_kernel evaluates r_k (eq. 3.8) in FP64 with
//              ||r||_inf and the leaf diagonals; fk_stop_kernel then sets a
//              device flag when the pass has converged (or is not finite),
//              and every later kernel of the pass returns at once;
//   A.  fold:  fk_fold_kernel, one CTA per tile of TS consecutive elements,
//              folds the tile's leaves P <- J_k P, b <- J_k b - r_k into a
//              dense tile aggregate (P = I + S, b); the tridiagonal leaf is
//              applied as a stencil in registers (halo rows by warp
//              shuffles), 3 d^2 per element instead of 2 d^3;
//   B.  up-sweep: pairs of aggregates are composed level by level (eq. 3.3),
//              (I + S2)(I + S1) = I + (S2 + S1 + S2 S1),  b = b2 + b1 + S2 b1,
//              up to the level below the root (the root aggregate is never
//              read).  FP64: fk_compose_f64, one launch per level on CUDA
//              cores.  Mixed precision: fk_upsweep_tc_kernel, one launch per
//              pass, S2 S1 on tensor cores (tcgen05.mma, TMEM accumulator,
//              FP32 accumulation), sums in FP32; a CTA composes its level-1
//              node and climbs while it is the second child to arrive at the
//              parent's counter;
//   C.  replay: fk_replay_kernel, one 128-thread CTA per tile, one row per
//              thread.  Each tile first walks the tree from the root to its
//              leaf: the walk starts from dx_1 = -r_0 and, at each right
//              turn, applies the left sibling's aggregate to the vector
//              (every prefix from element 0 has matrix 0, so only vectors
//              are needed); this is the down-sweep, folded into the replay.
//              The tile then re-runs its leaves in FP64 from that vector
//              with the exact tridiagonal Jacobians, writes x + dx and
//              records the guard index.
// Aggregates are stored padded to 128 x 128, column-major (S[col][row]).
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "compose_tc.cuh"
#include "fpconv.cuh"
#include "solver.h"

namespace pitn {

constexpr int FD = 128;  // padded state dimension
constexpr int FK_TS = 64;  // elements per tile
constexpr int kFkMaxLevels = 40;  // tree levels (2^40 tiles: far above the step limit)

struct FkParams {
    const double* X;   // current iterate [N][d]
    const double* x0;  // [d]
    double* Xn;        // next iterate [N][d]
    double* r;         // residuals [N][d]
    float* rf;         // mixed precision: the residuals rounded to FP32 [N][d], the fold's and the
                       // replay's input (null for the FP64 scan)
    long long N;
    int d;
    int TS;
    long long q;       // lazy fill index of X
    long long T;       // tiles
    double h, Dc, o, cap;
    double a0;         // 1 - 2 o + h: the leaf diagonal is a0 - 2 h u
    double tol;
    int* stop;         // set on the device after the residual: converged or non-finite, so the
                       // scan and the update of this pass are skipped
    int rs;            // > 0: the fold runs scaled by o^-k, renormalised every rs steps (0: unscaled)
    double o_rs;       // o^rs
    unsigned long long cap_bits;  // bits of cap: |dz| bits above it are cut
    unsigned long long* res_bits;  // this iteration's slot
    int* nonfinite;
    unsigned long long* qenc;
    unsigned* cnt;     // up-sweep arrival counters, one per tree node (zero between passes)
    int L;             // levels of the aggregate tree above the tiles
    long long toff[kFkMaxLevels + 1];  // node offset of each level in S / b (level 0: the tiles)
};

__device__ __forceinline__ double fk_x(const FkParams& p, long long k, int i) {
    // state at buffer index k (x_{k+1}); k < 0 is x0; guard fill beyond q
    if (k < 0) return p.x0[i];
    if (k < p.q) return p.X[k * p.d + i];
    if (p.q > 0) return p.X[(p.q - 1) * p.d + i];
    return p.x0[i];
}

// Fold layout: each column of the tile aggregate is split over TPC threads
// of R rows each (registers); the shared-memory row of leaf coefficients is
// padded per segment so the TPC segments read in the same instruction fall in
// different banks.
template <typename Real> struct FoldTraits;
template <> struct FoldTraits<float> {
    static constexpr int R = 16, TPC = 8, PADR = 4, THREADS = FD * TPC;
};
template <> struct FoldTraits<double> {
    static constexpr int R = 32, TPC = 4, PADR = 2, THREADS = FD * TPC;
};
template <typename Real>
__host__ __device__ constexpr int fold_row_stride() {
    return FD + FoldTraits<Real>::TPC * FoldTraits<Real>::PADR;
}
template <typename Real>
__device__ __forceinline__ int pidx(int i) {
    return i + (i / FoldTraits<Real>::R) * FoldTraits<Real>::PADR;
}

__device__ __forceinline__ void fk_reduce_res(unsigned long long my_res, bool my_nf,
                                              const FkParams& p) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, my_res, off);
        my_res = o > my_res ? o : my_res;
    }
    bool nf = __any_sync(0xffffffffu, my_nf);
    if ((threadIdx.x & 31) == 0) {
        if (my_res) atomicMax(p.res_bits, my_res);
        if (nf) atomicOr(p.nonfinite, 1);
    }
}

// ---------------------------------------------------------------------------
// A0. residual (FP64) and leaf diagonals (working precision), one thread per
// entry, grid-stride: r_k = x_{k+1} - phi(x_k) (eq. 3.8) into p.r (and, for
// the mixed-precision scan, rounded to FP32 into p.rf), the diagonal 1 + e of
// J_k into a_out [N][128] (1 on padding rows), ||r||_inf.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) fk_residual_kernel(FkParams p, Real* __restrict__ a_out) {
    const int d = p.d;
    const long long total = p.N * FD;
    const Real hR = (Real)p.h, oR = (Real)p.o;
    unsigned long long my_res = 0ull;
    bool my_nf = false;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long k = idx / FD;
        const int i = (int)(idx - k * FD);
        Real a = (Real)1.0;
        if (i < d) {
            const double um = (i > 0) ? fk_x(p, k - 1, i - 1) : 0.0;
            const double u = fk_x(p, k - 1, i);
            const double up = (i < d - 1) ? fk_x(p, k - 1, i + 1) : 0.0;
            const double un = fk_x(p, k, i);
            const double f = fma(p.Dc, fma(-2.0, u, um) + up, fma(-u, u, u));   // D Lu + u (1 - u)
            const double rr = un - (u + p.h * f);
            // (an FP32 leaf takes u by the integer-pipe conversion: a hardware
            // F2F would issue on the FP64 pipe)
            if constexpr (std::is_same<Real, float>::value) {
                const float uR = d2f_int(u);
                a = 1.f + (hR * (1.f - 2.f * uR) - 2.f * oR);
            } else {
                a = fma(-2.0 * p.h, u, p.a0);   // one FP64 instruction, as in the replay
            }
            p.r[k * d + i] = rr;
            if constexpr (std::is_same<Real, float>::value) p.rf[k * d + i] = d2f_int(rr);
            const unsigned long long b = abs_bits(rr);
            my_res = b > my_res ? b : my_res;
            my_nf |= b >= kInfBitsAbs;
        }
        a_out[idx] = a;
    }
    fk_reduce_res(my_res, my_nf, p);
}

// The pass's decision, on the device: the scan and the update that follow in
// the stream return at once when the residual already meets tol (or is not
// finite), so the converged pass costs its residual only.
__global__ void fk_stop_kernel(FkParams p) {
    const double res = __longlong_as_double((long long)*p.res_bits);
    *p.stop = (*p.nonfinite != 0 || res <= p.tol) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// A. tile fold.  The threads own the 128 columns of P (TPC
// threads per column, R rows each, in registers); halo rows move by warp
// shuffles, so the fold needs no block barrier per step.  Warp 0 then folds
// the vector b (4 rows per lane).
//
// A leaf is L = diag(a) + o (sub + super) with one off-diagonal value o, so
// its product with P costs an add, a multiply and an FMA per entry.  With
// rs > 0 the fold carries P / o^k instead (k = steps since the last
// renormalisation): then (L P) / o^(k+1) = diag(a / o) P~ + (sub + super) P~,
// an add and an FMA per entry; every rs steps P~ is multiplied by o^rs, and
// at the end by o^k, so its magnitude stays within the working precision's
// range (rs is chosen on the host from |log2 o|).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(FoldTraits<Real>::THREADS, 1)
    fk_fold_kernel(FkParams p, const Real* __restrict__ a_in, Real* __restrict__ S_out,
                   Real* __restrict__ b_out) {
    using Tr = FoldTraits<Real>;
    constexpr int R = Tr::R, TPC = Tr::TPC;
    constexpr int FDP = fold_row_stride<Real>();
    extern __shared__ __align__(16) unsigned char smem[];
    Real* a_s = reinterpret_cast<Real*>(smem);            // [TS][FDP]  1 + e (leaf diagonal)
    Real* r_s = a_s + (size_t)p.TS * FDP;                  // [TS][FDP]  residual (for the vector fold)
    if (*p.stop) return;
    const long long t = blockIdx.x;
    const long long k0 = 1 + t * p.TS;
    const long long k1 = min(p.N, k0 + p.TS);
    const int len = (int)max(0LL, k1 - k0);
    const int d = p.d;

    // leaf diagonals (divided by o when the fold runs scaled) and residuals of
    // this tile's elements, staged in shared memory
    const bool scaled = p.rs > 0;
    const Real inv_o = scaled ? (Real)(1.0 / p.o) : (Real)1.0;
    for (int idx = threadIdx.x; idx < p.TS * FD; idx += blockDim.x) {
        const int s = idx / FD, i = idx - s * FD;
        Real a = (Real)1.0, rr = (Real)0.0;
        if (s < len) {
            const long long k = k0 + s;
            a = a_in[k * FD + i];
            if (i < d) {
                if constexpr (std::is_same<Real, float>::value) rr = p.rf[k * d + i];
                else rr = p.r[k * d + i];
            }
        }
        a_s[s * FDP + pidx<Real>(i)] = scaled ? a * inv_o : a;
        r_s[s * FDP + pidx<Real>(i)] = rr;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Real o = (Real)p.o;
    {
        const int j = threadIdx.x / TPC, part = threadIdx.x % TPC;
        const int row0 = part * R;
        const int sbase = pidx<Real>(row0);
        Real s[R];
#pragma unroll
        for (int i = 0; i < R; ++i) s[i] = (row0 + i == j) ? (Real)1.0 : (Real)0.0;
        const int nrow_live = max(0, min(R, d - row0));  // rows at or beyond d couple to nothing
        // the unscaled fold multiplies the neighbour sum by o; the scaled one by
        // 1 (live rows) -- with every row live, not at all
        const Real ow = scaled ? (Real)1.0 : o;
        const bool all_live = scaled && nrow_live == R;
        const Real o_rs = (Real)p.o_rs;
        int since = 0;                                   // steps since the last renormalisation
        auto fold_steps = [&](auto all_live_c) {
            constexpr bool kAllLive = decltype(all_live_c)::value;
            for (int st = 0; st < len; ++st) {
                // this thread's R leaf diagonals; in FP32 by 16-byte shared-memory
                // loads (the segment starts at a multiple of 16 bytes: FDP and sbase
                // are), 4x fewer load instructions for the FP32 pipe's fast steps
                Real a_reg[std::is_same<Real, float>::value ? R : 1];
                const Real* a = a_s + st * FDP + sbase;
                if constexpr (std::is_same<Real, float>::value) {
                    const uint4* src = reinterpret_cast<const uint4*>(a);
#pragma unroll
                    for (int v = 0; v < R / 4; ++v) {
                        const uint4 w = src[v];
                        a_reg[4 * v] = __uint_as_float(w.x);
                        a_reg[4 * v + 1] = __uint_as_float(w.y);
                        a_reg[4 * v + 2] = __uint_as_float(w.z);
                        a_reg[4 * v + 3] = __uint_as_float(w.w);
                    }
                    a = a_reg;
                }
                (void)a_reg;
                const Real above = __shfl_up_sync(0xffffffffu, s[R - 1], 1);
                const Real below = __shfl_down_sync(0xffffffffu, s[0], 1);
                const Real bot = (part < TPC - 1) ? below : (Real)0.0;
                Real prev = (part > 0) ? above : (Real)0.0;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const Real cur = s[i];
                    const Real nxt = (i < R - 1) ? s[i + 1] : bot;
                    if constexpr (kAllLive) {
                        s[i] = fma(cur, a[i], prev + nxt);
                    } else {
                        const Real oi = (i < nrow_live) ? ow : (Real)0.0;
                        s[i] = fma(cur, a[i], oi * (prev + nxt));
                    }
                    prev = cur;
                }
                if (scaled && ++since == p.rs) {
#pragma unroll
                    for (int i = 0; i < R; ++i) s[i] *= o_rs;
                    since = 0;
                }
            }
        };
        if (all_live) fold_steps(std::true_type{});
        else fold_steps(std::false_type{});
        Real tail = (Real)1.0;                           // o^since
        for (int c = 0; c < since; ++c) tail *= o;
        Real* col = S_out + ((size_t)t * FD + j) * FD + row0;
#pragma unroll
        for (int i = 0; i < R; ++i) col[i] = s[i] * tail - ((row0 + i == j) ? (Real)1.0 : (Real)0.0);
    }
    if (warp == 0) {
        // vector part of the aggregate, in the working precision
        Real b[4] = {(Real)0.0, (Real)0.0, (Real)0.0, (Real)0.0};
        const int r0 = 4 * lane;
        for (int st = 0; st < len; ++st) {
            const Real* a = a_s + st * FDP;
            const Real* rr = r_s + st * FDP;
            const Real up = __shfl_up_sync(0xffffffffu, b[3], 1);
            const Real dn = __shfl_down_sync(0xffffffffu, b[0], 1);
            Real prev = (lane == 0) ? (Real)0.0 : up;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const Real cur = b[i];
                const Real nxt = (i < 3) ? b[i + 1] : ((lane == 31) ? (Real)0.0 : dn);
                const Real ai = a[pidx<Real>(r0 + i)], ri = rr[pidx<Real>(r0 + i)];
                if (scaled) {   // a / o is staged: b' = o (a/o b + [live] (prev + nxt)) - r
                    const Real nb = (r0 + i < d) ? prev + nxt : (Real)0.0;
                    b[i] = fma(o, fma(ai, cur, nb), -ri);
                } else {
                    const Real oi = (r0 + i < d) ? o : (Real)0.0;
                    b[i] = ai * cur + oi * (prev + nxt) - ri;
                }
                prev = cur;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) b_out[(size_t)t * FD + r0 + i] = b[i];
    }
}

// ---------------------------------------------------------------------------
// B1. up-sweep composes.  Node m of the new level = child 2m+1 (later) o
// child 2m (earlier); a lone last child is copied.
// ---------------------------------------------------------------------------
struct LevelArgs {
    const void* S_in;   // child level aggregates
    const void* b_in;
    void* S_out;
    void* b_out;
    long long n_in;     // child count
    const int* stop;    // skip the level (converged pass)
};

// FP64: grid (nodes, 128 / CW): each CTA computes CW = 8 CPT columns of
// S2 + S1 + S2 S1 (thread (tm, tn): rows 4tm.., columns CPT tn..).  The host
// takes narrower column blocks on the levels near the root, where the nodes
// alone would leave most SMs idle.
template <int CPT>
__global__ void __launch_bounds__(256) fk_compose_f64(LevelArgs a) {
    constexpr int CW = 8 * CPT;
    extern __shared__ __align__(16) unsigned char smem[];
    double* As = reinterpret_cast<double*>(smem);   // [k][m] 128 x 128 (S2, column-major copy)
    double* Bs = As + FD * FD;                      // [n][k] CW x 128  (S1 columns)
    const long long m = blockIdx.x;
    const int cb = blockIdx.y;
    const double* Sin = (const double*)a.S_in;
    const double* bin = (const double*)a.b_in;
    double* Sout = (double*)a.S_out;
    double* bout = (double*)a.b_out;
    if (*a.stop) return;
    const long long ce = 2 * m, cl = 2 * m + 1;
    const double* S1 = Sin + (size_t)ce * FD * FD;
    double* So = Sout + (size_t)m * FD * FD;
    if (cl >= a.n_in) {  // copy
        for (int idx = threadIdx.x; idx < CW * FD; idx += blockDim.x)
            So[(size_t)cb * CW * FD + idx] = S1[(size_t)cb * CW * FD + idx];
        if (cb == 0)
            for (int i = threadIdx.x; i < FD; i += blockDim.x) bout[m * FD + i] = bin[ce * FD + i];
        return;
    }
    const double* S2 = Sin + (size_t)cl * FD * FD;
    for (int idx = threadIdx.x; idx < FD * FD; idx += blockDim.x) As[idx] = S2[idx];
    for (int idx = threadIdx.x; idx < CW * FD; idx += blockDim.x) Bs[idx] = S1[(size_t)cb * CW * FD + idx];
    __syncthreads();
    const int tm = threadIdx.x & 31, tn = threadIdx.x >> 5;
    double acc[4][CPT];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < CPT; ++y) acc[x][y] = 0.0;
#pragma unroll 4
    for (int k = 0; k < FD; ++k) {
        double av[4], bv[CPT];
#pragma unroll
        for (int x = 0; x < 4; ++x) av[x] = As[k * FD + 4 * tm + x];
#pragma unroll
        for (int y = 0; y < CPT; ++y) bv[y] = Bs[(CPT * tn + y) * FD + k];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < CPT; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < CPT; ++y) {
        const int n = cb * CW + CPT * tn + y;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int mm = 4 * tm + x;
            So[(size_t)n * FD + mm] = As[n * FD + mm] + Bs[(CPT * tn + y) * FD + mm] + acc[x][y];
        }
    }
    if (cb == 0 && threadIdx.x < FD) {
        // b = b2 + b1 + S2 b1
        const int i = threadIdx.x;
        const double* b1 = bin + ce * FD;
        double s = bin[cl * FD + i] + b1[i];
        for (int k = 0; k < FD; ++k) s = fma(As[k * FD + i], b1[k], s);
        bout[m * FD + i] = s;
    }
}

// Mixed, tensor cores of the 5th generation: one CTA of 256 threads per
// compose (see compose_tc.cuh); a lone last child is copied.
struct CombineArgs {
    const float* S2; const float* b2;  // later elements (stride FD*FD / FD)
    const float* S1; const float* b1;  // earlier elements
    float* S; float* b;                // results
    long long n;                       // composes
    long long stride_in;               // element stride of the inputs in matrices (2 for tree levels)
    long long n_lone;                  // index of a lone earlier element to copy (or -1)
    int* err;
    const int* stop;                   // nullable: skip the launch when set (converged pass)
    unsigned long long load_polls, mma_polls;  // wait bounds of the compose
};

// Operand precision of the tensor-core composes: BF16 (operands converted,
// bulk copies for fresh inputs) or TF32 (FP32 aggregates as they stand).
struct TcBf16 {
    using Smem = tc::ComposeSmem;
    static constexpr size_t kSmem = sizeof(Smem) + 1024;
    static __device__ __forceinline__ int compose(Smem& sm, const float* S2, const float* b2, const float* S1,
                                                  const float* b1, float* So, float* bo, uint32_t phase,
                                                  bool bulk, uint64_t lp, uint64_t mp) {
        return tc::compose_tc(sm, S2, b2, S1, b1, So, bo, phase, bulk, lp, mp);
    }
};
struct TcTf32 {
    using Smem = tc::ComposeSmem32;
    static constexpr size_t kSmem = sizeof(Smem) + 1024;
    static __device__ __forceinline__ int compose(Smem& sm, const float* S2, const float* b2, const float* S1,
                                                  const float* b1, float* So, float* bo, uint32_t phase, bool,
                                                  uint64_t, uint64_t mp) {
        return tc::compose_tc32(sm, S2, b2, S1, b1, So, bo, phase, mp);
    }
};

template <class Op>
__global__ void __launch_bounds__(256) fk_compose_tc_kernel(CombineArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    typename Op::Smem& sm =
        *reinterpret_cast<typename Op::Smem*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const long long m = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t MM = (size_t)FD * FD;
    if (a.stop && *a.stop) return;
    if (m == a.n_lone) {  // copy the lone earlier element
        const float4* src = reinterpret_cast<const float4*>(a.S1 + (size_t)m * a.stride_in * MM);
        float4* dst = reinterpret_cast<float4*>(a.S + (size_t)m * MM);
        for (int i = tid; i < (int)(MM / 4); i += blockDim.x) dst[i] = src[i];
        if (tid < FD) a.b[m * FD + tid] = a.b1[m * a.stride_in * FD + tid];
        return;
    }
    if (warp == 0) tc::tmem_alloc(&sm.tmem, FD);
    tc::init_barriers(sm);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const int rc = Op::compose(sm, a.S2 + (size_t)m * a.stride_in * MM, a.b2 + m * a.stride_in * FD,
                               a.S1 + (size_t)m * a.stride_in * MM, a.b1 + m * a.stride_in * FD,
                               a.S + (size_t)m * MM, a.b + m * FD, 0u, true, a.load_polls, a.mma_polls);
    if (rc != tc::kTcOk && tid == 0) raise_error(a.err, PITN_ETIMEOUT);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    // an operation still in flight keeps the TMEM it writes (kTcStuck)
    if (rc != tc::kTcStuck && warp == 0) tc::tmem_dealloc(sm.tmem, FD);
}

// The whole up-sweep of the mixed-precision tree in one launch: one CTA per
// level-1 node.  A CTA composes its node, then climbs: it counts itself in
// the parent's arrival counter, and the second of the two children to
// arrive composes the parent (a lone child's CTA climbs without counting).
// The first to arrive leaves, so no CTA ever waits on another.  Inputs that
// another CTA wrote are read through L2 after the counter's acquire; the
// second arrival resets the counter for the next pass.  The climb stops
// below the root, whose aggregate nothing reads.
struct UpArgs {
    float* S;
    float* b;
    long long off[kFkMaxLevels + 1];
    long long n[kFkMaxLevels + 1];
    int L;
    unsigned* cnt;   // one arrival counter per node, indexed like S / b
    int* err;
    const int* stop;
    unsigned long long load_polls, mma_polls;  // wait bounds of the composes
};

template <class Op>
__global__ void __launch_bounds__(256) fk_upsweep_tc_kernel(UpArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    typename Op::Smem& sm =
        *reinterpret_cast<typename Op::Smem*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    __shared__ int s_go;
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t MM = (size_t)FD * FD;
    if (*a.stop) return;
    if (warp == 0) tc::tmem_alloc(&sm.tmem, FD);
    tc::init_barriers(sm);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    long long m = blockIdx.x;
    unsigned composes = 0;
    int rc = tc::kTcOk;
    for (int lv = 1; lv < a.L; ++lv) {
        const long long n_in = a.n[lv - 1];
        const float* Sin = a.S + (size_t)a.off[lv - 1] * MM;
        const float* bin = a.b + (size_t)a.off[lv - 1] * FD;
        float* So = a.S + (size_t)(a.off[lv] + m) * MM;
        float* bo = a.b + (size_t)(a.off[lv] + m) * FD;
        if ((n_in & 1) && m == n_in / 2) {
            // lone earlier child (written by an earlier launch or by this CTA)
            const float4* __restrict__ src = reinterpret_cast<const float4*>(Sin + (size_t)(2 * m) * MM);
            float4* __restrict__ dst = reinterpret_cast<float4*>(So);
            constexpr int U = 4;   // loads in flight per thread
            for (int i0 = tid; i0 < (int)(MM / 4); i0 += U * blockDim.x) {
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i < (int)(MM / 4)) v[u] = __ldcg(src + i);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u * blockDim.x;
                    if (i < (int)(MM / 4)) dst[i] = v[u];
                }
            }
            if (tid < FD) bo[tid] = __ldcg(bin + (2 * m) * FD + tid);
        } else {
            rc = Op::compose(sm, Sin + (size_t)(2 * m + 1) * MM, bin + (2 * m + 1) * FD,
                             Sin + (size_t)(2 * m) * MM, bin + (2 * m) * FD, So, bo, composes & 1u, lv == 1,
                             a.load_polls, a.mma_polls);
            ++composes;
            if (rc != tc::kTcOk) {   // uniform over the CTA: the compose decides CTA-wide
                if (tid == 0) raise_error(a.err, PITN_ETIMEOUT);
                break;               // this node is not written: no parent can be composed
            }
        }
        if (lv + 1 >= a.L) break;
        // release this node, then climb if both children of the parent are done
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            int go = 1;
            const long long n_here = a.n[lv];
            if (!((n_here & 1) && m == n_here - 1)) {
                unsigned* c = a.cnt + a.off[lv + 1] + m / 2;
                go = (atomicAdd(c, 1u) == 1u) ? 1 : 0;
                if (go) {
                    *c = 0u;
                    __threadfence();
                }
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        m >>= 1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (rc != tc::kTcStuck && warp == 0) tc::tmem_dealloc(sm.tmem, FD);
}

// ---------------------------------------------------------------------------
// B2. down-sweep, inside the replay: the incoming vector of tile t follows the
// path from the root to the leaf.  The root's is -r_0 (dx_1 = -h_1, the head
// element a_0 = (0, -r_0)); going down to a left child keeps it, going down to
// a right child c applies the left sibling's aggregate:
// z <- z + S_{c-1} z + b_{c-1} (the operator of eq. 3.3 in the delta form).
// Each of the FD threads owns one row; the row's dot product runs as
// kDownParts partial chains over quarters of k, added in order, so the
// result does not depend on which tile computes a node's vector.
// ---------------------------------------------------------------------------
constexpr int kDownParts = 4;

template <typename Real>
__device__ __forceinline__ Real fk_tile_z(const FkParams& p, const Real* __restrict__ S,
                                          const Real* __restrict__ b, long long t, int row, Real* zs) {
    Real z = (row < p.d) ? (Real)(-p.r[row]) : (Real)0.0;
    for (int lv = p.L; lv >= 1; --lv) {
        const long long c = t >> (lv - 1);
        if (!(c & 1)) continue;
        const long long node = p.toff[lv - 1] + c - 1;
        const Real* Sn = S + (size_t)node * FD * FD;
        __syncthreads();   // zs may still be read from the previous right turn
        zs[row] = z;
        __syncthreads();
        constexpr int KP = FD / kDownParts;
        Real part[kDownParts];
#pragma unroll
        for (int pt = 0; pt < kDownParts; ++pt) part[pt] = 0;
#pragma unroll 8
        for (int k = 0; k < KP; ++k) {
#pragma unroll
            for (int pt = 0; pt < kDownParts; ++pt)
                part[pt] = fma(Sn[(size_t)(pt * KP + k) * FD + row], zs[pt * KP + k], part[pt]);
        }
        Real tz = z + b[(size_t)node * FD + row];
#pragma unroll
        for (int pt = 0; pt < kDownParts; ++pt) tz += part[pt];
        z = tz;
    }
    return z;
}

// ---------------------------------------------------------------------------
// C. replay: one CTA of 128 threads per tile, one row per thread.  Neighbour
// rows come from the same warp by shuffles and, at the four warps' edges,
// through shared memory (a slot per step parity and one block barrier per
// step).  The recursion runs in the scan's working precision Real: FP64 for
// the FP64 scan (exact leaves); FP32 for the mixed-precision scans, whose
// composes already make the Newton step inexact -- there it takes the FP32
// leaf diagonals and residuals the residual kernel wrote (the fold's inputs),
// and the FP32 correction is added to the FP64 state exactly (the update
// stays FP64).  A warp's FP64 instruction holds its FP64 unit for ~70 cycles
// on this part: the FP64 recursion spends five per entry and step, the FP32
// one a single addition.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(FD) fk_replay_kernel(FkParams p, const Real* __restrict__ S,
                                                       const Real* __restrict__ b,
                                                       const Real* __restrict__ a_in) {
    if (*p.stop) return;
    constexpr bool kF32 = std::is_same<Real, float>::value;
    __shared__ Real s_edge[2][2][4];   // [parity][first / last lane][warp]
    __shared__ Real s_z[FD];
    const int row = threadIdx.x, warp = row >> 5, lane = row & 31;
    const long long t = blockIdx.x;
    const int d = p.d;
    const bool live = row < d;
    const long long k0 = 1 + t * p.TS;
    const long long k1 = min(p.N, k0 + p.TS);
    unsigned long long my_q = 0ull;
    // |dz| beyond the cut bound (or not finite) cuts the step; in FP32 the
    // bound is at most the largest finite float, so an overflow to
    // infinity is caught
    const float capf = (float)fmin(p.cap, (double)FLT_MAX);
    auto cut = [&](Real v) -> bool {
        if constexpr (kF32) return !(fabsf(v) <= capf);
        else return abs_bits(v) > p.cap_bits;
    };
    auto to_double = [](Real v) -> double {
        if constexpr (kF32) return f2d_int(v);
        else return v;
    };
    Real z = fk_tile_z<Real>(p, S, b, t, row, s_z);
    if (!live) z = (Real)0;
    double xprev = live ? fk_x(p, k0 - 1, row) : 0.0;
    if (t == 0 && live) {
        // element 0: dx_1 = -r_0 (already the incoming vector of tile 0)
        if (cut(z)) my_q = ~0ull;  // ~0 = index 0
        p.Xn[row] = xprev + to_double(z);
    }
    const Real m2h = (Real)(-2.0 * p.h), a0 = (Real)p.a0, o = (Real)p.o;
    // steps in groups of G: the loads of a group are issued together so their
    // latency overlaps; the recurrence itself is serial in k
    constexpr int G = 4;
    int par = 0;
    for (long long kg = k0; kg < k1; kg += G) {
        double xc[G];
        Real rk[G], ak[G];
#pragma unroll
        for (int gq = 0; gq < G; ++gq) {
            const long long k = kg + gq;
            const bool ld = (k < k1) && live;
            xc[gq] = ld ? fk_x(p, k, row) : 0.0;
            if constexpr (kF32) {
                rk[gq] = ld ? p.rf[k * d + row] : 0.f;
                ak[gq] = ld ? a_in[k * FD + row] : 0.f;
            } else {
                rk[gq] = ld ? p.r[k * d + row] : 0.0;
                ak[gq] = 0.0;
            }
        }
#pragma unroll
        for (int gq = 0; gq < G; ++gq) {
            const long long k = kg + gq;
            if (k >= k1) break;
            // dz_{k+1} = J_k dz_k - r_k with J_k = diag(a0 - 2 h x_k) + o (sub + super)
            if (lane == 0) s_edge[par][0][warp] = z;
            if (lane == 31) s_edge[par][1][warp] = z;
            __syncthreads();
            Real up = __shfl_up_sync(0xffffffffu, z, 1);
            Real dn = __shfl_down_sync(0xffffffffu, z, 1);
            if (lane == 0) up = (warp > 0) ? s_edge[par][1][warp - 1] : (Real)0;
            if (lane == 31) dn = (warp < 3) ? s_edge[par][0][warp + 1] : (Real)0;
            par ^= 1;
            // leaf diagonal a0 - 2 h x_k (FP64: from the state; FP32: as staged)
            Real a;
            if constexpr (kF32) a = ak[gq];
            else a = fma(m2h, xprev, a0);
            const Real nz = live ? fma(a, z, fma(o, up + dn, -rk[gq])) : (Real)0;
            z = nz;
            if (live) {
                if (cut(z)) {
                    const unsigned long long e = ~(unsigned long long)k;
                    my_q = e > my_q ? e : my_q;
                }
                p.Xn[k * d + row] = xc[gq] + to_double(z);
            }
            xprev = xc[gq];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, my_q, off);
        my_q = o2 > my_q ? o2 : my_q;
    }
    if (lane == 0 && my_q) atomicMax(p.qenc, my_q);
}

// Final iterate with its fill into the destination.
__global__ void fk_finalize_kernel(const double* __restrict__ X, const double* __restrict__ x0,
                                   double* __restrict__ out, long long N, int d, long long q,
                                   int skip_prefix) {
    const long long total = N * d;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long k = idx / d;
        const int i = (int)(idx - k * d);
        if (skip_prefix && k < q) continue;
        double v;
        if (k < q) v = X[k * d + i];
        else if (q > 0) v = X[(q - 1) * d + i];
        else v = x0[i];
        out[idx] = v;
    }
}

}  // namespace pitn

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
namespace pitn_host {

using namespace pitn;

namespace {
template <typename Real>
size_t fold_smem_bytes(int TS) {
    return 2 * sizeof(Real) * (size_t)TS * fold_row_stride<Real>();
}

struct Tree {
    std::vector<long long> n;    // nodes per level
    std::vector<long long> off;  // node offset of each level
    long long total = 0;
};

Tree make_tree(long long T) {
    Tree tr;
    long long n = T;
    tr.n.push_back(n);
    tr.off.push_back(0);
    tr.total = n;
    while (n > 1) {
        n = (n + 1) / 2;
        tr.off.push_back(tr.total);
        tr.n.push_back(n);
        tr.total += n;
    }
    return tr;
}

template <typename Real>
int run_iteration(FkParams& p, const Tree& tr, Real* S, Real* b, Real* abuf, bool mixed,
                  int* err, cudaStream_t st, bool residual_only, bool tf32) {
    const size_t smemA = fold_smem_bytes<Real>(p.TS);
    {
        auto tok = timed_begin("fkpp_residual", st);
        const long long total = p.N * FD;
        const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
        fk_residual_kernel<Real><<<grid, 256, 0, st>>>(p, abuf);
        timed_end(tok, st);
        count_launch(1);
    }
    if (residual_only) return cudaGetLastError() == cudaSuccess ? PITN_OK : PITN_ECUDA;
    fk_stop_kernel<<<1, 1, 0, st>>>(p);
    count_launch(1);
    {
        auto tok = timed_begin("fkpp_fold", st);
        fk_fold_kernel<Real><<<(unsigned)p.T, FoldTraits<Real>::THREADS, smemA, st>>>(p, abuf, S, b);
        timed_end(tok, st);
        count_launch(1);
    }
    // up-sweep, levels 1 .. L-1 (the root's aggregate is never read: the
    // replay's walk applies only left siblings)
    const int L = (int)tr.n.size() - 1;
    if (mixed) {
        if (L >= 2) {
            UpArgs ua;
            ua.S = reinterpret_cast<float*>(S);
            ua.b = reinterpret_cast<float*>(b);
            for (int lv = 0; lv <= L; ++lv) {
                ua.off[lv] = tr.off[lv];
                ua.n[lv] = tr.n[lv];
            }
            ua.L = L;
            ua.cnt = p.cnt;
            ua.err = err;
            ua.stop = p.stop;
            ua.load_polls = wait_limits().load_polls;
            ua.mma_polls = wait_limits().mma_polls;
            auto tok = timed_begin("fkpp_compose", st);
            if (tf32) fk_upsweep_tc_kernel<TcTf32><<<(unsigned)tr.n[1], 256, TcTf32::kSmem, st>>>(ua);
            else fk_upsweep_tc_kernel<TcBf16><<<(unsigned)tr.n[1], 256, TcBf16::kSmem, st>>>(ua);
            timed_end(tok, st);
            count_launch(1);
        }
    } else {
        for (int lv = 1; lv < L; ++lv) {
            LevelArgs la;
            la.S_in = S + (size_t)tr.off[lv - 1] * FD * FD;
            la.b_in = b + (size_t)tr.off[lv - 1] * FD;
            la.S_out = S + (size_t)tr.off[lv] * FD * FD;
            la.b_out = b + (size_t)tr.off[lv] * FD;
            la.n_in = tr.n[lv - 1];
            la.stop = p.stop;
            auto tok = timed_begin("fkpp_compose", st);
            // column block per CTA: enough CTAs for two per SM where the level allows
            const long long nodes = tr.n[lv];
            const int cpt = nodes >= 76 ? 4 : (nodes >= 19 ? 2 : 1);
            const size_t sm = (size_t)(FD * FD + 8 * cpt * FD) * sizeof(double);
            const dim3 grid((unsigned)nodes, (unsigned)(FD / (8 * cpt)));
            if (cpt == 4) fk_compose_f64<4><<<grid, 256, sm, st>>>(la);
            else if (cpt == 2) fk_compose_f64<2><<<grid, 256, sm, st>>>(la);
            else fk_compose_f64<1><<<grid, 256, sm, st>>>(la);
            timed_end(tok, st);
            count_launch(1);
        }
    }
    {
        auto tok = timed_begin("fkpp_replay", st);
        fk_replay_kernel<Real><<<(unsigned)p.T, FD, 0, st>>>(p, S, b, abuf);
        timed_end(tok, st);
        count_launch(1);
    }
    return cudaGetLastError() == cudaSuccess ? PITN_OK : PITN_ECUDA;
}

template <typename Real>
int fkpp_solve_t(const SolveIO& io, double h, int64_t N, int d, double tol, int max_iter,
                 const pitn_options& o, cudaStream_t st, SolveOutcome* out, bool mixed) {
    // Tile length: FK_TS steps, shortened once there is at least one full wave
    // of tiles so that the tile count is a whole number of waves of the fold
    // (one CTA per tile; the replay has one per tile too).
    int TS = FK_TS;
    {
        const int smem0 = (int)fold_smem_bytes<Real>(FK_TS);
        int per_sm = 0;
        if (cudaFuncSetAttribute(fk_fold_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem0) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fk_fold_kernel<Real>,
                                                          FoldTraits<Real>::THREADS, smem0) == cudaSuccess &&
            per_sm > 0) {
            const long long slots = (long long)per_sm * props().multiProcessorCount;
            const long long T0 = (N - 1 + FK_TS - 1) / FK_TS;
            if (T0 >= slots) {
                const long long Tw = (T0 + slots - 1) / slots * slots;
                TS = (int)((N - 1 + Tw - 1) / Tw);
            }
        }
        cudaGetLastError();
    }
    const long long T = std::max(1LL, (long long)((N - 1 + TS - 1) / TS));
    Tree tr = make_tree(T);
    // scratch: X1 | r ; aggregates S | b ; control
    const size_t nd = (size_t)N * d;
    double* X1 = (double*)workspace(nd * sizeof(double) * 2, kSlotX1);
    if (!X1) return PITN_ENOMEM;
    double* r = X1 + nd;
    const size_t aggBytes = (size_t)tr.total * FD * FD * sizeof(Real) + (size_t)tr.total * FD * sizeof(Real);
    Real* S = (Real*)workspace(aggBytes, kSlotAux);
    // leaf diagonals [N][128] in the working precision, and for the mixed
    // scan the FP32 residuals [N][d] after them
    Real* abuf = (Real*)workspace((size_t)N * FD * sizeof(Real) + (mixed ? nd * sizeof(float) : 0), kSlotAux2);
    if (!S || !abuf) return PITN_ENOMEM;
    Real* b = S + (size_t)tr.total * FD * FD;
    // per-pass slots | up-sweep arrival counters | stop flag and error word
    const size_t cntOff = ((size_t)(max_iter + 1) * (8 + 8 + 4) + 15) & ~(size_t)15;
    const size_t ctrlBytes = cntOff + (((size_t)tr.total * sizeof(unsigned) + 15) & ~(size_t)15) + 64;
    char* ctrl = (char*)workspace(ctrlBytes, kSlotCtrl);
    if (!ctrl) return PITN_ENOMEM;
    unsigned long long* res_bits = (unsigned long long*)ctrl;
    unsigned long long* qenc = res_bits + (max_iter + 1);
    int* nonfinite = (int*)(qenc + (max_iter + 1));
    int* err_d = (int*)(ctrl + ctrlBytes - 16);
    int* stop_d = (int*)(ctrl + ctrlBytes - 32);
    if (cudaMemsetAsync(ctrl, 0, ctrlBytes, st) != cudaSuccess) return PITN_ECUDA;
    struct HostCtl { unsigned long long res, q; int nf; int err; };
    HostCtl* hc = (HostCtl*)pinned(sizeof(HostCtl));
    if (!hc) return PITN_ENOMEM;

    {
        const int smemA = (int)fold_smem_bytes<Real>(TS);
        cudaFuncSetAttribute(fk_fold_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemA);
        cudaFuncSetAttribute(fk_compose_f64<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((FD * FD + 32 * FD) * sizeof(double)));
        cudaFuncSetAttribute(fk_compose_f64<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((FD * FD + 16 * FD) * sizeof(double)));
        cudaFuncSetAttribute(fk_compose_f64<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((FD * FD + 8 * FD) * sizeof(double)));
        cudaFuncSetAttribute(fk_upsweep_tc_kernel<TcBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcBf16::kSmem);
        cudaFuncSetAttribute(fk_upsweep_tc_kernel<TcTf32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcTf32::kSmem);
    }

    const bool guarded = o.guard_B > 0.0 && std::isfinite(o.guard_B);
    FkParams p{};
    p.x0 = io.x0_dev;
    p.r = r;
    p.rf = mixed ? reinterpret_cast<float*>(abuf + (size_t)N * FD) : nullptr;
    p.N = N;
    p.d = d;
    p.TS = TS;
    p.T = T;
    const double dx = 1.0 / (double)(d + 1);
    p.h = h;
    p.Dc = io.params[0] / (dx * dx);
    p.o = h * p.Dc;
    p.a0 = 1.0 - 2.0 * p.o + h;
    // scaled fold (see fk_fold_kernel): renormalise before the scaled product
    // can move more than ~100 (FP32) / ~900 (FP64) binary orders of magnitude
    p.rs = 0;
    p.o_rs = 1.0;
    if (std::isnormal(p.o) && std::isnormal(1.0 / p.o)) {
        const double bits_per_step = std::fabs(std::log2(p.o)) + 2.0;
        const double budget = std::is_same<Real, float>::value ? 100.0 : 900.0;
        p.rs = (int)std::max(1.0, std::min((double)TS, std::floor(budget / bits_per_step)));
        p.o_rs = std::pow(p.o, p.rs);
    }
    p.cap = guarded ? o.guard_B : DBL_MAX;
    p.tol = tol;
    p.stop = stop_d;
    p.cnt = (unsigned*)(ctrl + cntOff);
    std::memcpy(&p.cap_bits, &p.cap, sizeof(p.cap));
    if ((int)tr.n.size() - 1 > kFkMaxLevels) return PITN_EINVAL;
    p.L = (int)tr.n.size() - 1;
    for (int lv = 0; lv <= p.L; ++lv) p.toff[lv] = tr.off[lv];
    double* bufs[2] = {io.traj_dev, X1};
    int cur = 0;
    long long q = io.have_guess ? N : 0;
    long long last_cut = N;
    int it = 0, status = PITN_NOT_CONVERGED;
    double final_res = 0.0;
    out->history.clear();
    out->cuts.clear();
    for (;;) {
        p.X = bufs[cur];
        p.Xn = bufs[cur ^ 1];
        p.q = q;
        p.res_bits = res_bits + it;
        p.qenc = qenc + it;
        p.nonfinite = nonfinite + it;
        int rc = run_iteration<Real>(p, tr, S, b, abuf, mixed, err_d, st, it == max_iter,
                                     o.precision == PITN_PREC_MIXED_TF32);
        if (rc != PITN_OK) return rc;
        if (cudaMemcpyAsync(&hc->res, res_bits + it, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&hc->q, qenc + it, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&hc->nf, nonfinite + it, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&hc->err, err_d, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return PITN_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
        if (hc->err) return hc->err;
        double res;
        std::memcpy(&res, &hc->res, sizeof(res));
        const long long cut = hc->q ? (long long)(~hc->q) : (long long)N;
        out->history.push_back(res);
        final_res = res;
        if (hc->nf) { status = PITN_NONFINITE; break; }
        if (res <= tol) { status = PITN_OK; break; }
        if (it == max_iter) { status = PITN_NOT_CONVERGED; break; }
        out->cuts.push_back(cut);
        if (!guarded && cut < N) { status = PITN_NONFINITE; break; }
        cur ^= 1;
        q = guarded ? cut : N;
        last_cut = cut;
        ++it;
    }
    // materialise the final iterate (buffer + guard fill) into the trajectory
    const double* Xc = bufs[cur];
    const bool same = (Xc == io.traj_dev);
    if (!same || q < N) {
        fk_finalize_kernel<<<1024, 256, 0, st>>>(Xc, io.x0_dev, io.traj_dev, N, d, q, same ? 1 : 0);
        count_launch(1);
        if (cudaGetLastError() != cudaSuccess) return PITN_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
    out->iters = it;
    out->status = status;
    out->final_res = final_res;
    out->guard_index = last_cut;
    return PITN_OK;
}
}  // namespace

int fkpp_solve(const SolveIO& io, double h, int64_t N, int d, double tol, int max_iter,
               const pitn_options& o, cudaStream_t st, SolveOutcome* out) {
    if (d > FD) return PITN_EINVAL;
    if (o.precision == PITN_PREC_MIXED_BF16 || o.precision == PITN_PREC_MIXED_TF32) {
        if (d < 64) return PITN_EINVAL;
        return fkpp_solve_t<float>(io, h, N, d, tol, max_iter, o, st, out, true);
    }
    return fkpp_solve_t<double>(io, h, N, d, tol, max_iter, o, st, out, false);
}

}  // namespace pitn_host

// ---------------------------------------------------------------------------
// C-ABI primitive: n independent dense delta-form combines on tensor cores.
// ---------------------------------------------------------------------------
namespace {
template <class Op>
int combine_delta(int64_t n, const float* S2, const float* b2, const float* S1, const float* b1, float* S,
                  float* b, void* stream) {
    using namespace pitn;
    using namespace pitn_host;
    if (n < 1 || !S2 || !b2 || !S1 || !b1 || !S || !b) return PITN_EINVAL;
    if (!is_device_ptr(S2) || !is_device_ptr(b2) || !is_device_ptr(S1) || !is_device_ptr(b1) ||
        !is_device_ptr(S) || !is_device_ptr(b))
        return PITN_EINVAL;
    if (((uintptr_t)S2 | (uintptr_t)S1 | (uintptr_t)S) & 15) return PITN_EINVAL;
    if (any_foreign({S2, b2, S1, b1, S, b})) return PITN_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(api_mutex());
    cudaStream_t st = (cudaStream_t)stream;
    int* err = (int*)workspace(64, kSlotCtrl);
    if (!err) return PITN_ENOMEM;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return PITN_ECUDA;
    cudaFuncSetAttribute(fk_compose_tc_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Op::kSmem);
    CombineArgs ca;
    ca.S2 = S2; ca.b2 = b2; ca.S1 = S1; ca.b1 = b1; ca.S = S; ca.b = b;
    ca.n = n; ca.stride_in = 1; ca.n_lone = -1; ca.err = err; ca.stop = nullptr;
    ca.load_polls = wait_limits().load_polls;
    ca.mma_polls = wait_limits().mma_polls;
    auto tok = timed_begin("fkpp_compose", st);
    fk_compose_tc_kernel<Op><<<(unsigned)n, 256, Op::kSmem, st>>>(ca);
    timed_end(tok, st);
    count_launch(1);
    if (cudaGetLastError() != cudaSuccess) return PITN_ECUDA;
    int h_err = 0;
    if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PITN_ECUDA;
    return h_err ? h_err : PITN_OK;
}
}  // namespace

extern "C" int pitn_affine_combine_delta(int64_t n, const float* S2, const float* b2, const float* S1,
                                         const float* b1, float* S, float* b, void* stream) {
    return combine_delta<pitn::TcBf16>(n, S2, b2, S1, b1, S, b, stream);
}

extern "C" int pitn_affine_combine_delta_tf32(int64_t n, const float* S2, const float* b2, const float* S1,
                                              const float* b1, float* S, float* b, void* stream) {
    return combine_delta<pitn::TcTf32>(n, S2, b2, S1, b1, S, b, stream);
}
