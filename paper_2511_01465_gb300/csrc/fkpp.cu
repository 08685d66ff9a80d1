// fkpp.cu -- Newton solve for the Fisher-KPP method-of-lines systems
// (d >= 3 interior nodes, d <= 128), FP64 or mixed precision.
//
// The step map is phi(u) = u + h f(u) with f_i = D (u_{i-1} - 2u_i + u_{i+1})/dx^2
// + u_i (1 - u_i), so the Jacobian of every leaf element is tridiagonal:
//   J_k = I + S_k,  S_k = h (D L/dx^2 + diag(1 - 2 u_k)),
// diagonal a_i = 1 + h (1 - 2 u_i) - 2 o and off-diagonals o = h D / dx^2.
// The Newton step (eq. 3.13) is solved as a reduce-then-scan:
//   A. fold:   one CTA per tile of TS consecutive elements computes the
//              residuals (eq. 3.8, with ||r||_inf) and folds the tile's leaves
//              P <- J_k P, b <- J_k b - r_k into a dense tile aggregate
//              (P = I + S, b); the tridiagonal leaf is applied as a stencil,
//              so the fold costs 3 d^2 per element instead of 2 d^3;
//   B. tree:   an up-sweep composes pairs of aggregates (eq. 3.3),
//              (I + S2)(I + S1) = I + (S2 + S1 + S2 S1),  b = b2 + b1 + S2 b1,
//              the dense S2 S1 product in FP64 on CUDA cores, or in mixed
//              precision on tensor cores (BF16 operands, FP32 accumulation,
//              sums in FP32; the delta form keeps the identity exact); a
//              down-sweep then pushes the prefix vector dx (the root starts
//              at dx_1 = -r_0) to the start of every tile with matrix-vector
//              products only (every prefix from element 0 has matrix 0);
//   C. replay: one warp per tile re-runs the tile's leaves in FP64 from its
//              incoming vector with the exact Jacobians, writes x + dx and
//              records the guard index.
// Aggregates are stored padded to 128 x 128, column-major (S[col][row]).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "solver.h"

namespace pitn {

constexpr int FD = 128;  // padded state dimension
constexpr int FK_TS = 64;  // elements per tile

struct FkParams {
    const double* X;   // current iterate [N][d]
    const double* x0;  // [d]
    double* Xn;        // next iterate [N][d]
    double* r;         // residuals [N][d]
    long long N;
    int d;
    int TS;
    long long q;       // lazy fill index of X
    long long T;       // tiles
    double h, Dc, o, cap;
    unsigned long long* res_bits;  // this iteration's slot
    int* nonfinite;
    unsigned long long* qenc;
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
    static constexpr int R = 32, TPC = 4, PADR = 8, THREADS = FD * TPC;
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
// A. residual + tile fold.  The threads own the 128 columns of P (TPC
// threads per column, R rows each, in registers); halo rows move by warp
// shuffles, so the fold needs no block barrier per step.  Warp 0 then folds
// the vector b (4 rows per lane).
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(FoldTraits<Real>::THREADS, 1)
    fk_fold_kernel(FkParams p, Real* __restrict__ S_out, Real* __restrict__ b_out) {
    using Tr = FoldTraits<Real>;
    constexpr int R = Tr::R, TPC = Tr::TPC;
    constexpr int FDP = fold_row_stride<Real>();
    extern __shared__ __align__(16) unsigned char smem[];
    Real* a_s = reinterpret_cast<Real*>(smem);            // [TS][FDP]  1 + e (leaf diagonal)
    Real* r_s = a_s + (size_t)p.TS * FDP;                  // [TS][FDP]  residual (for the vector fold)
    const long long t = blockIdx.x;
    const long long k0 = 1 + t * p.TS;
    const long long k1 = min(p.N, k0 + p.TS);
    const int len = (int)max(0LL, k1 - k0);
    const int d = p.d;

    unsigned long long my_res = 0ull;
    bool my_nf = false;
    const Real hR = (Real)p.h, oR = (Real)p.o;
    for (int idx = threadIdx.x; idx < p.TS * FD; idx += blockDim.x) {
        const int s = idx / FD, i = idx - s * FD;
        Real a = (Real)1.0;
        double rr = 0.0;
        if (s < len && i < d) {
            const long long k = k0 + s;
            const double um = (i > 0) ? fk_x(p, k - 1, i - 1) : 0.0;
            const double u = fk_x(p, k - 1, i);
            const double up = (i < d - 1) ? fk_x(p, k - 1, i + 1) : 0.0;
            const double un = fk_x(p, k, i);
            const double f = p.Dc * (um - 2.0 * u + up) + u * (1.0 - u);
            rr = un - (u + p.h * f);
            // leaf diagonal in the working precision of the fold
            const Real uR = (Real)u;
            a = (Real)1.0 + (hR * ((Real)1.0 - (Real)2.0 * uR) - (Real)2.0 * oR);
            p.r[k * d + i] = rr;
            unsigned long long b = (unsigned long long)__double_as_longlong(fabs(rr));
            my_res = b > my_res ? b : my_res;
            my_nf |= !isfinite(rr);
        }
        a_s[s * FDP + pidx<Real>(i)] = a;
        r_s[s * FDP + pidx<Real>(i)] = (Real)rr;
    }
    if (t == 0) {  // element 0: r_0 = x_1 - phi(x0)
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const double um = (i > 0) ? p.x0[i - 1] : 0.0;
            const double u = p.x0[i];
            const double up = (i < d - 1) ? p.x0[i + 1] : 0.0;
            const double un = fk_x(p, 0, i);
            const double f = p.Dc * (um - 2.0 * u + up) + u * (1.0 - u);
            const double rr = un - (u + p.h * f);
            p.r[i] = rr;
            unsigned long long b = (unsigned long long)__double_as_longlong(fabs(rr));
            my_res = b > my_res ? b : my_res;
            my_nf |= !isfinite(rr);
        }
    }
    fk_reduce_res(my_res, my_nf, p);
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
        for (int st = 0; st < len; ++st) {
            const Real* a = a_s + st * FDP + sbase;
            const Real above = __shfl_up_sync(0xffffffffu, s[R - 1], 1);
            const Real below = __shfl_down_sync(0xffffffffu, s[0], 1);
            const Real bot = (part < TPC - 1) ? below : (Real)0.0;
            Real prev = (part > 0) ? above : (Real)0.0;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const Real cur = s[i];
                const Real nxt = (i < R - 1) ? s[i + 1] : bot;
                const Real oi = (i < nrow_live) ? o : (Real)0.0;
                s[i] = fma(cur, a[i], oi * (prev + nxt));
                prev = cur;
            }
        }
        Real* col = S_out + ((size_t)t * FD + j) * FD + row0;
#pragma unroll
        for (int i = 0; i < R; ++i) col[i] = s[i] - ((row0 + i == j) ? (Real)1.0 : (Real)0.0);
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
                const Real oi = (r0 + i < d) ? o : (Real)0.0;
                b[i] = a[pidx<Real>(r0 + i)] * cur + oi * (prev + nxt) - rr[pidx<Real>(r0 + i)];
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
};

// FP64: grid (nodes, 4): each CTA computes 32 columns of S2 + S1 + S2 S1.
__global__ void __launch_bounds__(256) fk_compose_f64(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* As = reinterpret_cast<double*>(smem);   // [k][m] 128 x 128 (S2, column-major copy)
    double* Bs = As + FD * FD;                      // [n][k] 32 x 128  (S1 columns)
    const long long m = blockIdx.x;
    const int cb = blockIdx.y;
    const double* Sin = (const double*)a.S_in;
    const double* bin = (const double*)a.b_in;
    double* Sout = (double*)a.S_out;
    double* bout = (double*)a.b_out;
    const long long ce = 2 * m, cl = 2 * m + 1;
    const double* S1 = Sin + (size_t)ce * FD * FD;
    double* So = Sout + (size_t)m * FD * FD;
    if (cl >= a.n_in) {  // copy
        for (int idx = threadIdx.x; idx < 32 * FD; idx += blockDim.x)
            So[(size_t)cb * 32 * FD + idx] = S1[(size_t)cb * 32 * FD + idx];
        if (cb == 0)
            for (int i = threadIdx.x; i < FD; i += blockDim.x) bout[m * FD + i] = bin[ce * FD + i];
        return;
    }
    const double* S2 = Sin + (size_t)cl * FD * FD;
    for (int idx = threadIdx.x; idx < FD * FD; idx += blockDim.x) As[idx] = S2[idx];
    for (int idx = threadIdx.x; idx < 32 * FD; idx += blockDim.x) Bs[idx] = S1[(size_t)cb * 32 * FD + idx];
    __syncthreads();
    const int tm = threadIdx.x & 31, tn = threadIdx.x >> 5;  // rows 4tm.., cols 4tn..
    double acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = 0.0;
#pragma unroll 4
    for (int k = 0; k < FD; ++k) {
        double av[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) av[x] = As[k * FD + 4 * tm + x];
#pragma unroll
        for (int y = 0; y < 4; ++y) bv[y] = Bs[(4 * tn + y) * FD + k];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int n = cb * 32 + 4 * tn + y;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int mm = 4 * tm + x;
            So[(size_t)n * FD + mm] = As[n * FD + mm] + Bs[(4 * tn + y) * FD + mm] + acc[x][y];
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

// Mixed: one CTA (8 warps) per node; S2 S1 on tensor cores with
// mma.m16n8k16 BF16 -> FP32; S = S2 + S1 + S2 S1 and b in FP32.
constexpr int BSTR = FD + 8;  // bf16 row stride in smem (bank-conflict-free ldmatrix)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__global__ void __launch_bounds__(256) fk_compose_bf16(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);  // [k][m]  (S2 column-major)
    __nv_bfloat16* Bs = As + FD * BSTR;                           // [n][k]  (S1 column-major)
    float* b1s = reinterpret_cast<float*>(Bs + FD * BSTR);        // [FD]
    const long long m = blockIdx.x;
    const float* Sin = (const float*)a.S_in;
    const float* bin = (const float*)a.b_in;
    float* Sout = (float*)a.S_out;
    float* bout = (float*)a.b_out;
    const long long ce = 2 * m, cl = 2 * m + 1;
    const float* S1 = Sin + (size_t)ce * FD * FD;
    float* So = Sout + (size_t)m * FD * FD;
    if (cl >= a.n_in) {
        for (int idx = threadIdx.x; idx < FD * FD / 4; idx += blockDim.x)
            reinterpret_cast<float4*>(So)[idx] = reinterpret_cast<const float4*>(S1)[idx];
        for (int i = threadIdx.x; i < FD; i += blockDim.x) bout[m * FD + i] = bin[ce * FD + i];
        return;
    }
    const float* S2 = Sin + (size_t)cl * FD * FD;
    for (int idx = threadIdx.x; idx < FD * FD / 4; idx += blockDim.x) {
        const int c = idx / (FD / 4), r4 = (idx % (FD / 4)) * 4;
        const float4 va = reinterpret_cast<const float4*>(S2)[idx];
        const float4 vb = reinterpret_cast<const float4*>(S1)[idx];
        __nv_bfloat16* pa = As + c * BSTR + r4;
        __nv_bfloat16* pb = Bs + c * BSTR + r4;
        pa[0] = __float2bfloat16_rn(va.x); pa[1] = __float2bfloat16_rn(va.y);
        pa[2] = __float2bfloat16_rn(va.z); pa[3] = __float2bfloat16_rn(va.w);
        pb[0] = __float2bfloat16_rn(vb.x); pb[1] = __float2bfloat16_rn(vb.y);
        pb[2] = __float2bfloat16_rn(vb.z); pb[3] = __float2bfloat16_rn(vb.w);
    }
    for (int i = threadIdx.x; i < FD; i += blockDim.x) b1s[i] = bin[ce * FD + i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp & 3) * 32;   // 4 warps along m
    const int wn = (warp >> 2) * 64;  // 2 warps along n
    float acc[2][8][4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) acc[x][y][z] = 0.f;
    const int mat = lane >> 3, rr = lane & 7;
#pragma unroll
    for (int k0 = 0; k0 < FD; k0 += 16) {
        unsigned af[2][4];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            // A tile rows m = wm+16x.., k = k0..: stored As[k][m] -> ldmatrix.trans
            const int kk = k0 + rr + ((mat & 2) ? 8 : 0);
            const int mm = wm + 16 * x + ((mat & 1) ? 8 : 0);
            const unsigned addr = smem_u32(As + kk * BSTR + mm);
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                         : "=r"(af[x][0]), "=r"(af[x][1]), "=r"(af[x][2]), "=r"(af[x][3])
                         : "r"(addr));
        }
#pragma unroll
        for (int y2 = 0; y2 < 4; ++y2) {
            // two n-tiles (8 each) x two k halves: stored Bs[n][k] -> ldmatrix (no trans)
            unsigned bf[4];
            const int nn = wn + 16 * y2 + ((mat & 2) ? 8 : 0);
            const int kk = k0 + ((mat & 1) ? 8 : 0);
            const unsigned addr = smem_u32(Bs + (nn + rr) * BSTR + kk);
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                         : "=r"(bf[0]), "=r"(bf[1]), "=r"(bf[2]), "=r"(bf[3])
                         : "r"(addr));
#pragma unroll
            for (int x = 0; x < 2; ++x) {
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    float* c = acc[x][2 * y2 + h2];
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                        : "r"(af[x][0]), "r"(af[x][1]), "r"(af[x][2]), "r"(af[x][3]),
                          "r"(bf[2 * h2]), "r"(bf[2 * h2 + 1]));
                }
            }
        }
    }
    // epilogue: S = S2 + S1 + acc, column-major
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) {
                const int mm = wm + 16 * x + g + ((z & 2) ? 8 : 0);
                const int nn = wn + 8 * y + 2 * tq + (z & 1);
                const size_t off = (size_t)nn * FD + mm;
                So[off] = S2[off] + S1[off] + acc[x][y][z];
            }
    if (threadIdx.x < FD) {
        const int i = threadIdx.x;
        float s = bin[cl * FD + i] + b1s[i];
        for (int k = 0; k < FD; ++k) s = fmaf(S2[(size_t)k * FD + i], b1s[k], s);
        bout[m * FD + i] = s;
    }
}

// ---------------------------------------------------------------------------
// B2. down-sweep: z(child 2m) = z(m); z(child 2m+1) = z(m) + S_{2m} z(m) + b_{2m}.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(128) fk_down_kernel(const Real* __restrict__ S_child,
                                                      const Real* __restrict__ b_child,
                                                      const Real* __restrict__ z_parent,
                                                      Real* __restrict__ z_child, long long n_child,
                                                      const double* __restrict__ r0, int d) {
    __shared__ Real zs[FD];
    const long long m = blockIdx.x;
    const int i = threadIdx.x;
    Real zi;
    if (r0) zi = (i < d) ? (Real)(-r0[i]) : (Real)0.0;  // root: dx_1 = -h_1
    else zi = z_parent[m * FD + i];
    zs[i] = zi;
    __syncthreads();
    z_child[(2 * m) * FD + i] = zi;
    if (2 * m + 1 < n_child) {
        const Real* S = S_child + (size_t)(2 * m) * FD * FD;
        Real s = zi + b_child[(2 * m) * FD + i];
#pragma unroll 8
        for (int k = 0; k < FD; ++k) s = fma(S[(size_t)k * FD + i], zs[k], s);
        z_child[(2 * m + 1) * FD + i] = s;
    }
}

// ---------------------------------------------------------------------------
// C. replay: one warp per tile (4 rows per lane), exact FP64 leaves.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(128) fk_replay_kernel(FkParams p, const Real* __restrict__ z_tiles) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * 4 + warp;
    unsigned long long my_q = 0ull;
    if (t < p.T) {
        const int d = p.d, r0 = 4 * lane;
        const long long k0 = 1 + t * p.TS;
        const long long k1 = min(p.N, k0 + p.TS);
        double z[4], xprev[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = r0 + i;
            z[i] = (row < d) ? (double)z_tiles[t * FD + row] : 0.0;
            xprev[i] = (row < d) ? fk_x(p, k0 - 1, row) : 0.0;
        }
        if (t == 0) {
            // element 0: dx_1 = -r_0 (already the incoming vector of tile 0)
            bool bad = false;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = r0 + i;
                if (row < d) {
                    bad |= !(fabs(z[i]) <= p.cap);
                    p.Xn[row] = xprev[i] + z[i];
                }
            }
            if (bad) my_q = ~0ull;  // ~0 = index 0
        }
        // steps in groups of G: the loads of a group are issued together so
        // their latency overlaps; the recurrence itself is serial in k
        constexpr int G = 4;
        for (long long kg = k0; kg < k1; kg += G) {
            double xc[G][4], rk[G][4];
#pragma unroll
            for (int gq = 0; gq < G; ++gq) {
                const long long k = kg + gq;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int row = r0 + i;
                    const bool live = (k < k1) && (row < d);
                    xc[gq][i] = live ? fk_x(p, k, row) : 0.0;
                    rk[gq][i] = live ? p.r[k * d + row] : 0.0;
                }
            }
#pragma unroll
            for (int gq = 0; gq < G; ++gq) {
                const long long k = kg + gq;
                if (k >= k1) break;
                double a[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = 1.0 + (p.h * (1.0 - 2.0 * xprev[i]) - 2.0 * p.o);
                const double up = __shfl_up_sync(0xffffffffu, z[3], 1);
                const double dn = __shfl_down_sync(0xffffffffu, z[0], 1);
                double prev = (lane == 0) ? 0.0 : up;
                double nz[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const double cur = z[i];
                    const double nxt = (i < 3) ? z[i + 1] : ((lane == 31) ? 0.0 : dn);
                    const double oi = (r0 + i < d) ? p.o : 0.0;
                    nz[i] = (r0 + i < d) ? (a[i] * cur + oi * (prev + nxt) - rk[gq][i]) : 0.0;
                    prev = cur;
                }
                bool bad = false;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    z[i] = nz[i];
                    const int row = r0 + i;
                    if (row < d) {
                        bad |= !(fabs(z[i]) <= p.cap);
                        p.Xn[k * d + row] = xc[gq][i] + z[i];
                    }
                    xprev[i] = xc[gq][i];
                }
                if (bad) {
                    const unsigned long long e = ~(unsigned long long)k;
                    my_q = e > my_q ? e : my_q;
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, my_q, off);
        my_q = o > my_q ? o : my_q;
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
int run_iteration(FkParams& p, const Tree& tr, Real* S, Real* b, Real* z, bool mixed,
                  cudaStream_t st) {
    const size_t smemA = fold_smem_bytes<Real>(p.TS);
    {
        auto tok = timed_begin("fkpp_fold", st);
        fk_fold_kernel<Real><<<(unsigned)p.T, FoldTraits<Real>::THREADS, smemA, st>>>(p, S, b);
        timed_end(tok, st);
        count_launch(1);
    }
    // up-sweep
    for (size_t lv = 1; lv < tr.n.size(); ++lv) {
        LevelArgs la;
        la.S_in = S + (size_t)tr.off[lv - 1] * FD * FD;
        la.b_in = b + (size_t)tr.off[lv - 1] * FD;
        la.S_out = S + (size_t)tr.off[lv] * FD * FD;
        la.b_out = b + (size_t)tr.off[lv] * FD;
        la.n_in = tr.n[lv - 1];
        auto tok = timed_begin("fkpp_compose", st);
        if (mixed) {
            const size_t sm = 2 * (size_t)FD * BSTR * sizeof(__nv_bfloat16) + FD * sizeof(float);
            fk_compose_bf16<<<(unsigned)tr.n[lv], 256, sm, st>>>(la);
        } else {
            const size_t sm = (size_t)(FD * FD + 32 * FD) * sizeof(double);
            fk_compose_f64<<<dim3((unsigned)tr.n[lv], 4), 256, sm, st>>>(la);
        }
        timed_end(tok, st);
        count_launch(1);
    }
    // down-sweep
    const int L = (int)tr.n.size() - 1;
    if (L == 0) {
        auto tok = timed_begin("fkpp_down", st);
        fk_down_kernel<Real><<<1, FD, 0, st>>>(S, b, z, z, 1, p.r, p.d);  // z(tile 0) = -r_0
        timed_end(tok, st);
        count_launch(1);
    }
    for (int lv = L; lv >= 1; --lv) {
        const Real* zpar = z + (size_t)tr.off[lv] * FD;
        Real* zch = z + (size_t)tr.off[lv - 1] * FD;
        auto tok = timed_begin("fkpp_down", st);
        fk_down_kernel<Real><<<(unsigned)tr.n[lv], FD, 0, st>>>(
            S + (size_t)tr.off[lv - 1] * FD * FD, b + (size_t)tr.off[lv - 1] * FD, zpar, zch,
            tr.n[lv - 1], lv == L ? p.r : nullptr, p.d);
        timed_end(tok, st);
        count_launch(1);
    }
    {
        auto tok = timed_begin("fkpp_replay", st);
        fk_replay_kernel<Real><<<(unsigned)((p.T + 3) / 4), 128, 0, st>>>(p, z);
        timed_end(tok, st);
        count_launch(1);
    }
    return cudaGetLastError() == cudaSuccess ? PITN_OK : PITN_ECUDA;
}

template <typename Real>
int fkpp_solve_t(const SolveIO& io, double h, int64_t N, int d, double tol, int max_iter,
                 const pitn_options& o, cudaStream_t st, SolveOutcome* out, bool mixed) {
    const int TS = FK_TS;
    const long long T = std::max(1LL, (long long)((N - 1 + TS - 1) / TS));
    Tree tr = make_tree(T);
    // scratch: X1 | r ; aggregates S | b | z ; control
    const size_t nd = (size_t)N * d;
    double* X1 = (double*)workspace(nd * sizeof(double) * 2, kSlotX1);
    if (!X1) return PITN_ENOMEM;
    double* r = X1 + nd;
    const size_t aggBytes = (size_t)tr.total * FD * FD * sizeof(Real) +
                            2 * (size_t)tr.total * FD * sizeof(Real);
    Real* S = (Real*)workspace(aggBytes, kSlotAux);
    if (!S) return PITN_ENOMEM;
    Real* b = S + (size_t)tr.total * FD * FD;
    Real* z = b + (size_t)tr.total * FD;
    const size_t ctrlBytes = (size_t)(max_iter + 1) * (8 + 8 + 4) + 64;
    char* ctrl = (char*)workspace(ctrlBytes, kSlotCtrl);
    if (!ctrl) return PITN_ENOMEM;
    unsigned long long* res_bits = (unsigned long long*)ctrl;
    unsigned long long* qenc = res_bits + (max_iter + 1);
    int* nonfinite = (int*)(qenc + (max_iter + 1));
    if (cudaMemsetAsync(ctrl, 0, ctrlBytes, st) != cudaSuccess) return PITN_ECUDA;
    struct HostCtl { unsigned long long res, q; int nf; int pad; };
    HostCtl* hc = (HostCtl*)pinned(sizeof(HostCtl));
    if (!hc) return PITN_ENOMEM;

    {
        const int smemA = (int)fold_smem_bytes<Real>(TS);
        cudaFuncSetAttribute(fk_fold_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemA);
        cudaFuncSetAttribute(fk_compose_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((FD * FD + 32 * FD) * sizeof(double)));
        cudaFuncSetAttribute(fk_compose_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * FD * BSTR * sizeof(__nv_bfloat16) + FD * sizeof(float)));
    }

    const bool guarded = o.guard_B > 0.0 && std::isfinite(o.guard_B);
    FkParams p{};
    p.x0 = io.x0_dev;
    p.r = r;
    p.N = N;
    p.d = d;
    p.TS = TS;
    p.T = T;
    const double dx = 1.0 / (double)(d + 1);
    p.h = h;
    p.Dc = io.params[0] / (dx * dx);
    p.o = h * p.Dc;
    p.cap = guarded ? o.guard_B : DBL_MAX;
    double* bufs[2] = {io.traj_dev, X1};
    int cur = 0;
    long long q = io.have_guess ? N : 0;
    long long last_cut = N;
    int it = 0, status = PITN_NOT_CONVERGED;
    double final_res = 0.0;
    out->history.clear();
    for (;;) {
        p.X = bufs[cur];
        p.Xn = bufs[cur ^ 1];
        p.q = q;
        p.res_bits = res_bits + it;
        p.qenc = qenc + it;
        p.nonfinite = nonfinite + it;
        int rc = run_iteration<Real>(p, tr, S, b, z, mixed, st);
        if (rc != PITN_OK) return rc;
        if (cudaMemcpyAsync(&hc->res, res_bits + it, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&hc->q, qenc + it, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&hc->nf, nonfinite + it, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return PITN_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
        double res;
        std::memcpy(&res, &hc->res, sizeof(res));
        const long long cut = hc->q ? (long long)(~hc->q) : (long long)N;
        out->history.push_back(res);
        final_res = res;
        if (hc->nf) { status = PITN_NONFINITE; break; }
        if (res <= tol) { status = PITN_OK; break; }
        if (it == max_iter) { status = PITN_NOT_CONVERGED; break; }
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
    if (o.precision == PITN_PREC_MIXED_BF16) {
        if (d < 64) return PITN_EINVAL;
        return fkpp_solve_t<float>(io, h, N, d, tol, max_iter, o, st, out, true);
    }
    return fkpp_solve_t<double>(io, h, N, d, tol, max_iter, o, st, out, false);
}

}  // namespace pitn_host
