// scan_policy.cuh -- the arithmetic of a reduced-precision small-state scan,
// as a policy of the kernels that run it (newton_small_mixed.cuh, the
// three-phase pass; newton_fused_mixed.cuh, the fused pass):
//   ScanF32:  FP32 in the delta form (elements (I + S, c), S = J - I), the
//             PITN_PREC_MIXED_FP32 solve;
//   ScanFF:   float-float (ffarith.cuh, ~2^-47 relative) in the plain form
//             (J, c) of eq. 3.3, the PITN_PREC_FP64_FF solve.
// Both keep the residual, the stopping test and the update x + dx in FP64,
// so the root is the FP64 root; the Newton step carries the scan's rounding.
// Included by newton_small_mixed.cuh after the delta-form helpers.
#pragma once

#include "ffarith.cuh"

namespace pitn {

// FP32 delta form: the existing mixed-precision arithmetic.
struct ScanF32 {
    using T = float;
    static constexpr int kMinBlocks = 0;   // no occupancy request: the compiler's own register choice
    template <class Sys>
    static constexpr int min_blocks() { return 0; }
    static constexpr bool kRollScans = false;
    // per-IVP batch kernel: threads per CTA at most, CTAs per SM at least
    static constexpr int kBatchThreads = 256, kBatchMinBlocks = 0;   // (0: the compiler's own choice)
    // fused pass: L1 prefetch of the next step's scratch and state lines
    static constexpr bool kPrefetchL1 = true;
    template <int D>
    static __device__ __forceinline__ void ident(T* Q, T* c) { dz_zero<D>(Q, c); }
    template <int D>
    static __device__ __forceinline__ void compose(const T* Q2, const T* c2, const T* Q1, const T* c1, T* Q, T* c) {
        dz_compose<D>(Q2, c2, Q1, c1, Q, c);
    }
    template <int D>
    static __device__ __forceinline__ void apply(const T* Q, const T* c, const T* v, T* o) { dz_apply<D>(Q, c, v, o); }
    // a_0 = (0, -r_0): S = -I
    template <int D>
    static __device__ __forceinline__ void head(const T* r, T* Q, T* c) {
#pragma unroll
        for (int j = 0; j < D * D; ++j) Q[j] = (j % (D + 1) == 0) ? -1.f : 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) c[j] = -r[j];
    }
    template <class Sys>
    static __device__ __forceinline__ void setup(Sys&, const SmallArgs&) {}
    // one IVP of a batch: the FP32 constants come with Sys::init
    template <class Sys>
    static __device__ __forceinline__ void setup_ivp(Sys&, const double*, double) {}
    template <class Sys>
    static __device__ __forceinline__ void eval(const Sys& sys, const double* xp, const double* xc, double* r,
                                                T* sv) {
        sys.eval_mixed(xp, xc, r, sv);
    }
    // (Q, c) <- (element) o (Q, c)
    template <class Sys>
    static __device__ __forceinline__ void leaf(const Sys& sys, const T* sv, const T* r, T* Q, T* c) {
        T S[Sys::D * Sys::D];
        sys.sfull(sv, S);
        dz_leaf<Sys::D>(S, r, Q, c);
    }
    // the element alone, (S, -r)
    template <class Sys>
    static __device__ __forceinline__ void elem(const Sys& sys, const T* sv, const T* r, T* Q, T* c) {
        sys.sfull(sv, Q);
#pragma unroll
        for (int j = 0; j < Sys::D; ++j) c[j] = -r[j];
    }
    // z <- J z - r = z + S z - r
    template <class Sys>
    static __device__ __forceinline__ void replay(const Sys& sys, const T* sv, const T* r, T* z) {
        constexpr int D = Sys::D;
        T S[D * D], t[D];
        sys.sfull(sv, S);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            float sacc = z[i] - r[i];
#pragma unroll
            for (int l = 0; l < D; ++l) sacc = fmaf(S[i * D + l], z[l], sacc);
            t[i] = sacc;
        }
#pragma unroll
        for (int j = 0; j < D; ++j) z[j] = t[j];
    }
    static __device__ __forceinline__ T from_double(double v) { return d2f_int(v); }
    static __device__ __forceinline__ T neg(T v) { return -v; }
    static __device__ __forceinline__ T zero() { return 0.f; }
    static __device__ __forceinline__ double add_to(double x, T z) { return x + f2d_int(z); }
    static __device__ __forceinline__ bool within(T z, float cap) { return fabsf(z) <= cap; }
    static __device__ __forceinline__ T shfl_up(T v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
};

// float-float, plain form (J, c).
struct ScanFF {
    using T = ff;
    static constexpr int kMinBlocks = 2;   // 128 registers: two 256-thread CTAs per SM
    // (a dense Jacobian -- the RK4 map's chain rule -- needs more registers
    // than two CTAs per SM leave: one CTA per SM there)
    template <class Sys>
    static constexpr int min_blocks() { return Sys::JN > Sys::D ? 1 : kMinBlocks; }
    // A float-float compose of 3 x 3 elements is ~400 instructions; for
    // d >= 3 the scans' levels run as loops, so that the kernel's code stays
    // within the instruction caches (unrolled, the d = 3 kernel's warps
    // waited on instruction fetch more than on anything else).
    static constexpr bool kRollScans = true;
    // per-IVP batch kernel: 128-thread CTAs, three per SM (at most 170
    // registers: the d = 3 kernel's 194 left two per SM)
    static constexpr int kBatchThreads = 128, kBatchMinBlocks = 3;
    static constexpr bool kPrefetchL1 = false;
    template <int D>
    static __device__ __forceinline__ void ident(T* P, T* c) {
#pragma unroll
        for (int j = 0; j < D * D; ++j) P[j] = (j % (D + 1) == 0) ? ff_one() : ff_zero();
#pragma unroll
        for (int j = 0; j < D; ++j) c[j] = ff_zero();
    }
    // (P, c) <- (P2, c2) o (P1, c1) = (P2 P1, P2 c1 + c2), eq. 3.3
    template <int D>
    static __device__ __forceinline__ void compose(const T* P2, const T* c2, const T* P1, const T* c1, T* P, T* c) {
        T tP[D * D], tc[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                T sacc = ff_mul(P2[i * D], P1[j]);
#pragma unroll
                for (int l = 1; l < D; ++l) sacc = ff_fma(P2[i * D + l], P1[l * D + j], sacc);
                tP[i * D + j] = sacc;
            }
            T sacc = c2[i];
#pragma unroll
            for (int l = 0; l < D; ++l) sacc = ff_fma(P2[i * D + l], c1[l], sacc);
            tc[i] = sacc;
        }
#pragma unroll
        for (int j = 0; j < D * D; ++j) P[j] = tP[j];
#pragma unroll
        for (int j = 0; j < D; ++j) c[j] = tc[j];
    }
    // o = P v + c
    template <int D>
    static __device__ __forceinline__ void apply(const T* P, const T* c, const T* v, T* o) {
        T t[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T sacc = c[i];
#pragma unroll
            for (int l = 0; l < D; ++l) sacc = ff_fma(P[i * D + l], v[l], sacc);
            t[i] = sacc;
        }
#pragma unroll
        for (int j = 0; j < D; ++j) o[j] = t[j];
    }
    // a_0 = (0, -r_0), eq. 3.4
    template <int D>
    static __device__ __forceinline__ void head(const T* r, T* P, T* c) {
#pragma unroll
        for (int j = 0; j < D * D; ++j) P[j] = ff_zero();
#pragma unroll
        for (int j = 0; j < D; ++j) c[j] = ff_neg(r[j]);
    }
    // constants from the host (see SmallArgs::fc, dc)
    template <class Sys>
    static __device__ __forceinline__ void setup(Sys& sys, const SmallArgs& a) { sys.init_ff(a.fc, a.dc); }
    // one IVP of a batch: its constants split here, from its own parameters
    template <class Sys>
    static __device__ __forceinline__ void setup_ivp(Sys& sys, const double* p, double h) {
        float fc[16];
        double dc[4];
        Sys::ff_consts(p, h, fc, dc);
        sys.init_ff(fc, dc);
    }
    template <class Sys>
    static __device__ __forceinline__ void eval(const Sys& sys, const double* xp, const double* xc, double* r,
                                                T* jv) {
        sys.eval_ff(xp, xc, r, jv);
    }
    template <class Sys>
    static __device__ __forceinline__ void leaf(const Sys& sys, const T* jv, const T* r, T* P, T* c) {
        sys.leaf_ff(jv, r, P, c);
    }
    template <class Sys>
    static __device__ __forceinline__ void elem(const Sys& sys, const T* jv, const T* r, T* P, T* c) {
        sys.jfull_ff(jv, P);
#pragma unroll
        for (int j = 0; j < Sys::D; ++j) c[j] = ff_neg(r[j]);
    }
    template <class Sys>
    static __device__ __forceinline__ void replay(const Sys& sys, const T* jv, const T* r, T* z) {
        sys.replay_ff(jv, r, z);
    }
    static __device__ __forceinline__ T from_double(double v) { return ff_from_double(v); }
    static __device__ __forceinline__ T neg(T v) { return ff_neg(v); }
    static __device__ __forceinline__ T zero() { return ff_zero(); }
    static __device__ __forceinline__ double add_to(double x, T z) { return ff_add_to_double(x, z); }
    static __device__ __forceinline__ bool within(T z, float cap) { return fabsf(z.hi) <= cap; }
    static __device__ __forceinline__ T shfl_up(T v, int off) { return ff_shfl_up(v, off); }
};

// Inclusive warp scan and exclusive block scan of policy elements, in the
// fixed order of block_scan (newton_small.cuh).
template <class Pol, int D>
__device__ __forceinline__ void pol_warp_scan(typename Pol::T* Q, typename Pol::T* c, int lane) {
    using T = typename Pol::T;
    auto level = [&](int off) {
        T uQ[D * D], uc[D];
#pragma unroll
        for (int j = 0; j < D * D; ++j) uQ[j] = Pol::shfl_up(Q[j], off);
#pragma unroll
        for (int j = 0; j < D; ++j) uc[j] = Pol::shfl_up(c[j], off);
        if (lane >= off) Pol::template compose<D>(Q, c, uQ, uc, Q, c);
    };
    if constexpr (Pol::kRollScans && D >= 3) {
#pragma unroll 1
        for (int off = 1; off < 32; off <<= 1) level(off);
    } else {
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) level(off);
    }
}

template <class Pol, int D>
__device__ __forceinline__ void pol_block_scan(typename Pol::T* Q, typename Pol::T* c, typename Pol::T* eQ,
                                               typename Pol::T* ec, typename Pol::T (*s_wex)[D * D + D],
                                               typename Pol::T* s_tot) {
    using T = typename Pol::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    pol_warp_scan<Pol, D>(Q, c, lane);
#pragma unroll
    for (int j = 0; j < D * D; ++j) eQ[j] = Pol::shfl_up(Q[j], 1);
#pragma unroll
    for (int j = 0; j < D; ++j) ec[j] = Pol::shfl_up(c[j], 1);
    if (lane == 0) Pol::template ident<D>(eQ, ec);
    __syncthreads();
    if (lane == 31) {
#pragma unroll
        for (int j = 0; j < D * D; ++j) s_wex[warp][j] = Q[j];
#pragma unroll
        for (int j = 0; j < D; ++j) s_wex[warp][D * D + j] = c[j];
    }
    __syncthreads();
    if (warp == 0) {
        T wQ[D * D], wc[D];
        if (lane < nwarps) {
#pragma unroll
            for (int j = 0; j < D * D; ++j) wQ[j] = s_wex[lane][j];
#pragma unroll
            for (int j = 0; j < D; ++j) wc[j] = s_wex[lane][D * D + j];
        } else {
            Pol::template ident<D>(wQ, wc);
        }
        auto level = [&](int off) {
            T uQ[D * D], uc[D];
#pragma unroll
            for (int j = 0; j < D * D; ++j) uQ[j] = Pol::shfl_up(wQ[j], off);
#pragma unroll
            for (int j = 0; j < D; ++j) uc[j] = Pol::shfl_up(wc[j], off);
            if (lane >= off) Pol::template compose<D>(wQ, wc, uQ, uc, wQ, wc);
        };
        // lanes from nwarps on hold identities
        if constexpr (Pol::kRollScans && D >= 3) {
#pragma unroll 1
            for (int off = 1; off < nwarps; off <<= 1) level(off);
        } else {
#pragma unroll
            for (int off = 1; off < kMaxWarps; off <<= 1) {
                if (off >= nwarps) break;
                level(off);
            }
        }
        T xQ[D * D], xc[D];
#pragma unroll
        for (int j = 0; j < D * D; ++j) xQ[j] = Pol::shfl_up(wQ[j], 1);
#pragma unroll
        for (int j = 0; j < D; ++j) xc[j] = Pol::shfl_up(wc[j], 1);
        __syncwarp();
        if (lane < nwarps) {
            if (lane == 0) Pol::template ident<D>(xQ, xc);
#pragma unroll
            for (int j = 0; j < D * D; ++j) s_wex[lane][j] = xQ[j];
#pragma unroll
            for (int j = 0; j < D; ++j) s_wex[lane][D * D + j] = xc[j];
        }
        if (lane == nwarps - 1) {
#pragma unroll
            for (int j = 0; j < D * D; ++j) s_tot[j] = wQ[j];
#pragma unroll
            for (int j = 0; j < D; ++j) s_tot[D * D + j] = wc[j];
        }
    }
    __syncthreads();
}

// L2-coherent loads of aggregates written by other CTAs before a grid barrier
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ ff ld_cg(const ff* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return ff{v.x, v.y};
}


}  // namespace pitn
