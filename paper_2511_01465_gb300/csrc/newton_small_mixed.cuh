// newton_small_mixed.cuh -- the small-state Newton solve with a reduced-
// precision scan (an inexact Newton step), included by newton_small.cu.
//
// Same three-phase persistent kernel as the FP64 one (residual + fold, fixed-
// order scan of the CTA aggregates, replay + update, two grid barriers per
// iteration), with one change of arithmetic: the residual, the stopping test
// and the update x + dx stay FP64, while the affine elements are kept in FP32
// in the delta form A = I + S (S = J - I = h df/dx keeps its full relative
// precision, where rounding J itself to FP32 would lose the O(h) part):
//   (I + S2, c2) o (I + S1, c1) = (I + S2 + S1 + S2 S1, c2 + c1 + S2 c1),
//   (I + S) v + c = v + S v + c,   head element a_0 = (S = -I, c = -r_0).
// The Newton step therefore carries FP32 rounding; the outer iteration
// converges to the FP64 tolerance because every residual is exact FP64.
// FP64 <-> FP32 conversions of per-step values (the residual into the scan,
// the correction into the update, the states feeding the FP32 Jacobian) use
// the integer-pipe routines of fpconv.cuh: a hardware conversion issues on
// the FP64 pipe, the resource this kernel is bound by.  Per step the FP64
// pipe then sees only the residual and the update.
#pragma once

namespace pitn {

template <int D>
__device__ __forceinline__ void dz_zero(float* Q, float* c) {
#pragma unroll
    for (int i = 0; i < D * D; ++i) Q[i] = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) c[i] = 0.f;
}

// (Q, c) <- (Q2, c2) o (Q1, c1) in the delta form
template <int D>
__device__ __forceinline__ void dz_compose(const float* Q2, const float* c2, const float* Q1, const float* c1,
                                           float* Q, float* c) {
    float tQ[D * D], tc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float s = Q2[i * D + j] + Q1[i * D + j];
#pragma unroll
            for (int l = 0; l < D; ++l) s = fmaf(Q2[i * D + l], Q1[l * D + j], s);
            tQ[i * D + j] = s;
        }
        float s = c2[i] + c1[i];
#pragma unroll
        for (int l = 0; l < D; ++l) s = fmaf(Q2[i * D + l], c1[l], s);
        tc[i] = s;
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) Q[i] = tQ[i];
#pragma unroll
    for (int i = 0; i < D; ++i) c[i] = tc[i];
}

// o = v + Q v + c
template <int D>
__device__ __forceinline__ void dz_apply(const float* Q, const float* c, const float* v, float* o) {
    float t[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float s = v[i] + c[i];
#pragma unroll
        for (int l = 0; l < D; ++l) s = fmaf(Q[i * D + l], v[l], s);
        t[i] = s;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) o[i] = t[i];
}

template <int D>
__device__ __forceinline__ void dz_warp_scan(float* Q, float* c, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float uQ[D * D], uc[D];
#pragma unroll
        for (int j = 0; j < D * D; ++j) uQ[j] = __shfl_up_sync(0xffffffffu, Q[j], off);
#pragma unroll
        for (int j = 0; j < D; ++j) uc[j] = __shfl_up_sync(0xffffffffu, c[j], off);
        if (lane >= off) dz_compose<D>(Q, c, uQ, uc, Q, c);
    }
}

// Exclusive block scan in the delta form (same fixed order as block_scan).
template <int D>
__device__ __forceinline__ void dz_block_scan(float* Q, float* c, float* eQ, float* ec,
                                              float (*s_wex)[D * D + D], float* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    dz_warp_scan<D>(Q, c, lane);
#pragma unroll
    for (int j = 0; j < D * D; ++j) eQ[j] = __shfl_up_sync(0xffffffffu, Q[j], 1);
#pragma unroll
    for (int j = 0; j < D; ++j) ec[j] = __shfl_up_sync(0xffffffffu, c[j], 1);
    if (lane == 0) dz_zero<D>(eQ, ec);
    __syncthreads();
    if (lane == 31) {
#pragma unroll
        for (int j = 0; j < D * D; ++j) s_wex[warp][j] = Q[j];
#pragma unroll
        for (int j = 0; j < D; ++j) s_wex[warp][D * D + j] = c[j];
    }
    __syncthreads();
    if (warp == 0) {
        float wQ[D * D], wc[D];
        if (lane < nwarps) {
#pragma unroll
            for (int j = 0; j < D * D; ++j) wQ[j] = s_wex[lane][j];
#pragma unroll
            for (int j = 0; j < D; ++j) wc[j] = s_wex[lane][D * D + j];
        } else {
            dz_zero<D>(wQ, wc);
        }
#pragma unroll
        for (int off = 1; off < kMaxWarps; off <<= 1) {
            if (off >= nwarps) break;   // lanes from nwarps on hold identities
            float uQ[D * D], uc[D];
#pragma unroll
            for (int j = 0; j < D * D; ++j) uQ[j] = __shfl_up_sync(0xffffffffu, wQ[j], off);
#pragma unroll
            for (int j = 0; j < D; ++j) uc[j] = __shfl_up_sync(0xffffffffu, wc[j], off);
            if (lane >= off) dz_compose<D>(wQ, wc, uQ, uc, wQ, wc);
        }
        float xQ[D * D], xc[D];
#pragma unroll
        for (int j = 0; j < D * D; ++j) xQ[j] = __shfl_up_sync(0xffffffffu, wQ[j], 1);
#pragma unroll
        for (int j = 0; j < D; ++j) xc[j] = __shfl_up_sync(0xffffffffu, wc[j], 1);
        __syncwarp();
        if (lane < nwarps) {
            if (lane == 0) dz_zero<D>(xQ, xc);
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

// (Q, c) <- (S, -r) o (Q, c) for one leaf: Q' = S + Q + S Q, c' = c + S c - r
template <int D>
__device__ __forceinline__ void dz_leaf(const float* S, const float* r, float* Q, float* c) {
    float tQ[D * D], tc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float s = S[i * D + j] + Q[i * D + j];
#pragma unroll
            for (int l = 0; l < D; ++l) s = fmaf(S[i * D + l], Q[l * D + j], s);
            tQ[i * D + j] = s;
        }
        float s = c[i] - r[i];
#pragma unroll
        for (int l = 0; l < D; ++l) s = fmaf(S[i * D + l], c[l], s);
        tc[i] = s;
    }
#pragma unroll
    for (int i = 0; i < D * D; ++i) Q[i] = tQ[i];
#pragma unroll
    for (int i = 0; i < D; ++i) c[i] = tc[i];
}

}  // namespace pitn

#include "scan_policy.cuh"

namespace pitn {

template <class Sys, class Pol>
__global__ void __launch_bounds__(256) newton_small_mixed_kernel(SmallArgs a) {
    using T = typename Pol::T;
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D, W = JN + D;
    Sys sys;
    sys.init(a.params, a.h);
    Pol::setup(sys, a);

    __shared__ T s_wex[kMaxWarps][E];
    __shared__ T s_tot[E];
    __shared__ T s_g[kMaxWarps][E];
    __shared__ T s_gtot[E];
    __shared__ T s_zin[D];
    extern __shared__ __align__(16) double s_dyn[];   // row-stage tiles (D == 2, stage_rows > 0)

    const int lane = threadIdx.x & 31;
    const long long N = a.N;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const unsigned G = gridDim.x;
    T* __restrict__ scr = reinterpret_cast<T*>(a.scratch);   // sizeof(T) <= sizeof(double)
    T* __restrict__ agg = reinterpret_cast<T*>(a.agg);
    double capd;
    {
        const unsigned long long cb = a.cap_bits;
        capd = __longlong_as_double((long long)cb);
    }
    const float capf = (float)fmin(capd, (double)FLT_MAX);

    int cur = 0;
    long long q = a.q_init;
    long long last_cut = N;
    int it = 0, status = PITN_NOT_CONVERGED;
    double final_res = 0.0;

    for (;;) {
        const double* __restrict__ Xc = cur ? a.X1 : a.X0;
        double* __restrict__ Xn = cur ? a.X0 : a.X1;
        const long long sfill = (q < N) ? (q > 1 ? q : 1LL) : N;
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
        const long long kreg = min(k1, max(k0, sfill));
        // scratch slot of component j of this thread's i-th regular element
        // (component-major, interleaved over the threads: coalesced)
        // slot of component j of step i: (j lcap + i) threads + gt, written so
        // that a step costs one multiply and the components fixed offsets
        const long long cstride = a.lcap * nthreads;
        auto sidx = [&](long long i, int j) -> long long { return i * nthreads + gt + j * cstride; };
        // ---- phase 1: FP64 residual, FP32 delta fold (two interleaved halves) ----
        unsigned long long my_res = 0ull;
        const long long Lr = kreg - k0;
        const long long LA = (Lr + 1) / 2, LB = Lr - LA, km = k0 + LA;
        T QA[D * D], cA[D], QB[D * D], cB[D];
        double xpA[D], xpB[D];
        Pol::template ident<D>(QA, cA);
        Pol::template ident<D>(QB, cB);
        // x of each half's next step is loaded one step ahead
        double xnA[D], xnB[D];
        if (LA > 0) {
            load_state<D>(Xc, a.x0, k0 - 1, q, xpA);
            load_state<D>(Xc, a.x0, k0, q, xnA);
        }
        if (LB > 0) {
            load_state<D>(Xc, a.x0, km - 1, q, xpB);
            load_state<D>(Xc, a.x0, km, q, xnB);
        }
        auto fold_step = [&](long long k, bool more, double* xp, double* xn, T* Q, T* c) {
            double x[D], r[D];
            T sv[JN], rf[D];
#pragma unroll
            for (int j = 0; j < D; ++j) x[j] = xn[j];
            if (more) load_state<D>(Xc, a.x0, k + 1, q, xn);
            Pol::eval(sys, xp, x, r, sv);
#pragma unroll
            for (int j = 0; j < JN; ++j) scr[sidx(k - k0, j)] = sv[j];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                rf[j] = Pol::from_double(r[j]);
                scr[sidx(k - k0, JN + j)] = rf[j];
                const unsigned long long b = abs_bits(r[j]);
                my_res = b > my_res ? b : my_res;
            }
            if (k == 0) Pol::template head<D>(rf, Q, c);   // a_0 = (0, -r_0), eq. 3.4
            else Pol::leaf(sys, sv, rf, Q, c);
#pragma unroll
            for (int j = 0; j < D; ++j) xp[j] = x[j];
        };
        for (long long i = 0; i < LA; ++i) {
            fold_step(k0 + i, i + 1 < LA, xpA, xnA, QA, cA);
            if (i < LB) fold_step(km + i, i + 1 < LB, xpB, xnB, QB, cB);
        }
        T Q[D * D], c[D];
        Pol::template compose<D>(QB, cB, QA, cA, Q, c);
        if (kreg < k1) {  // fill region: identical elements, binary powering
            double xf[D], rf64[D];
            T svf[JN], rff[D], EQ[D * D], Ec[D], RQ[D * D], Rc[D];
            load_state<D>(Xc, a.x0, q - 1, q, xf);
            Pol::eval(sys, xf, xf, rf64, svf);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const unsigned long long b = abs_bits(rf64[j]);
                my_res = b > my_res ? b : my_res;
                rff[j] = Pol::from_double(rf64[j]);
            }
            Pol::elem(sys, svf, rff, EQ, Ec);
            Pol::template ident<D>(RQ, Rc);
            for (long long e = k1 - kreg;;) {
                if (e & 1) Pol::template compose<D>(EQ, Ec, RQ, Rc, RQ, Rc);
                e >>= 1;
                if (!e) break;
                Pol::template compose<D>(EQ, Ec, EQ, Ec, EQ, Ec);
            }
            Pol::template compose<D>(RQ, Rc, Q, c, Q, c);
        }
        T eQ[D * D], ec[D];
        pol_block_scan<Pol, D>(Q, c, eQ, ec, s_wex, s_tot);
        if (threadIdx.x < E) agg[(size_t)blockIdx.x * E + threadIdx.x] = s_tot[threadIdx.x];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_res, off);
            my_res = o > my_res ? o : my_res;
        }
        if (lane == 0 && my_res) atomicMax(a.res_bits + it, my_res);
        if (!grid_barrier(a.bar, a.bar + 1, G, a.err, a.wait_ns)) return;

        const unsigned long long rb = __ldcg(a.res_bits + it);
        const double res = __longlong_as_double((long long)rb);
        final_res = res;
        if (rb >= kInfBits) { status = PITN_NONFINITE; break; }
        if (res <= a.tol) { status = PITN_OK; break; }
        if (it == a.max_iter) { status = PITN_NOT_CONVERGED; break; }

        // ---- incoming prefix: fixed-order scan of the CTA aggregates ----
        {
            const unsigned m = (G + blockDim.x - 1) / blockDim.x;
            T gQ[D * D], gc[D];
            Pol::template ident<D>(gQ, gc);
            for (unsigned i = threadIdx.x * m; i < min(G, (threadIdx.x + 1) * m); ++i) {
                T sQ[D * D], sc[D];
#pragma unroll
                for (int j = 0; j < D * D; ++j) sQ[j] = ld_cg(agg + (size_t)i * E + j);
#pragma unroll
                for (int j = 0; j < D; ++j) sc[j] = ld_cg(agg + (size_t)i * E + D * D + j);
                Pol::template compose<D>(sQ, sc, gQ, gc, gQ, gc);
            }
            T xQ[D * D], xc[D];
            pol_block_scan<Pol, D>(gQ, gc, xQ, xc, s_g, s_gtot);
            if (blockIdx.x > 0 && threadIdx.x == (blockIdx.x - 1) / m) {
                T v[D], t[D], zero[D];
#pragma unroll
                for (int j = 0; j < D; ++j) zero[j] = Pol::zero();
                Pol::template apply<D>(s_g[threadIdx.x >> 5], s_g[threadIdx.x >> 5] + D * D, zero, t);
                Pol::template apply<D>(xQ, xc, t, v);
                for (unsigned i = threadIdx.x * m; i <= blockIdx.x - 1; ++i) {
                    T sQ[D * D], sc[D];
#pragma unroll
                    for (int j = 0; j < D * D; ++j) sQ[j] = ld_cg(agg + (size_t)i * E + j);
#pragma unroll
                    for (int j = 0; j < D; ++j) sc[j] = ld_cg(agg + (size_t)i * E + D * D + j);
                    Pol::template apply<D>(sQ, sc, v, t);
#pragma unroll
                    for (int j = 0; j < D; ++j) v[j] = t[j];
                }
#pragma unroll
                for (int j = 0; j < D; ++j) s_zin[j] = v[j];
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
                for (int j = 0; j < D; ++j) s_zin[j] = Pol::zero();
            }
            __syncthreads();
        }

        // ---- phase 3: FP32 replay, FP64 update ----
        unsigned long long my_q = 0ull;
        {
            T zw[D], zA[D], zB[D];
            Pol::template apply<D>(s_wex[threadIdx.x >> 5], s_wex[threadIdx.x >> 5] + D * D, s_zin, zw);
            Pol::template apply<D>(eQ, ec, zw, zA);
            Pol::template apply<D>(QA, cA, zA, zB);
            bool foundA = false, foundB = false;
            long long firstA = 0, firstB = 0;
            // each half's next (S entries, r, x) is loaded one step ahead
            T fsA[W], fsB[W];
            double fxA[D], fxB[D];
            auto fetch = [&](long long k, T* fs, double* fx) {
#pragma unroll
                for (int j = 0; j < W; ++j) fs[j] = scr[sidx(k - k0, j)];   // this thread's phase-1 writes
                load_state<D>(Xc, a.x0, k, q, fx);
            };
            if (LA > 0) fetch(k0, fsA, fxA);
            if (LB > 0) fetch(km, fsB, fxB);
            const bool staged = (D == 2) && a.stage_rows > 0;
            RowStage stg;
            if (staged) stg.init(s_dyn);
            auto put_row = [&](int c, long long k, const double* v) {
                if constexpr (D == 2) {
                    if (staged) { stg.put(c, k, v[0], v[1], Xn); return; }
                }
#pragma unroll
                for (int j = 0; j < D; ++j) Xn[k * D + j] = v[j];
            };
            auto replay_step = [&](int c, long long k, bool more, T* fs, double* fx, T* z) -> bool {
                T sv[JN], rf[D];
                double x[D];
#pragma unroll
                for (int j = 0; j < JN; ++j) sv[j] = fs[j];
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    rf[j] = fs[JN + j];
                    x[j] = fx[j];
                }
                if (more) fetch(k + 1, fs, fx);
                if (k == 0) {
#pragma unroll
                    for (int j = 0; j < D; ++j) z[j] = Pol::neg(rf[j]);
                } else {
                    Pol::replay(sys, sv, rf, z);
                }
                bool bad = false;
                double xn[D];
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    xn[j] = Pol::add_to(x[j], z[j]);
                    bad |= !Pol::within(z[j], capf);
                }
                put_row(c, k, xn);
                return bad;
            };
            for (long long i = 0; i < LA && !foundA; ++i) {
                if (replay_step(0, k0 + i, i + 1 < LA, fsA, fxA, zA)) { foundA = true; firstA = k0 + i; }
                if (i < LB && !foundB && replay_step(1, km + i, i + 1 < LB, fsB, fxB, zB)) {
                    foundB = true;
                    firstB = km + i;
                }
            }
            const bool found = foundA || foundB;
            if (found) my_q = ~(unsigned long long)(foundA ? firstA : firstB);
            T z[D];
#pragma unroll
            for (int j = 0; j < D; ++j) z[j] = (LB > 0) ? zB[j] : zA[j];
            if (!found && kreg < k1) {
                double xf[D], rf64[D];
                T svf[JN], rfl[D];
                load_state<D>(Xc, a.x0, q - 1, q, xf);
                Pol::eval(sys, xf, xf, rf64, svf);
#pragma unroll
                for (int j = 0; j < D; ++j) rfl[j] = Pol::from_double(rf64[j]);
                for (long long k = kreg; k < k1; ++k) {
                    Pol::replay(sys, svf, rfl, z);
                    bool bad = false;
                    double xn[D];
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        xn[j] = Pol::add_to(xf[j], z[j]);
                        bad |= !Pol::within(z[j], capf);
                    }
                    put_row(1, k, xn);
                    if (bad) {
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
