// newton_fused_mixed.cuh -- the fused small-state pass (newton_fused.cuh) with
// the scan's elements in a reduced-precision arithmetic: one pass per Newton
// iteration replays the step, updates the FP64 state, and builds the next
// iteration's elements from an exact FP64 residual.  The thread-boundary and
// guard fix-ups after the pass's grid barrier are those of the FP64 fused
// kernel.  Included by newton_small.cuh.
//
// The arithmetic of the scan is a policy (scan_policy.cuh).
#pragma once

namespace pitn {

// A request to bring the line holding p into L1 (prefetch.global.L1).
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
// steps ahead at which a chain's state row is prefetched: one 128-byte line
// of d = 2 rows
constexpr long long kStatePrefetch = 8;

template <class Sys, class Pol>
__global__ void __launch_bounds__(256, Pol::template min_blocks<Sys>()) newton_fused_mixed_kernel(SmallArgs a) {
    using T = typename Pol::T;
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D;
    // L1 prefetch in the step loop: the FP32 scan with compact elements (van
    // der Pol FP32 scan 16.1 -> 15.3 ms); slower with float-float (27.1 ->
    // 28.0 ms) and with the dense RK4 elements, which keep it off
    constexpr bool kPrefetch = Pol::kPrefetchL1 && JN <= D;
    Sys sys;
    sys.init(a.params, a.h);
    Pol::setup(sys, a);

    __shared__ T s_wex[kMaxWarps][E];
    __shared__ T s_tot[E];
    __shared__ T s_g[kMaxWarps][E];
    __shared__ T s_gtot[E];
    __shared__ T s_zin[D];
    // the fill element (the same for every thread) and each thread's first
    // updated state per half, kept here rather than in registers through
    // the pass's step loop
    __shared__ T s_fill[JN + D];
    __shared__ double s_first[2 * D][256];
    extern __shared__ __align__(16) double s_dyn[];   // row-stage tiles (D == 2, stage_rows > 0)

    const int lane = threadIdx.x & 31;
    const long long N = a.N;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const unsigned G = gridDim.x;
    T* __restrict__ scr = reinterpret_cast<T*>(a.scratch);   // sizeof(T) <= sizeof(double)
    T* __restrict__ agg = reinterpret_cast<T*>(a.agg);
    float capf;
    {
        const double capd = __longlong_as_double((long long)a.cap_bits);
        capf = (float)fmin(capd, (double)FLT_MAX);
    }

    const long long C = (N + nthreads - 1) / nthreads;
    const long long k0 = min(N, gt * C), k1 = min(N, k0 + C);
    const long long L = k1 - k0, LA = (L + 1) / 2, LB = L - LA, km = k0 + LA;
    // slot of component j of step k: (j lcap + k - k0) threads + gt, written so
    // that a step costs one multiply and the components fixed offsets
    const long long cstride = a.lcap * nthreads;
    auto sidx = [&](long long k, int j) -> long long { return (k - k0) * nthreads + gt + j * cstride; };

    int cur = 0;
    long long q = a.q_init;
    long long last_cut = N;
    int it = 0, status = PITN_NOT_CONVERGED;
    double final_res = 0.0;

    T QA[D * D], cA[D], QB[D * D], cB[D];
    unsigned long long my_res = 0ull;

    // element k from the state pair (xp, xc): FP64 residual, scan element into
    // scratch, folded into (Q, c)
    auto fold_elem = [&](long long k, const double* xp, const double* xc, T* Q, T* c,
                         unsigned long long& res) {
        double r[D];
        T sv[JN], rf[D];
        Pol::eval(sys, xp, xc, r, sv);
#pragma unroll
        for (int j = 0; j < JN; ++j) scr[sidx(k, j)] = sv[j];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const unsigned long long b = abs_bits(r[j]);
            res = b > res ? b : res;
            rf[j] = Pol::from_double(r[j]);
            scr[sidx(k, JN + j)] = rf[j];
        }
        if (k == 0) Pol::template head<D>(rf, Q, c);   // a_0 = (0, -r_0), eq. 3.4
        else Pol::leaf(sys, sv, rf, Q, c);
    };
    auto prepend_elem = [&](long long k, const double* xp, const double* xc, T* Q, T* c,
                            unsigned long long& res) {
        T EQ[D * D], Ec[D];
        Pol::template ident<D>(EQ, Ec);
        fold_elem(k, xp, xc, EQ, Ec, res);
        Pol::template compose<D>(Q, c, EQ, Ec, Q, c);
    };
    auto append_fill = [&](long long count, const double* xf, T* Q, T* c, unsigned long long& res) {
        if (count <= 0) return;
        double rf64[D];
        T svf[JN], rff[D], EQ[D * D], Ec[D], RQ[D * D], Rc[D];
        Pol::eval(sys, xf, xf, rf64, svf);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const unsigned long long b = abs_bits(rf64[j]);
            res = b > res ? b : res;
            rff[j] = Pol::from_double(rf64[j]);
        }
        Pol::elem(sys, svf, rff, EQ, Ec);
        Pol::template ident<D>(RQ, Rc);
        for (long long e = count;;) {
            if (e & 1) Pol::template compose<D>(EQ, Ec, RQ, Rc, RQ, Rc);
            e >>= 1;
            if (!e) break;
            Pol::template compose<D>(EQ, Ec, EQ, Ec, EQ, Ec);
        }
        Pol::template compose<D>(RQ, Rc, Q, c, Q, c);
    };
    auto build_chain = [&](const double* X, long long s, long long e, long long qq, T* Q, T* c,
                           unsigned long long& res) {
        Pol::template ident<D>(Q, c);
        if (s >= e) return;
        const long long sf = (qq < N) ? (qq > 1 ? qq : 1LL) : N;
        const long long er = min(e, max(s, sf));
        if (s < er) {
            double xp[D];
            load_state<D>(X, a.x0, s - 1, qq, xp);
            for (long long k = s; k < er; ++k) {
                double x[D];
                load_state<D>(X, a.x0, k, qq, x);
                fold_elem(k, xp, x, Q, c, res);
#pragma unroll
                for (int j = 0; j < D; ++j) xp[j] = x[j];
            }
        }
        if (er < e) {
            double xf[D];
            load_state<D>(X, a.x0, qq - 1, qq, xf);
            append_fill(e - er, xf, Q, c, res);
        }
    };

    build_chain(a.X0, k0, km, q, QA, cA, my_res);
    build_chain(a.X0, km, k1, q, QB, cB, my_res);

    for (;;) {
        const double* __restrict__ Xc = cur ? a.X1 : a.X0;
        double* __restrict__ Xn = cur ? a.X0 : a.X1;

        T Q[D * D], c[D], eQ[D * D], ec[D];
        Pol::template compose<D>(QB, cB, QA, cA, Q, c);
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

        // ---- fused pass ----------------------------------------------------
        T zA[D], zB[D];
        {
            T zw[D];
            Pol::template apply<D>(s_wex[threadIdx.x >> 5], s_wex[threadIdx.x >> 5] + D * D, s_zin, zw);
            Pol::template apply<D>(eQ, ec, zw, zA);
            Pol::template apply<D>(QA, cA, zA, zB);
        }
        const long long sfill = (q < N) ? (q > 1 ? q : 1LL) : N;
        if (sfill < N && threadIdx.x == 0) {
            double xf[D], rf64[D];
            T svf[JN];
            load_state<D>(Xc, a.x0, q - 1, q, xf);
            Pol::eval(sys, xf, xf, rf64, svf);
#pragma unroll
            for (int j = 0; j < JN; ++j) s_fill[j] = svf[j];
#pragma unroll
            for (int j = 0; j < D; ++j) s_fill[JN + j] = Pol::from_double(rf64[j]);
        }
        __syncthreads();
        T NA[D * D], nA[D], NB[D * D], nB[D];
        Pol::template ident<D>(NA, nA);
        Pol::template ident<D>(NB, nB);
        unsigned long long resA = 0ull, resB = 0ull;
        double prevA[D], prevB[D];
        long long cutA = N, cutB = N;
        const bool staged = (D == 2) && a.stage_rows > 0;
        RowStage stg;
        if (staged) stg.init(s_dyn);
        auto put_row = [&](int ch, long long k, const double* v) {
            if constexpr (D == 2) {
                if (staged) { stg.put(ch, k, v[0], v[1], Xn); return; }
            }
#pragma unroll
            for (int j = 0; j < D; ++j) Xn[k * D + j] = v[j];
        };
        auto step = [&](int ch, long long k, long long s, T* z, double* prev, T* NQ,
                        T* nc, long long& cut, unsigned long long& res) {
            T sv[JN], r[D];
            // the next step's scratch lines and the state row a line ahead are
            // requested into L1 now (no registers held; nothing waits on them)
            if constexpr (kPrefetch) {
                if (k + 1 < sfill && k + 1 < k1) {   // (within this thread's scratch slots)
#pragma unroll
                    for (int j = 0; j < JN + D; ++j) prefetch_l1(scr + sidx(k + 1, j));
                }
                if (k + kStatePrefetch < q) prefetch_l1(Xc + (k + kStatePrefetch) * D);
            }
            if (k < sfill) {
#pragma unroll
                for (int j = 0; j < JN; ++j) sv[j] = scr[sidx(k, j)];
#pragma unroll
                for (int j = 0; j < D; ++j) r[j] = scr[sidx(k, JN + j)];
            } else {
#pragma unroll
                for (int j = 0; j < JN; ++j) sv[j] = s_fill[j];
#pragma unroll
                for (int j = 0; j < D; ++j) r[j] = s_fill[JN + j];
            }
            double x[D];
            load_state<D>(Xc, a.x0, k, q, x);
            if (k == 0) {
#pragma unroll
                for (int j = 0; j < D; ++j) z[j] = Pol::neg(r[j]);
            } else {
                Pol::replay(sys, sv, r, z);
            }
            double xn[D];
            bool bad = false;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                xn[j] = Pol::add_to(x[j], z[j]);
                bad |= !Pol::within(z[j], capf);
            }
            put_row(ch, k, xn);
            if (bad) {
                cut = k;
                return false;
            }
            if (k > s) fold_elem(k, prev, xn, NQ, nc, res);
            else {
#pragma unroll
                for (int j = 0; j < D; ++j) s_first[ch * D + j][threadIdx.x] = xn[j];
            }
#pragma unroll
            for (int j = 0; j < D; ++j) prev[j] = xn[j];
            return true;
        };
        bool liveA = LA > 0, liveB = LB > 0;
        for (long long i = 0; i < LA && liveA; ++i) {
            liveA = step(0, k0 + i, k0, zA, prevA, NA, nA, cutA, resA);
            if (liveB && i < LB) liveB = step(1, km + i, km, zB, prevB, NB, nB, cutB, resB);
        }
        if (cutA < N) {
            cutB = N;
            resB = 0ull;
        }
        if (staged) stg.finish(Xn);
        const long long kc = (cutA < N) ? cutA : cutB;
        if (LB > 0 && kc > km) {
            T EQ[D * D], Ec[D];
            Pol::template ident<D>(EQ, Ec);
            double firstB[D];
#pragma unroll
            for (int j = 0; j < D; ++j) firstB[j] = s_first[D + j][threadIdx.x];
            fold_elem(km, prevA, firstB, EQ, Ec, resB);
            Pol::template compose<D>(NB, nB, EQ, Ec, NB, nB);
        }
        unsigned long long my_q = (kc < N) ? ~(unsigned long long)kc : 0ull;
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

        const long long qn = a.guarded ? cut : N;
        const long long sfn = (qn < N) ? (qn > 1 ? qn : 1LL) : N;
        my_res = 0ull;
        if (k0 < k1) {
            if (sfn <= k0) {
                build_chain(Xn, k0, km, qn, NA, nA, my_res);
                build_chain(Xn, km, k1, qn, NB, nB, my_res);
            } else {
                my_res = resA > resB ? resA : resB;
                double xp[D], xc0[D];
                load_state<D>(Xn, a.x0, k0 - 1, qn, xp);
                if (k0 < qn) {
#pragma unroll
                    for (int j = 0; j < D; ++j) xc0[j] = s_first[j][threadIdx.x];
                } else {
                    load_state<D>(Xn, a.x0, k0, qn, xc0);
                }
                prepend_elem(k0, xp, xc0, NA, nA, my_res);
                if (sfn < k1) {
                    double xfn[D];
                    load_state<D>(Xn, a.x0, qn - 1, qn, xfn);
                    if (sfn < km) {
                        append_fill(km - sfn, xfn, NA, nA, my_res);
                        Pol::template ident<D>(NB, nB);
                        append_fill(LB, xfn, NB, nB, my_res);
                    } else {
                        append_fill(k1 - sfn, xfn, NB, nB, my_res);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < D * D; ++j) { QA[j] = NA[j]; QB[j] = NB[j]; }
#pragma unroll
        for (int j = 0; j < D; ++j) { cA[j] = nA[j]; cB[j] = nB[j]; }
        cur ^= 1;
        q = qn;
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
