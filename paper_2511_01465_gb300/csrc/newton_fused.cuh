// newton_fused.cuh -- the small-state Newton solve with the replay of one
// iteration and the residual / Jacobian / fold of the next one fused into a
// single pass over the trajectory (included by newton_small.cuh).
//
// The three-phase kernel (newton_small_kernel) runs, per iteration, a phase
// that is FP64-bound (residual, Jacobian and thread fold: 20 FP64 operations
// per van der Pol step, little memory) and, after the scan, a phase that is
// memory-bound (replay and update: 6 FP64 operations, 64 B per step).  Here a
// thread walks its steps once per iteration: it replays the Newton step of
// iteration i (eq. 3.13 / 3.19), writes x^{(i+1)}_k, and with the new state
// pair at hand evaluates the element a_k of iteration i + 1 (eq. 3.8, 3.9,
// 3.4) and folds it -- so the FP64 work of the next residual overlaps the
// memory traffic of the update, and the state is read once instead of twice.
//
// What the fused pass cannot know is resolved after the grid barrier that
// ends it:
//   * the first element of each thread uses the previous thread's last new
//     state: it is evaluated after the barrier and composed in front of the
//     thread's fold;
//   * the guard's cut q (first correction beyond the bound, reading R8) is a
//     grid-wide minimum: a thread whose range starts at or after q discards
//     its speculative elements and rebuilds its aggregate from the fill
//     element by binary powering; the thread holding q appends the fill
//     power for its steps from q on.
// A thread's range of steps is the same in every iteration (uniform split),
// so the scratch slots written for iteration i + 1 are the ones its replay of
// iteration i has just consumed.
#pragma once

namespace pitn {

template <class Sys>
__global__ void __launch_bounds__(256) newton_fused_kernel(SmallArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D;
    Sys sys;
    sys.init(a.params, a.h);

    __shared__ double s_wex[kMaxWarps][E];
    __shared__ double s_tot[E];
    __shared__ double s_g[kMaxWarps][E];
    __shared__ double s_gtot[E];
    __shared__ double s_zin[D];
    extern __shared__ __align__(16) double s_dyn[];   // row-stage tiles (D == 2, stage_rows > 0)

    const int lane = threadIdx.x & 31;
    const long long N = a.N;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const unsigned G = gridDim.x;
    double* __restrict__ scr = a.scratch;

    // uniform split: thread gt owns steps [k0, k1), chain A = [k0, km), chain B = [km, k1)
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

    // chain aggregates of the current iteration's elements
    double PA[D * D], cA[D], PB[D * D], cB[D];
    unsigned long long my_res = 0ull;

    auto absmax = [](unsigned long long m, const double* v) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const unsigned long long b = abs_bits(v[j]);
            m = b > m ? b : m;
        }
        return m;
    };
    // element k from the state pair (xp, xc): scratch + fold into (P, c)
    auto fold_elem = [&](long long k, const double* xp, const double* xc, double* P, double* c,
                         unsigned long long& res) {
        double r[D], jv[JN];
        sys.eval(xp, xc, r, jv);
#pragma unroll
        for (int j = 0; j < JN; ++j) scr[sidx(k, j)] = jv[j];
#pragma unroll
        for (int j = 0; j < D; ++j) scr[sidx(k, JN + j)] = r[j];
        res = absmax(res, r);
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
    };
    // (P, c) <- (P, c) o (element k): the element precedes what (P, c) folded
    auto prepend_elem = [&](long long k, const double* xp, const double* xc, double* P, double* c,
                            unsigned long long& res) {
        double EP[D * D], Ec[D];
        mat_identity<D>(EP);
#pragma unroll
        for (int j = 0; j < D; ++j) Ec[j] = 0.0;
        fold_elem(k, xp, xc, EP, Ec, res);
        compose<D>(P, c, EP, Ec, P, c);
    };
    // (P, c) <- (P, c) followed by `count` copies of the fill element at xf
    auto append_fill = [&](long long count, const double* xf, double* P, double* c, unsigned long long& res) {
        if (count <= 0) return;
        double rf[D], jvf[JN], EP[D * D], Ec[D], RP[D * D], Rc[D];
        sys.eval(xf, xf, rf, jvf);
        res = absmax(res, rf);
        sys.jfull(jvf, EP);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            Ec[j] = -rf[j];
            Rc[j] = 0.0;
        }
        mat_identity<D>(RP);
        for (long long e = count;;) {
            if (e & 1) compose<D>(EP, Ec, RP, Rc, RP, Rc);
            e >>= 1;
            if (!e) break;
            compose<D>(EP, Ec, EP, Ec, EP, Ec);
        }
        compose<D>(RP, Rc, P, c, P, c);
    };
    // elements of a chain [s, e) of iterate X with fill from q on, from scratch
    auto build_chain = [&](const double* X, long long s, long long e, long long qq, double* P, double* c,
                           unsigned long long& res) {
        mat_identity<D>(P);
#pragma unroll
        for (int j = 0; j < D; ++j) c[j] = 0.0;
        if (s >= e) return;
        const long long sf = (qq < N) ? (qq > 1 ? qq : 1LL) : N;   // element 0 is never a fill element
        const long long er = min(e, max(s, sf));
        if (s < er) {
            double xp[D];
            load_state<D>(X, a.x0, s - 1, qq, xp);
            for (long long k = s; k < er; ++k) {
                double x[D];
                load_state<D>(X, a.x0, k, qq, x);
                fold_elem(k, xp, x, P, c, res);
#pragma unroll
                for (int j = 0; j < D; ++j) xp[j] = x[j];
            }
        }
        if (er < e) {
            double xf[D];
            load_state<D>(X, a.x0, qq - 1, qq, xf);
            append_fill(e - er, xf, P, c, res);
        }
    };

    // ---- elements of iteration 0 -------------------------------------------
    build_chain(a.X0, k0, km, q, PA, cA, my_res);
    build_chain(a.X0, km, k1, q, PB, cB, my_res);

    for (;;) {
        const double* __restrict__ Xc = cur ? a.X1 : a.X0;
        double* __restrict__ Xn = cur ? a.X0 : a.X1;

        // ---- thread and CTA aggregates, residual ---------------------------
        double P[D * D], c[D], eP[D * D], ec[D];
        compose<D>(PB, cB, PA, cA, P, c);
        block_scan<D>(P, c, eP, ec, s_wex, s_tot);
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
        if (G <= 64) {
            cta_incoming<D>(a.agg, G, s_zin);
        } else {
            const unsigned m = (G + blockDim.x - 1) / blockDim.x;
            double gP[D * D], gc[D];
            mat_identity<D>(gP);
#pragma unroll
            for (int j = 0; j < D; ++j) gc[j] = 0.0;
            for (unsigned i = threadIdx.x * m; i < min(G, (threadIdx.x + 1) * m); ++i) {
                double sP[D * D], sc[D];
#pragma unroll
                for (int j = 0; j < D * D; ++j) sP[j] = __ldcg(a.agg + (size_t)i * E + j);
#pragma unroll
                for (int j = 0; j < D; ++j) sc[j] = __ldcg(a.agg + (size_t)i * E + D * D + j);
                compose<D>(sP, sc, gP, gc, gP, gc);
            }
            double xP[D * D], xc[D];
            block_scan<D>(gP, gc, xP, xc, s_g, s_gtot);
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

        // ---- fused pass: replay of this iteration, elements of the next ------
        double zA[D], zB[D];
        {
            double zw[D];
            apply<D>(s_wex[threadIdx.x >> 5], s_wex[threadIdx.x >> 5] + D * D, s_zin, zw);
            apply<D>(eP, ec, zw, zA);
            apply<D>(PA, cA, zA, zB);  // state entering chain B
        }
        const long long sfill = (q < N) ? (q > 1 ? q : 1LL) : N;
        double xf[D], rf[D], jvf[JN];
        const bool need_fill = sfill < k1 && k0 < k1;
        if (need_fill) {
            load_state<D>(Xc, a.x0, q - 1, q, xf);
            sys.eval(xf, xf, rf, jvf);
        }
        // next-iteration chain folds (their first elements are prepended later)
        double NA[D * D], nA[D], NB[D * D], nB[D];
        mat_identity<D>(NA);
        mat_identity<D>(NB);
#pragma unroll
        for (int j = 0; j < D; ++j) { nA[j] = 0.0; nB[j] = 0.0; }
        unsigned long long resA = 0ull, resB = 0ull;   // next-iteration residuals per chain
        double prevA[D], prevB[D], firstA[D], firstB[D];
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
        // one step of chain ch at k; false once the chain hit the guard's bound
        auto step = [&](int ch, long long k, long long s, double* z, double* prev, double* first, double* NP,
                        double* nc, long long& cut, unsigned long long& res) {
            double jv[JN], r[D], x[D];
            if (k < sfill) {
#pragma unroll
                for (int j = 0; j < JN; ++j) jv[j] = scr[sidx(k, j)];
#pragma unroll
                for (int j = 0; j < D; ++j) r[j] = scr[sidx(k, JN + j)];
            } else {
#pragma unroll
                for (int j = 0; j < JN; ++j) jv[j] = jvf[j];
#pragma unroll
                for (int j = 0; j < D; ++j) r[j] = rf[j];
            }
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
            double xn[D];
            unsigned long long zb = 0ull;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                xn[j] = x[j] + z[j];
                const unsigned long long b = abs_bits(z[j]);
                zb = b > zb ? b : zb;
            }
            put_row(ch, k, xn);
            if (zb > a.cap_bits) {
                cut = k;
                return false;
            }
            if (k > s) fold_elem(k, prev, xn, NP, nc, res);
            else {
#pragma unroll
                for (int j = 0; j < D; ++j) first[j] = xn[j];
            }
#pragma unroll
            for (int j = 0; j < D; ++j) prev[j] = xn[j];
            return true;
        };
        {
            bool liveA = LA > 0, liveB = LB > 0;
            for (long long i = 0; i < LA && liveA; ++i) {
                liveA = step(0, k0 + i, k0, zA, prevA, firstA, NA, nA, cutA, resA);
                if (liveB && i < LB) liveB = step(1, km + i, km, zB, prevB, firstB, NB, nB, cutB, resB);
            }
            // everything after a cut in chain A lies beyond it: chain B's work is void
            if (cutA < N) {
                cutB = N;
                resB = 0ull;
            }
            if (staged) stg.finish(Xn);
            const long long kc = (cutA < N) ? cutA : cutB;   // first cut in this thread's steps
            // chain B's first element pairs chain A's last new state with its own first one
            if (LB > 0 && kc > km) {
                double EP[D * D], Ec[D];
                mat_identity<D>(EP);
#pragma unroll
                for (int j = 0; j < D; ++j) Ec[j] = 0.0;
                fold_elem(km, prevA, firstB, EP, Ec, resB);
                compose<D>(NB, nB, EP, Ec, NB, nB);
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

            // ---- elements of the next iteration, now that the cut is known ----
            const long long qn = a.guarded ? cut : N;
            const long long sfn = (qn < N) ? (qn > 1 ? qn : 1LL) : N;
            my_res = 0ull;
            if (k0 < k1) {
                if (sfn <= k0) {
                    // every step of this thread lies beyond the cut: its states are the
                    // fill, its speculative elements are void
                    build_chain(Xn, k0, km, qn, NA, nA, my_res);
                    build_chain(Xn, km, k1, qn, NB, nB, my_res);
                } else {
                    my_res = resA > resB ? resA : resB;
                    // first element of chain A: the previous thread's last new state
                    // (x0 for element 0; the fill if the cut is at element 0)
                    double xp[D], xc0[D];
                    load_state<D>(Xn, a.x0, k0 - 1, qn, xp);
                    if (k0 < qn) {
#pragma unroll
                        for (int j = 0; j < D; ++j) xc0[j] = firstA[j];
                    } else {
                        load_state<D>(Xn, a.x0, k0, qn, xc0);
                    }
                    prepend_elem(k0, xp, xc0, NA, nA, my_res);
                    if (sfn < k1) {
                        // this thread holds the cut: its steps from sfn on repeat the fill element
                        double xfn[D];
                        load_state<D>(Xn, a.x0, qn - 1, qn, xfn);
                        if (sfn < km) {
                            append_fill(km - sfn, xfn, NA, nA, my_res);
                            mat_identity<D>(NB);
#pragma unroll
                            for (int j = 0; j < D; ++j) nB[j] = 0.0;
                            append_fill(LB, xfn, NB, nB, my_res);
                        } else {
                            append_fill(k1 - sfn, xfn, NB, nB, my_res);
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < D * D; ++j) { PA[j] = NA[j]; PB[j] = NB[j]; }
#pragma unroll
            for (int j = 0; j < D; ++j) { cA[j] = nA[j]; cB[j] = nB[j]; }
            cur ^= 1;
            q = qn;
            last_cut = cut;
            ++it;
        }
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
