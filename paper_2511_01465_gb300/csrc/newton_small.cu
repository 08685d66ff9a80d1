// newton_small.cu -- the whole Newton solve for small state dimension
// (d = 2, 3) in ONE persistent cooperative kernel.
//
// Per Newton iteration every CTA walks its tiles of BLOCK*C consecutive steps
// and, in a single pass over the trajectory:
//   1. loads x_{k-1}, x_k (lazy fill of the guard, see below) and evaluates
//      the residual r_k = x_{k+1} - phi(x_k) (eq. 3.8) and the compact
//      Jacobian J_k = dphi/dx(x_k) into registers; accumulates ||r||_inf and a
//      non-finite flag;
//   2. folds its C affine elements (J_k, -r_k) (eq. 3.4; element 0 has matrix
//      0) into a thread aggregate (P, c) with the operator of eq. 3.3;
//   3. scans the thread aggregates: Kogge-Stone over the warp with shuffles,
//      then over the warps through shared memory;
//   4. publishes the tile aggregate and resolves its incoming prefix by a
//      decoupled look-back over the preceding tiles' published aggregates /
//      inclusive prefixes (only the vector part of an inclusive prefix is
//      needed: every prefix that starts at element 0 has matrix 0);
//   5. replays its C elements from the incoming vector: dx_{k+1} = J_k dx_k -
//      r_k (eq. 3.13) and writes x_k + dx_k into the other trajectory buffer,
//      recording the first index whose correction is not finite or exceeds
//      the guard bound.
// A grid barrier then makes the iteration's ||r||_inf, non-finite flag and
// guard index visible to all CTAs, which take the same stop/continue
// decision.  The guard's fill (states from q on set to state q-1) is never
// written during the loop: the next pass reads x_k for k >= q as x_{q-1}.
//
// The decision order per iteration is the oracle's: non-finite residual ->
// NONFINITE; ||r|| <= tol -> OK; max_iter updates -> NOT_CONVERGED; plain
// Newton with a non-finite correction -> NONFINITE (iterate kept); otherwise
// accept the step.
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
    double* scratch;    // [N][JN + D]: compact Jacobian and residual of every step
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
};

constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
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

// x_k of the current iterate with the guard's lazy fill (L2-coherent loads).
template <int D>
__device__ __forceinline__ void load_state(const double* __restrict__ X, const double* __restrict__ x0,
                                           long long k, long long q, double* o) {
    const double* src;
    if (k < 0) src = x0;
    else if (k < q) src = X + k * D;
    else if (q > 0) src = X + (q - 1) * D;
    else src = x0;
#pragma unroll
    for (int i = 0; i < D; ++i) o[i] = ldcg(src + i);
}

constexpr int kMaxWarps = 8;  // BLOCK <= 256

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

// Exclusive block scan of per-thread elements.  On return (eP, ec) is the
// lane-exclusive prefix within the warp, s_wex[warp] the warp-exclusive
// prefix, and s_tot the block total.  All in a fixed order.
template <int D>
__device__ __forceinline__ void block_scan(double* P, double* c, double* eP, double* ec,
                                           double (*s_wex)[D * D + D], double* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    warp_scan<D>(P, c, lane);
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
            for (int j = 0; j < JN; ++j) scr[k * W + j] = jv[j];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                scr[k * W + JN + j] = r[j];
                const unsigned long long b = (unsigned long long)__double_as_longlong(r[j]) & kAbsMask;
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
                const unsigned long long b = (unsigned long long)__double_as_longlong(rf[j]) & kAbsMask;
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
        block_scan<D>(P, c, eP, ec, s_wex, s_tot);
        if (threadIdx.x < E) a.agg[(size_t)blockIdx.x * E + threadIdx.x] = s_tot[threadIdx.x];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_res, off);
            my_res = o > my_res ? o : my_res;
        }
        if (lane == 0 && my_res) atomicMax(a.res_bits + it, my_res);
        if (!grid_barrier(a.bar, a.bar + 1, G, a.err)) return;

        // ---- decision --------------------------------------------------------
        const unsigned long long rb = __ldcg(a.res_bits + it);
        const double res = __longlong_as_double((long long)rb);
        final_res = res;
        if (rb >= kInfBits) { status = PITN_NONFINITE; break; }
        if (res <= a.tol) { status = PITN_OK; break; }
        if (it == a.max_iter) { status = PITN_NOT_CONVERGED; break; }

        // ---- incoming prefix of this CTA: fixed-order scan of the aggregates ----
        {
            const unsigned m = (G + blockDim.x - 1) / blockDim.x;   // aggregates per thread
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
            auto replay_step = [&](long long k, double* z) -> bool {
                double jv[JN], r[D], x[D];
#pragma unroll
                for (int j = 0; j < JN; ++j) jv[j] = __ldcg(scr + k * W + j);
#pragma unroll
                for (int j = 0; j < D; ++j) r[j] = __ldcg(scr + k * W + JN + j);
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
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    Xn[k * D + j] = x[j] + z[j];
                    const unsigned long long b = (unsigned long long)__double_as_longlong(z[j]) & kAbsMask;
                    zb = b > zb ? b : zb;
                }
                return zb > a.cap_bits;
            };
            for (long long i = 0; i < LA && !foundA; ++i) {
                if (replay_step(k0 + i, zA)) { foundA = true; firstA = k0 + i; }
                if (i < LB && !foundB && replay_step(km + i, zB)) { foundB = true; firstB = km + i; }
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
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        z[j] = tz[j];
                        Xn[k * D + j] = xf[j] + z[j];
                        const unsigned long long b = (unsigned long long)__double_as_longlong(z[j]) & kAbsMask;
                        zb = b > zb ? b : zb;
                    }
                    if (zb > a.cap_bits) {
                        my_q = ~(unsigned long long)k;
                        break;
                    }
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_q, off);
            my_q = o > my_q ? o : my_q;
        }
        if (lane == 0 && my_q) atomicMax(a.qenc + it, my_q);
        if (!grid_barrier(a.bar, a.bar + 1, G, a.err)) return;
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

namespace pitn {

template <class Sys, bool MIXED = false>
static cudaError_t launch_small(SmallArgs& a, int grid, int block, cudaStream_t st) {
    void* args[] = {(void*)&a};
    auto tok = pitn_host::timed_begin("newton_small", st);
    const void* kern;
    if constexpr (MIXED) kern = (const void*)newton_small_mixed_kernel<Sys>;
    else kern = (const void*)newton_small_kernel<Sys>;
    cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(block), args, 0, st);
    pitn_host::timed_end(tok, st);
    pitn_host::count_launch(1);
    return e;
}

template <class Sys, bool MIXED = false>
static int max_blocks_per_sm(int block) {
    int per_sm = 0;
    cudaError_t e;
    if constexpr (MIXED) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_small_mixed_kernel<Sys>, block, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_small_kernel<Sys>, block, 0);
    if (e != cudaSuccess) return 0;
    return per_sm;
}

}  // namespace pitn

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

// One solve with an explicit launch shape: `block` threads per CTA and at
// most `per_sm_cap` co-resident CTAs per SM (cooperative launch).
int small_launch(int system_id, const SolveIO& io, double h, int64_t N, int d, double tol,
                 int max_iter, const pitn_options& o, cudaStream_t st, SolveOutcome* out, int block,
                 int per_sm_cap) {
    using namespace pitn;
    int cmin = 4;
    if (o.tile_elems > 0) cmin = o.tile_elems;
    const bool rk4 = o.method == PITN_STEP_RK4;
    const bool mixed = o.precision == PITN_PREC_MIXED_FP32;
    int per_sm = 0;
    int W = 0;
    if (mixed) {
        // FP32 scratch: W floats per step fit in the W-double slots
        switch (system_id) {
        case PITN_LORENZ63: per_sm = max_blocks_per_sm<Lorenz63, true>(block); W = Lorenz63::JN + 3; break;
        case PITN_VDP: per_sm = max_blocks_per_sm<VanDerPol, true>(block); W = VanDerPol::JN + 2; break;
        case PITN_LINEAR_OSC: per_sm = max_blocks_per_sm<LinearOsc, true>(block); W = LinearOsc::JN + 2; break;
        default: return PITN_EUNSUPPORTED;
        }
    } else if (rk4 && system_id == PITN_VDP) {
        per_sm = max_blocks_per_sm<RK4Map<VdpRhs>>(block);
        W = RK4Map<VdpRhs>::JN + 2;
    } else if (rk4 && system_id == PITN_LOGISTIC) {
        per_sm = max_blocks_per_sm<RK4Map<LogisticRhs>>(block);
        W = RK4Map<LogisticRhs>::JN + 1;
    } else if (rk4) {
        return PITN_EUNSUPPORTED;
    } else {
        switch (system_id) {
        case PITN_LORENZ63: per_sm = max_blocks_per_sm<Lorenz63>(block); W = Lorenz63::JN + 3; break;
        case PITN_VDP: per_sm = max_blocks_per_sm<VanDerPol>(block); W = VanDerPol::JN + 2; break;
        case PITN_LINEAR_OSC: per_sm = max_blocks_per_sm<LinearOsc>(block); W = LinearOsc::JN + 2; break;
        case PITN_LOGISTIC: per_sm = max_blocks_per_sm<EulerMap<LogisticRhs>>(block); W = 2; break;
        default: return PITN_EINVAL;
        }
    }
    if (per_sm < 1) return PITN_EUNSUPPORTED;  // shape does not fit on an SM
    per_sm = std::min(per_sm, per_sm_cap);
    const long long max_grid = (long long)per_sm * props().multiProcessorCount;
    const long long want = (N + (long long)block * cmin - 1) / ((long long)block * cmin);
    const int grid = (int)std::max(1LL, std::min(max_grid, want));
    const long long chunk = (N + (long long)grid * block - 1) / ((long long)grid * block);
    const int E = d * d + d;

    double* X1 = (double*)workspace((size_t)N * d * sizeof(double), kSlotX1);
    double* scratch = (double*)workspace((size_t)N * W * sizeof(double), kSlotAux);
    // control block: agg | res_bits | qenc | bar | err | record
    size_t off_agg = 0;
    size_t off_res = off_agg + (size_t)grid * E * sizeof(double);
    size_t off_q = off_res + sizeof(unsigned long long) * (size_t)(max_iter + 1);
    size_t off_bar = (off_q + sizeof(unsigned long long) * (size_t)(max_iter + 1) + 15) & ~(size_t)15;
    size_t off_err = off_bar + 16;
    size_t off_rec = off_err + 16;
    size_t total = off_rec + sizeof(SolveRecord);
    char* ctrl = (char*)workspace(total, kSlotCtrl);
    // host mirror: err | record | history
    size_t hbytes = 16 + sizeof(SolveRecord) + sizeof(double) * (size_t)(max_iter + 1);
    char* hbuf = (char*)pinned(hbytes);
    if (!X1 || !scratch || !ctrl || !hbuf) return PITN_ENOMEM;

    SmallArgs a{};
    a.x0 = io.x0_dev;
    a.X0 = io.traj_dev;
    a.X1 = X1;
    a.out = io.traj_dev;
    a.scratch = scratch;
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

    if (cudaMemsetAsync(ctrl, 0, total, st) != cudaSuccess) return PITN_ECUDA;
    cudaError_t e;
    if (mixed) {
        switch (system_id) {
        case PITN_LORENZ63: e = launch_small<Lorenz63, true>(a, grid, block, st); break;
        case PITN_VDP: e = launch_small<VanDerPol, true>(a, grid, block, st); break;
        default: e = launch_small<LinearOsc, true>(a, grid, block, st); break;
        }
    } else if (rk4 && system_id == PITN_VDP) e = launch_small<RK4Map<VdpRhs>>(a, grid, block, st);
    else if (rk4) e = launch_small<RK4Map<LogisticRhs>>(a, grid, block, st);
    else {
        switch (system_id) {
        case PITN_LORENZ63: e = launch_small<Lorenz63>(a, grid, block, st); break;
        case PITN_VDP: e = launch_small<VanDerPol>(a, grid, block, st); break;
        case PITN_LOGISTIC: e = launch_small<EulerMap<LogisticRhs>>(a, grid, block, st); break;
        default: e = launch_small<LinearOsc>(a, grid, block, st); break;
        }
    }
    if (e != cudaSuccess) { cudaGetLastError(); return PITN_ECUDA; }
    int* h_err = (int*)hbuf;
    SolveRecord* h_rec = (SolveRecord*)(hbuf + 16);
    unsigned long long* h_hist = (unsigned long long*)(hbuf + 16 + sizeof(SolveRecord));
    if (cudaMemcpyAsync(h_err, ctrl + off_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_rec, ctrl + off_rec, sizeof(SolveRecord), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_hist, ctrl + off_res, sizeof(unsigned long long) * (max_iter + 1),
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
    return PITN_OK;
}

// Launch shapes the autotuner tries (threads per CTA, CTAs per SM).
static const int kSmallShapes[][2] = {{128, 1}, {128, 2}, {128, 3}, {128, 4}, {256, 1}, {256, 2}, {512, 1}};

int small_solve_full(int system_id, const SolveIO& io, double h, int64_t N, int d, double tol,
                     int max_iter, const pitn_options& o, cudaStream_t st, SolveOutcome* out) {
    int block = 0, cmin = 0;
    small_default_config(d, N, &block, &cmin);
    int cap = 2;
    const bool guarded = o.guard_B > 0.0 && std::isfinite(o.guard_B);
    char key[96];
    std::snprintf(key, sizeof(key), "small:%d:%d:%d:%d%s%s", system_id, d, tune_bucket(N), guarded ? 1 : 0,
                  o.method == PITN_STEP_RK4 ? ":rk4" : "", o.precision == PITN_PREC_MIXED_FP32 ? ":f32" : "");
    int tb = 0, tc = 0;
    if (tune_lookup(key, &tb, &tc)) {
        block = tb;
        cap = tc;
    } else if (tune_enabled() && !io.have_guess) {
        // time every shape on this very solve; the cost per Newton pass decides
        double best = 1e300;
        for (const auto& shp : kSmallShapes) {
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
            SolveOutcome tmp;
            const int rc = small_launch(system_id, io, h, N, d, tol, max_iter, o, st, &tmp, shp[0], shp[1]);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc != PITN_OK) continue;
            const double per_pass = ms / (double)(tmp.iters + 1);
            if (per_pass < best) {
                best = per_pass;
                block = shp[0];
                cap = shp[1];
            }
        }
        tune_store(key, block, cap);
    }
    return small_launch(system_id, io, h, N, d, tol, max_iter, o, st, out, block, cap);
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
constexpr size_t kNaScratch = kNaX1 + (size_t)kNaMaxSteps * 3;         // [N][6]
constexpr size_t kNaAgg = kNaScratch + (size_t)kNaMaxSteps * 6;        // [CTAs][12]
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
    switch (system_id) {
    case PITN_LORENZ63:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_small_kernel<Lorenz63>, block, 0);
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
    void* args[] = {(void*)&a};
    const void* kern = (system_id == PITN_LORENZ63) ? (const void*)newton_small_kernel<Lorenz63>
                       : (system_id == PITN_VDP)    ? (const void*)newton_small_kernel<VanDerPol>
                                                    : (const void*)newton_small_kernel<LinearOsc>;
    if (cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(block), args, 0, st) != cudaSuccess) {
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
