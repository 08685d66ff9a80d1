// batch.cu -- B independent IVPs of uneven length solved together
// (pitn_solve_batch): one segmented scan per Newton iteration.
//
// The trajectories are concatenated (IVP b occupies global steps
// offsets[b] .. offsets[b+1]-1).  The first element of every IVP has matrix
// 0 (eq. 3.4), and an element with matrix 0 cuts every dependency on the
// elements before it, so the segmented scan is the ordinary affine scan over
// the concatenation: no head flags are needed inside the combine.
// Per Newton iteration four kernels run (captured once into a CUDA graph and
// replayed):
//   A  residual + compact Jacobian + thread fold + block scan; each CTA
//      stores its aggregate and every thread its exclusive prefix within the
//      CTA; per-IVP ||r||_inf by atomics;
//   D  per IVP: stop test (non-finite -> NONFINITE, ||r|| <= tol -> OK,
//      max_iter -> NOT_CONVERGED); an IVP that stops is frozen;
//   C  per CTA: incoming prefix from the aggregates of the preceding CTAs
//      back to the one holding the head of its first IVP (fixed order, so
//      results are deterministic); replay, update into the IVP's other
//      buffer, per-IVP first guard cut;
//   E  per IVP: accept the step (flip the IVP's buffer, set its guard fill)
//      or stop it (plain Newton, non-finite correction); counts the IVPs
//      still running.
// Each IVP keeps its own current buffer and guard fill, so frozen IVPs are
// never copied.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "newton_small.cuh"   // the reduced-precision scan policies (scan_policy.cuh)
#include "solver.h"
#include "systems.cuh"

namespace pitn {

struct IvpState {
    long long q;            // lazy-fill index of the current iterate
    long long guard_index;  // cut of the last update
    unsigned long long res; // ||r||_inf bits of this iteration
    unsigned long long qenc;// max of ~cut of this iteration
    double final_res;
    int cur;                // buffer holding the current iterate
    int active;             // residual evaluated this iteration
    int stepping;           // Newton step applied this iteration
    int iters;
    int status;
    int pad;
};

struct BatchArgs {
    const double* params;   // [B][P]
    const double* x0;       // [B][d]
    const double* h;        // [B]
    const long long* off;   // [B+1]
    double* X0;
    double* X1;
    double* scratch;        // [M][JN + D]
    double* agg;            // [G][E]
    double* texcl;          // [G*block][E]
    IvpState* st;           // [B]
    unsigned* running;      // [0] IVPs still running after the iteration, [1] iterations run,
                            // [2..3] next IVP of the per-IVP queue (64-bit)
    unsigned long long* work;  // [2] per-IVP path: steps evaluated (residual, Jacobian, fold), steps replayed
    long long B, M, chunk;
    double tol;
    unsigned long long cap_bits;
    int guarded, max_iter;
};

constexpr unsigned long long kInf = 0x7ff0000000000000ull;
constexpr int kBWarps = 8;
constexpr int kIvpWarps = 16;   // per-IVP path: up to 512 threads per CTA

template <int D>
__device__ __forceinline__ void b_identity(double* P) {
#pragma unroll
    for (int i = 0; i < D * D; ++i) P[i] = (i % (D + 1) == 0) ? 1.0 : 0.0;
}
template <int D>
__device__ __forceinline__ void b_compose(const double* P2, const double* c2, const double* P1,
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
template <int D>
__device__ __forceinline__ void b_apply(const double* P, const double* c, const double* v, double* o) {
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

// IVP holding global step k (largest b with off[b] <= k).
__device__ __forceinline__ long long seg_of(const long long* __restrict__ off, long long B, long long k) {
    long long lo = 0, hi = B;  // off[lo] <= k < off[hi]
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (off[mid] <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int D>
__device__ __forceinline__ void b_state(const BatchArgs& a, const IvpState& s, long long b, long long base,
                                        long long j, double* o) {
    const double* X = s.cur ? a.X1 : a.X0;
    const double* src;
    if (j < 0) src = a.x0 + b * D;
    else if (j < s.q) src = X + (base + j) * D;
    else if (s.q > 0) src = X + (base + s.q - 1) * D;
    else src = a.x0 + b * D;
#pragma unroll
    for (int i = 0; i < D; ++i) o[i] = src[i];
}

template <int D>
__device__ __forceinline__ void b_flush_res(const BatchArgs& a, long long b, unsigned long long v) {
    if (v) atomicMax(&a.st[b].res, v);
}

// Whether any IVP overlapping the steps [kf, kl) is active (stepping: has a
// Newton step to apply).  A CTA whose steps all belong to frozen IVPs skips
// the pass: late in a batch, when most IVPs have converged, the scans of
// their identity elements would otherwise cost as much as real work.
__device__ __forceinline__ bool cta_has_work(const BatchArgs& a, long long kf, long long kl, bool stepping) {
    __shared__ int s_any;
    if (threadIdx.x == 0) {
        int any = 0;
        if (kf < a.M) {
            const long long kend = min(kl, a.M);
            for (long long b = seg_of(a.off, a.B, kf); b < a.B && a.off[b] < kend; ++b) {
                if (stepping ? a.st[b].stepping : a.st[b].active) {
                    any = 1;
                    break;
                }
            }
        }
        s_any = any;
    }
    __syncthreads();
    return s_any != 0;
}

// Adds a thread's step counts (evaluated, replayed) to the solve's totals;
// every thread of the warp calls it.
__device__ __forceinline__ void b_flush_work(const BatchArgs& a, unsigned long long ev, unsigned long long rep) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, off);
        rep += __shfl_xor_sync(0xffffffffu, rep, off);
    }
    if ((threadIdx.x & 31) == 0 && a.work) {
        atomicAdd(a.work, ev);
        atomicAdd(a.work + 1, rep);
    }
}

// ---- A ----------------------------------------------------------------------
template <class Sys>
__global__ void __launch_bounds__(256) batch_fold_kernel(BatchArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D, W = JN + D;
    __shared__ double s_w[kBWarps][E];
    __shared__ double s_tot[E];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k0 = gt * a.chunk;
    const long long k1 = min(a.M, k0 + a.chunk);
    {
        const long long kf = (long long)blockIdx.x * blockDim.x * a.chunk;
        if (!cta_has_work(a, kf, kf + (long long)blockDim.x * a.chunk, false)) {
            // all frozen: the CTA aggregate is the identity (no thread prefix is read)
            if (threadIdx.x < E)
                a.agg[(size_t)blockIdx.x * E + threadIdx.x] =
                    (threadIdx.x < D * D && threadIdx.x % (D + 1) == 0) ? 1.0 : 0.0;
            return;
        }
    }

    double P[D * D], c[D];
    b_identity<D>(P);
#pragma unroll
    for (int j = 0; j < D; ++j) c[j] = 0.0;
    long long b = -1, base = 0, next = 0;
    unsigned long long mres = 0ull, n_ev = 0ull;
    IvpState s{};
    Sys sys;
    double xp[D];
    for (long long k = k0; k < k1; ++k) {
        if (k >= next || b < 0) {
            if (b >= 0) b_flush_res<D>(a, b, mres);
            mres = 0ull;
            b = (b < 0) ? seg_of(a.off, a.B, k) : b + 1;
            while (a.off[b + 1] <= k) ++b;  // skip empty segments (not produced by the API)
            base = a.off[b];
            next = a.off[b + 1];
            s = a.st[b];
            sys.init(a.params + b * Sys::P, a.h[b]);
            if (s.active) b_state<D>(a, s, b, base, k - base - 1, xp);
        }
        if (!s.active) continue;  // frozen IVP: identity element
        const long long j = k - base;
        {
            // steps from the guard's fill start on all hold x_{q-1} (x0 at the
            // constant guess): this chunk's share of them is one element,
            // raised to its count by binary powering; their scratch rows are
            // not written (the replay evaluates the element itself)
            const long long nb = next - base;
            const long long sf = (s.q < nb) ? (s.q > 1 ? s.q : 1LL) : nb;
            if (j >= sf) {
                const long long kend = min(k1, next);
                double xf[D], rf[D], jvf[JN], EP[D * D], Ec[D], RP[D * D], Rc[D];
                b_state<D>(a, s, b, base, s.q - 1, xf);
                sys.eval(xf, xf, rf, jvf);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const unsigned long long bits = abs_bits(rf[i]);
                    mres = bits > mres ? bits : mres;
                    Ec[i] = -rf[i];
                    Rc[i] = 0.0;
                }
                ++n_ev;
                sys.jfull(jvf, EP);
                b_identity<D>(RP);
                for (long long e = kend - k;;) {
                    if (e & 1) b_compose<D>(EP, Ec, RP, Rc, RP, Rc);
                    e >>= 1;
                    if (!e) break;
                    b_compose<D>(EP, Ec, EP, Ec, EP, Ec);
                }
                b_compose<D>(RP, Rc, P, c, P, c);
                k = kend - 1;   // the IVP's last step in this chunk
                continue;
            }
        }
        double x[D], r[D], jv[JN];
        b_state<D>(a, s, b, base, j, x);
        sys.eval(xp, x, r, jv);
        ++n_ev;
#pragma unroll
        for (int i = 0; i < JN; ++i) a.scratch[k * W + i] = jv[i];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            a.scratch[k * W + JN + i] = r[i];
            const unsigned long long bits = abs_bits(r[i]);
            mres = bits > mres ? bits : mres;
        }
        if (j == 0) {
#pragma unroll
            for (int i = 0; i < D * D; ++i) P[i] = 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i) c[i] = -r[i];
        } else {
            double tP[D * D], tc[D];
            sys.jmul(jv, P, tP);
            sys.jvec_sub(jv, c, r, tc);
#pragma unroll
            for (int i = 0; i < D * D; ++i) P[i] = tP[i];
#pragma unroll
            for (int i = 0; i < D; ++i) c[i] = tc[i];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) xp[i] = x[i];
    }
    // per-IVP residual: one atomic per warp when the warp ends in one IVP
    {
        const long long b0 = __shfl_sync(0xffffffffu, b, 0);
        const bool uniform = __all_sync(0xffffffffu, b == b0);
        if (uniform) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, mres, off);
                mres = o > mres ? o : mres;
            }
            if (lane == 0 && b >= 0) b_flush_res<D>(a, b, mres);
        } else if (b >= 0) {
            b_flush_res<D>(a, b, mres);
        }
    }
    // block scan: thread exclusive (lane part composed onto warp part), CTA total
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        double uP[D * D], uc[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) uP[i] = __shfl_up_sync(0xffffffffu, P[i], off);
#pragma unroll
        for (int i = 0; i < D; ++i) uc[i] = __shfl_up_sync(0xffffffffu, c[i], off);
        if (lane >= off) b_compose<D>(P, c, uP, uc, P, c);
    }
    double eP[D * D], ec[D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) eP[i] = __shfl_up_sync(0xffffffffu, P[i], 1);
#pragma unroll
    for (int i = 0; i < D; ++i) ec[i] = __shfl_up_sync(0xffffffffu, c[i], 1);
    if (lane == 0) {
        b_identity<D>(eP);
#pragma unroll
        for (int i = 0; i < D; ++i) ec[i] = 0.0;
    }
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < D * D; ++i) s_w[warp][i] = P[i];
#pragma unroll
        for (int i = 0; i < D; ++i) s_w[warp][D * D + i] = c[i];
    }
    __syncthreads();
    if (warp == 0) {
        double wP[D * D], wc[D];
        if (lane < nwarps) {
#pragma unroll
            for (int i = 0; i < D * D; ++i) wP[i] = s_w[lane][i];
#pragma unroll
            for (int i = 0; i < D; ++i) wc[i] = s_w[lane][D * D + i];
        } else {
            b_identity<D>(wP);
#pragma unroll
            for (int i = 0; i < D; ++i) wc[i] = 0.0;
        }
#pragma unroll
        for (int off = 1; off < kBWarps; off <<= 1) {
            double uP[D * D], uc[D];
#pragma unroll
            for (int i = 0; i < D * D; ++i) uP[i] = __shfl_up_sync(0xffffffffu, wP[i], off);
#pragma unroll
            for (int i = 0; i < D; ++i) uc[i] = __shfl_up_sync(0xffffffffu, wc[i], off);
            if (lane >= off) b_compose<D>(wP, wc, uP, uc, wP, wc);
        }
        double xP[D * D], xc[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) xP[i] = __shfl_up_sync(0xffffffffu, wP[i], 1);
#pragma unroll
        for (int i = 0; i < D; ++i) xc[i] = __shfl_up_sync(0xffffffffu, wc[i], 1);
        __syncwarp();
        if (lane < nwarps) {
            if (lane == 0) {
                b_identity<D>(xP);
#pragma unroll
                for (int i = 0; i < D; ++i) xc[i] = 0.0;
            }
#pragma unroll
            for (int i = 0; i < D * D; ++i) s_w[lane][i] = xP[i];
#pragma unroll
            for (int i = 0; i < D; ++i) s_w[lane][D * D + i] = xc[i];
        }
        if (lane == nwarps - 1) {
#pragma unroll
            for (int i = 0; i < D * D; ++i) s_tot[i] = wP[i];
#pragma unroll
            for (int i = 0; i < D; ++i) s_tot[D * D + i] = wc[i];
        }
    }
    __syncthreads();
    // thread exclusive = lane-exclusive o warp-exclusive
    double tP[D * D], tc[D];
    b_compose<D>(eP, ec, s_w[warp], s_w[warp] + D * D, tP, tc);
    double* te = a.texcl + (size_t)gt * E;
#pragma unroll
    for (int i = 0; i < D * D; ++i) te[i] = tP[i];
#pragma unroll
    for (int i = 0; i < D; ++i) te[D * D + i] = tc[i];
    if (threadIdx.x < E) a.agg[(size_t)blockIdx.x * E + threadIdx.x] = s_tot[threadIdx.x];
    b_flush_work(a, n_ev, 0ull);
}

// ---- D ----------------------------------------------------------------------
__global__ void batch_decide_kernel(BatchArgs a) {
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < a.B;
         b += (long long)gridDim.x * blockDim.x) {
        IvpState s = a.st[b];
        s.stepping = 0;
        if (s.active) {
            const double res = __longlong_as_double((long long)s.res);
            s.final_res = res;
            if (s.res >= kInf) { s.status = PITN_NONFINITE; s.active = 0; }
            else if (res <= a.tol) { s.status = PITN_OK; s.active = 0; }
            else if (s.iters >= a.max_iter) { s.status = PITN_NOT_CONVERGED; s.active = 0; }
            else s.stepping = 1;
        }
        a.st[b] = s;
    }
}

// ---- C ----------------------------------------------------------------------
template <class Sys>
__global__ void __launch_bounds__(256) batch_replay_kernel(BatchArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D, W = JN + D;
    __shared__ double s_zin[D];
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k0 = gt * a.chunk;
    const long long k1 = min(a.M, k0 + a.chunk);
    const long long cta_span = (long long)blockDim.x * a.chunk;
    if (!cta_has_work(a, (long long)blockIdx.x * cta_span, (long long)(blockIdx.x + 1) * cta_span, true)) return;
    if (threadIdx.x == 0) {
        // incoming prefix of this CTA
        double z[D];
#pragma unroll
        for (int i = 0; i < D; ++i) z[i] = 0.0;
        const long long kf = (long long)blockIdx.x * cta_span;
        if (kf < a.M && blockIdx.x > 0) {
            const long long b0 = seg_of(a.off, a.B, kf);
            const long long head = a.off[b0];
            if (head < kf) {
                const long long c0 = head / cta_span;  // CTA holding the head
                for (long long cc = c0; cc < blockIdx.x; ++cc) {
                    const double* g = a.agg + (size_t)cc * E;
                    double t[D];
                    b_apply<D>(g, g + D * D, z, t);
#pragma unroll
                    for (int i = 0; i < D; ++i) z[i] = t[i];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) s_zin[i] = z[i];
    }
    __syncthreads();
    unsigned long long n_rep = 0ull;
    double z[D];
    if (k0 < k1) {
        const double* te = a.texcl + (size_t)gt * E;
        double tP[D * D], tc[D], zi[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) tP[i] = te[i];
#pragma unroll
        for (int i = 0; i < D; ++i) { tc[i] = te[D * D + i]; zi[i] = s_zin[i]; }
        b_apply<D>(tP, tc, zi, z);
    }
    long long b = -1, base = 0, next = 0, sf = 0;
    IvpState s{};
    Sys sys;
    bool found = false, have_fill = false;
    double xf[D], rf[D], jvf[JN];   // the IVP's fill element (its scratch rows are not written)
    for (long long k = k0; k < k1; ++k) {
        if (k >= next || b < 0) {
            b = (b < 0) ? seg_of(a.off, a.B, k) : b + 1;
            while (a.off[b + 1] <= k) ++b;
            base = a.off[b];
            next = a.off[b + 1];
            s = a.st[b];
            sys.init(a.params + b * Sys::P, a.h[b]);
            found = false;
            have_fill = false;
            const long long nb = next - base;
            sf = (s.q < nb) ? (s.q > 1 ? s.q : 1LL) : nb;
        }
        if (!s.stepping) continue;
        if (found) {   // past this thread's first cut: never read again
            k = next - 1;
            continue;
        }
        const long long j = k - base;
        double jv[JN], r[D], x[D];
        if (j < sf) {
#pragma unroll
            for (int i = 0; i < JN; ++i) jv[i] = a.scratch[k * W + i];
#pragma unroll
            for (int i = 0; i < D; ++i) r[i] = a.scratch[k * W + JN + i];
            b_state<D>(a, s, b, base, j, x);
        } else {
            if (!have_fill) {
                b_state<D>(a, s, b, base, s.q - 1, xf);
                sys.eval(xf, xf, rf, jvf);
                have_fill = true;
            }
#pragma unroll
            for (int i = 0; i < JN; ++i) jv[i] = jvf[i];
#pragma unroll
            for (int i = 0; i < D; ++i) { r[i] = rf[i]; x[i] = xf[i]; }
        }
        if (j == 0) {
#pragma unroll
            for (int i = 0; i < D; ++i) z[i] = -r[i];
        } else {
            double tz[D];
            sys.jvec_sub(jv, z, r, tz);
#pragma unroll
            for (int i = 0; i < D; ++i) z[i] = tz[i];
        }
        double* Xn = s.cur ? a.X0 : a.X1;
        unsigned long long zb = 0ull;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            Xn[k * D + i] = x[i] + z[i];
            const unsigned long long bits = abs_bits(z[i]);
            zb = bits > zb ? bits : zb;
        }
        ++n_rep;
        if (!found && zb > a.cap_bits) {
            found = true;
            atomicMax(&a.st[b].qenc, ~(unsigned long long)j);
        }
    }
    b_flush_work(a, 0ull, n_rep);   // (threads without steps took no pass through the loop)
}

// ---- E ----------------------------------------------------------------------
__global__ void batch_end_kernel(BatchArgs a) {
    unsigned running = 0;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < a.B;
         b += (long long)gridDim.x * blockDim.x) {
        IvpState s = a.st[b];
        if (s.stepping) {
            const long long n = a.off[b + 1] - a.off[b];
            const long long cut = s.qenc ? (long long)(~s.qenc) : n;
            if (!a.guarded && cut < n) {
                s.status = PITN_NONFINITE;
                s.active = 0;
            } else {
                s.cur ^= 1;
                s.q = a.guarded ? cut : n;
                s.guard_index = cut;
                s.iters += 1;
            }
            s.stepping = 0;
        }
        s.res = 0ull;
        s.qenc = 0ull;
        running += s.active ? 1u : 0u;
        a.st[b] = s;
    }
    if (running) atomicAdd(a.running, running);
}

// ---- init / finalize --------------------------------------------------------
// ---- per-IVP solve ----------------------------------------------------------
// Exclusive scan of the CTA's per-thread elements in thread order (later on
// the left): Kogge-Stone within each warp, then over the warp totals.
template <int D>
__device__ __forceinline__ void b_cta_scan(double* P, double* c, double (*s_w)[D * D + D], double* tP,
                                           double* tc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        double uP[D * D], uc[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) uP[i] = __shfl_up_sync(0xffffffffu, P[i], off);
#pragma unroll
        for (int i = 0; i < D; ++i) uc[i] = __shfl_up_sync(0xffffffffu, c[i], off);
        if (lane >= off) b_compose<D>(P, c, uP, uc, P, c);
    }
    double eP[D * D], ec[D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) eP[i] = __shfl_up_sync(0xffffffffu, P[i], 1);
#pragma unroll
    for (int i = 0; i < D; ++i) ec[i] = __shfl_up_sync(0xffffffffu, c[i], 1);
    if (lane == 0) {
        b_identity<D>(eP);
#pragma unroll
        for (int i = 0; i < D; ++i) ec[i] = 0.0;
    }
    __syncthreads();   // s_w may still be read from the previous scan
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < D * D; ++i) s_w[warp][i] = P[i];
#pragma unroll
        for (int i = 0; i < D; ++i) s_w[warp][D * D + i] = c[i];
    }
    __syncthreads();
    if (warp == 0) {
        double wP[D * D], wc[D];
        if (lane < nwarps) {
#pragma unroll
            for (int i = 0; i < D * D; ++i) wP[i] = s_w[lane][i];
#pragma unroll
            for (int i = 0; i < D; ++i) wc[i] = s_w[lane][D * D + i];
        } else {
            b_identity<D>(wP);
#pragma unroll
            for (int i = 0; i < D; ++i) wc[i] = 0.0;
        }
#pragma unroll
        for (int off = 1; off < kIvpWarps; off <<= 1) {
            if (off >= nwarps) break;
            double uP[D * D], uc[D];
#pragma unroll
            for (int i = 0; i < D * D; ++i) uP[i] = __shfl_up_sync(0xffffffffu, wP[i], off);
#pragma unroll
            for (int i = 0; i < D; ++i) uc[i] = __shfl_up_sync(0xffffffffu, wc[i], off);
            if (lane >= off) b_compose<D>(wP, wc, uP, uc, wP, wc);
        }
        double xP[D * D], xc[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) xP[i] = __shfl_up_sync(0xffffffffu, wP[i], 1);
#pragma unroll
        for (int i = 0; i < D; ++i) xc[i] = __shfl_up_sync(0xffffffffu, wc[i], 1);
        __syncwarp();
        if (lane < nwarps) {
            if (lane == 0) {
                b_identity<D>(xP);
#pragma unroll
                for (int i = 0; i < D; ++i) xc[i] = 0.0;
            }
#pragma unroll
            for (int i = 0; i < D * D; ++i) s_w[lane][i] = xP[i];
#pragma unroll
            for (int i = 0; i < D; ++i) s_w[lane][D * D + i] = xc[i];
        }
    }
    __syncthreads();
    b_compose<D>(eP, ec, s_w[warp], s_w[warp] + D * D, tP, tc);
}

// Work weight of a regular step against a fill step in the per-IVP path's
// partition of an IVP's steps over the CTA's threads.  Past the iteration's
// new cut a fill step costs nothing (its replay has stopped, and the fold
// powers one element), before it only its replay.
constexpr long long kBatchFillWeight = 4;


// One CTA solves whole IVPs, taken from a queue in the host's order (longest
// first): the Newton loop of each IVP runs with CTA-level scans only, so no
// IVP waits on another and nothing synchronises the grid.  Per iteration:
// residuals, compact Jacobians and thread folds over contiguous chunks
// (eqs. 3.8, 3.9, 3.4), the CTA scan (eq. 3.3), the decision on ||r||_inf,
// the replay of the Newton step (eq. 3.13) into the other buffer with the
// guard's first cut.  The IVP's record is left as the graph path leaves it.
template <class Sys>
__global__ void __launch_bounds__(512) batch_ivp_kernel(BatchArgs a, const long long* __restrict__ order,
                                                        unsigned long long* __restrict__ queue) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D, W = JN + D;
    __shared__ double s_w[kIvpWarps][E];
    __shared__ long long s_b;
    __shared__ unsigned long long s_res, s_q;
    const int lane = threadIdx.x & 31;
    unsigned long long n_ev = 0ull, n_rep = 0ull;   // steps evaluated / replayed by this thread
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long i = atomicAdd(queue, 1ull);
            s_b = (i < (unsigned long long)a.B) ? order[i] : -1;
        }
        __syncthreads();
        const long long b = s_b;
        if (b < 0) break;
        const long long base = a.off[b], n = a.off[b + 1] - base;
        Sys sys;
        sys.init(a.params + b * Sys::P, a.h[b]);
        const double* x0 = a.x0 + b * D;
        double* const XA = a.X0 + base * D;
        double* const XB = a.X1 + base * D;
        double* scr = a.scratch + base * W;
        const long long T = blockDim.x;
        int cur = 0, it = 0, status = PITN_NOT_CONVERGED;
        long long q = 0, last_cut = n;
        double final_res = 0.0;
        auto state = [&](const double* X, long long j, double* o) {
            const double* src;
            if (j < 0) src = x0;
            else if (j < q) src = X + j * D;
            else if (q > 0) src = X + (q - 1) * D;
            else src = x0;
#pragma unroll
            for (int i = 0; i < D; ++i) o[i] = src[i];
        };
        for (;; ++it) {
            const double* Xc = cur ? XB : XA;
            double* Xn = cur ? XA : XB;
            if (threadIdx.x == 0) { s_res = 0ull; s_q = 0ull; }
            // Steps from sfill on lie in the guard's fill region (every state
            // x_{q-1}; at the constant guess every state x0): all their
            // elements are the same element, folded by binary powering.  The
            // steps are dealt out to the threads by their work weight
            // (kBatchFillWeight), each thread a contiguous range.
            const long long sfill = (q < n) ? (q > 1 ? q : 1LL) : n;
            long long k0, k1;
            {
                constexpr long long kw = kBatchFillWeight;
                const long long wreg = kw * sfill, wtot = wreg + (n - sfill);
                const long long per = (wtot + T - 1) / T;
                const long long w0 = (long long)threadIdx.x * per, w1 = w0 + per;
                k0 = min(n, (w0 <= wreg) ? (w0 + kw - 1) / kw : sfill + (w0 - wreg));
                k1 = min(n, (w1 <= wreg) ? (w1 + kw - 1) / kw : sfill + (w1 - wreg));
            }
            const long long kreg = min(k1, max(k0, sfill));   // regular steps: [k0, kreg)
            // residuals, Jacobians and the thread fold
            double P[D * D], c[D];
            b_identity<D>(P);
#pragma unroll
            for (int i = 0; i < D; ++i) c[i] = 0.0;
            unsigned long long mres = 0ull;
            if (k0 < kreg) {
                double xp[D];
                state(Xc, k0 - 1, xp);
                for (long long k = k0; k < kreg; ++k) {
                    double x[D], r[D], jv[JN];
                    state(Xc, k, x);
                    sys.eval(xp, x, r, jv);
#pragma unroll
                    for (int i = 0; i < JN; ++i) scr[k * W + i] = jv[i];
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        scr[k * W + JN + i] = r[i];
                        const unsigned long long bits = abs_bits(r[i]);
                        mres = bits > mres ? bits : mres;
                    }
                    if (k == 0) {
#pragma unroll
                        for (int i = 0; i < D * D; ++i) P[i] = 0.0;
#pragma unroll
                        for (int i = 0; i < D; ++i) c[i] = -r[i];
                    } else {
                        double tP[D * D], tc[D];
                        sys.jmul(jv, P, tP);
                        sys.jvec_sub(jv, c, r, tc);
#pragma unroll
                        for (int i = 0; i < D * D; ++i) P[i] = tP[i];
#pragma unroll
                        for (int i = 0; i < D; ++i) c[i] = tc[i];
                    }
#pragma unroll
                    for (int i = 0; i < D; ++i) xp[i] = x[i];
                }
            }
            n_ev += (unsigned long long)(kreg - k0) + (kreg < k1 ? 1ull : 0ull);
            double xf[D], rf[D], jvf[JN];
            if (kreg < k1) {   // the fill element (J(x_f), -r_f), raised to the power k1 - kreg
                double EP[D * D], Ec[D], RP[D * D], Rc[D];
                state(Xc, q - 1, xf);
                sys.eval(xf, xf, rf, jvf);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const unsigned long long bits = abs_bits(rf[i]);
                    mres = bits > mres ? bits : mres;
                    Ec[i] = -rf[i];
                    Rc[i] = 0.0;
                }
                sys.jfull(jvf, EP);
                b_identity<D>(RP);
                for (long long e = k1 - kreg;;) {
                    if (e & 1) b_compose<D>(EP, Ec, RP, Rc, RP, Rc);
                    e >>= 1;
                    if (!e) break;
                    b_compose<D>(EP, Ec, EP, Ec, EP, Ec);
                }
                b_compose<D>(RP, Rc, P, c, P, c);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, mres, off);
                mres = o > mres ? o : mres;
            }
            double tP[D * D], tc[D];
            b_cta_scan<D>(P, c, s_w, tP, tc);   // (its barriers also order s_res's reset)
            if (lane == 0 && mres) atomicMax(&s_res, mres);
            __syncthreads();
            const unsigned long long rb = s_res;
            final_res = __longlong_as_double((long long)rb);
            if (rb >= kInf) { status = PITN_NONFINITE; break; }
            if (final_res <= a.tol) { status = PITN_OK; break; }
            if (it >= a.max_iter) { status = PITN_NOT_CONVERGED; break; }
            // replay of the Newton step from the thread's incoming vector (the
            // element of step 0 has matrix 0, so the prefix's vector is it).  A
            // thread stops at its first cut: every later state of its range
            // lies beyond the iteration's cut and is never read again.
            unsigned long long my_q = 0ull;
            if (k0 < k1) {
                double z[D];
#pragma unroll
                for (int i = 0; i < D; ++i) z[i] = tc[i];
                bool found = false;
                auto step = [&](long long k, const double* jv, const double* r, const double* x) {
                    ++n_rep;
                    if (k == 0) {
#pragma unroll
                        for (int i = 0; i < D; ++i) z[i] = -r[i];
                    } else {
                        double tz[D];
                        sys.jvec_sub(jv, z, r, tz);
#pragma unroll
                        for (int i = 0; i < D; ++i) z[i] = tz[i];
                    }
                    unsigned long long zb = 0ull;
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        Xn[k * D + i] = x[i] + z[i];
                        const unsigned long long bits = abs_bits(z[i]);
                        zb = bits > zb ? bits : zb;
                    }
                    if (zb > a.cap_bits) {
                        found = true;
                        my_q = ~(unsigned long long)k;
                    }
                };
                for (long long k = k0; k < kreg && !found; ++k) {
                    double jv[JN], r[D], x[D];
#pragma unroll
                    for (int i = 0; i < JN; ++i) jv[i] = scr[k * W + i];
#pragma unroll
                    for (int i = 0; i < D; ++i) r[i] = scr[k * W + JN + i];
                    state(Xc, k, x);
                    step(k, jv, r, x);
                }
                for (long long k = kreg; k < k1 && !found; ++k) step(k, jvf, rf, xf);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_q, off);
                my_q = o > my_q ? o : my_q;
            }
            if (lane == 0 && my_q) atomicMax(&s_q, my_q);
            __syncthreads();
            const unsigned long long qe = s_q;
            const long long cut = qe ? (long long)(~qe) : n;
            __syncthreads();   // s_res / s_q are reset at the top of the next iteration
            if (!a.guarded && cut < n) { status = PITN_NONFINITE; break; }
            q = a.guarded ? cut : n;
            cur ^= 1;
            last_cut = cut;
        }
        if (threadIdx.x == 0) {
            IvpState s = a.st[b];
            s.cur = cur;
            s.q = q;
            s.iters = it;
            s.status = status;
            s.final_res = final_res;
            s.guard_index = last_cut;
            s.active = 0;
            s.stepping = 0;
            a.st[b] = s;
        }
        __syncthreads();   // s_b is overwritten by the next pick
    }
    b_flush_work(a, n_ev, n_rep);
}

// The per-IVP solve with a reduced-precision scan (an inexact Newton step):
// the same Newton loop, with the residual, the stopping test and the update
// in FP64 and the elements, folds, CTA scan and replay in the scan policy's
// arithmetic (scan_policy.cuh: ScanF32, the FP32 delta form; ScanFF,
// float-float).  The scratch holds the policy's values (at most 8 bytes
// each, in the FP64 path's slots).
template <class Sys, class Pol>
__global__ void __launch_bounds__(Pol::kBatchThreads, Pol::kBatchMinBlocks) batch_ivp_mixed_kernel(BatchArgs a, const long long* __restrict__ order,
                                                              unsigned long long* __restrict__ queue) {
    using T = typename Pol::T;
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D, W = JN + D;
    static_assert(sizeof(T) <= sizeof(double), "scratch slots are 8 bytes");
    static_assert(Pol::kBatchThreads <= kMaxWarps * 32, "the policy's CTA scan holds kMaxWarps warps");
    __shared__ T s_wex[kMaxWarps][E];
    __shared__ T s_tot[E];
    __shared__ long long s_b;
    __shared__ unsigned long long s_res, s_q;
    const int lane = threadIdx.x & 31;
    const float capf = (float)fmin(__longlong_as_double((long long)a.cap_bits), (double)FLT_MAX);
    unsigned long long n_ev = 0ull, n_rep = 0ull;   // steps evaluated / replayed by this thread
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long i = atomicAdd(queue, 1ull);
            s_b = (i < (unsigned long long)a.B) ? order[i] : -1;
        }
        __syncthreads();
        const long long b = s_b;
        if (b < 0) break;
        const long long base = a.off[b], n = a.off[b + 1] - base;
        Sys sys;
        sys.init(a.params + b * Sys::P, a.h[b]);
        Pol::setup_ivp(sys, a.params + b * Sys::P, a.h[b]);
        const double* x0 = a.x0 + b * D;
        double* const XA = a.X0 + base * D;
        double* const XB = a.X1 + base * D;
        T* scr = reinterpret_cast<T*>(a.scratch + base * W);
        const long long Tn = blockDim.x;
        int cur = 0, it = 0, status = PITN_NOT_CONVERGED;
        long long q = 0, last_cut = n;
        double final_res = 0.0;
        auto state = [&](const double* X, long long j, double* o) {
            const double* src;
            if (j < 0) src = x0;
            else if (j < q) src = X + j * D;
            else if (q > 0) src = X + (q - 1) * D;
            else src = x0;
#pragma unroll
            for (int i = 0; i < D; ++i) o[i] = src[i];
        };
        for (;; ++it) {
            const double* Xc = cur ? XB : XA;
            double* Xn = cur ? XA : XB;
            if (threadIdx.x == 0) { s_res = 0ull; s_q = 0ull; }
            // regular steps [0, sfill) and the fill region, weighted as in
            // batch_ivp_kernel
            const long long sfill = (q < n) ? (q > 1 ? q : 1LL) : n;
            long long k0, k1;
            {
                constexpr long long kw = kBatchFillWeight;
                const long long wreg = kw * sfill, wtot = wreg + (n - sfill);
                const long long per = (wtot + Tn - 1) / Tn;
                const long long w0 = (long long)threadIdx.x * per, w1 = w0 + per;
                k0 = min(n, (w0 <= wreg) ? (w0 + kw - 1) / kw : sfill + (w0 - wreg));
                k1 = min(n, (w1 <= wreg) ? (w1 + kw - 1) / kw : sfill + (w1 - wreg));
            }
            const long long kreg = min(k1, max(k0, sfill));
            T Q[D * D], c[D];
            Pol::template ident<D>(Q, c);
            unsigned long long mres = 0ull;
            if (k0 < kreg) {
                double xp[D];
                state(Xc, k0 - 1, xp);
                for (long long k = k0; k < kreg; ++k) {
                    double x[D], r[D];
                    T sv[JN], rf[D];
                    state(Xc, k, x);
                    Pol::eval(sys, xp, x, r, sv);
#pragma unroll
                    for (int i = 0; i < JN; ++i) scr[k * W + i] = sv[i];
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        rf[i] = Pol::from_double(r[i]);
                        scr[k * W + JN + i] = rf[i];
                        const unsigned long long bits = abs_bits(r[i]);
                        mres = bits > mres ? bits : mres;
                    }
                    if (k == 0) Pol::template head<D>(rf, Q, c);   // a_0 = (0, -r_0), eq. 3.4
                    else Pol::leaf(sys, sv, rf, Q, c);
#pragma unroll
                    for (int i = 0; i < D; ++i) xp[i] = x[i];
                }
            }
            n_ev += (unsigned long long)(kreg - k0) + (kreg < k1 ? 1ull : 0ull);
            double xf[D];
            T svf[JN], rff[D];
            if (kreg < k1) {   // the fill element, raised to the power k1 - kreg
                double rf64[D];
                T EQ[D * D], Ec[D], RQ[D * D], Rc[D];
                state(Xc, q - 1, xf);
                Pol::eval(sys, xf, xf, rf64, svf);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    const unsigned long long bits = abs_bits(rf64[i]);
                    mres = bits > mres ? bits : mres;
                    rff[i] = Pol::from_double(rf64[i]);
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
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, mres, off);
                mres = o > mres ? o : mres;
            }
            T eQ[D * D], ec[D];
            pol_block_scan<Pol, D>(Q, c, eQ, ec, s_wex, s_tot);   // (its barriers order s_res's reset)
            if (lane == 0 && mres) atomicMax(&s_res, mres);
            __syncthreads();
            const unsigned long long rb = s_res;
            final_res = __longlong_as_double((long long)rb);
            if (rb >= kInf) { status = PITN_NONFINITE; break; }
            if (final_res <= a.tol) { status = PITN_OK; break; }
            if (it >= a.max_iter) { status = PITN_NOT_CONVERGED; break; }
            // replay from the thread's incoming vector, FP64 update; a thread
            // stops at its first cut
            unsigned long long my_q = 0ull;
            if (k0 < k1) {
                T z[D], zw[D], zero[D];
#pragma unroll
                for (int i = 0; i < D; ++i) zero[i] = Pol::zero();
                Pol::template apply<D>(s_wex[threadIdx.x >> 5], s_wex[threadIdx.x >> 5] + D * D, zero, zw);
                Pol::template apply<D>(eQ, ec, zw, z);
                bool found = false;
                auto step = [&](long long k, const T* sv, const T* rf, const double* x) {
                    ++n_rep;
                    if (k == 0) {
#pragma unroll
                        for (int i = 0; i < D; ++i) z[i] = Pol::neg(rf[i]);
                    } else {
                        Pol::replay(sys, sv, rf, z);
                    }
                    bool bad = false;
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        Xn[k * D + i] = Pol::add_to(x[i], z[i]);
                        bad |= !Pol::within(z[i], capf);
                    }
                    if (bad) {
                        found = true;
                        my_q = ~(unsigned long long)k;
                    }
                };
                for (long long k = k0; k < kreg && !found; ++k) {
                    T sv[JN], rf[D];
                    double x[D];
#pragma unroll
                    for (int i = 0; i < JN; ++i) sv[i] = scr[k * W + i];
#pragma unroll
                    for (int i = 0; i < D; ++i) rf[i] = scr[k * W + JN + i];
                    state(Xc, k, x);
                    step(k, sv, rf, x);
                }
                for (long long k = kreg; k < k1 && !found; ++k) step(k, svf, rff, xf);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_q, off);
                my_q = o > my_q ? o : my_q;
            }
            if (lane == 0 && my_q) atomicMax(&s_q, my_q);
            __syncthreads();
            const unsigned long long qe = s_q;
            const long long cut = qe ? (long long)(~qe) : n;
            __syncthreads();   // s_res / s_q are reset at the top of the next iteration
            if (!a.guarded && cut < n) { status = PITN_NONFINITE; break; }
            q = a.guarded ? cut : n;
            cur ^= 1;
            last_cut = cut;
        }
        if (threadIdx.x == 0) {
            IvpState s = a.st[b];
            s.cur = cur;
            s.q = q;
            s.iters = it;
            s.status = status;
            s.final_res = final_res;
            s.guard_index = last_cut;
            s.active = 0;
            s.stepping = 0;
            a.st[b] = s;
        }
        __syncthreads();   // s_b is overwritten by the next pick
    }
    b_flush_work(a, n_ev, n_rep);
}

__global__ void batch_init_kernel(BatchArgs a) {
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < a.B;
         b += (long long)gridDim.x * blockDim.x) {
        IvpState s{};
        const long long n = a.off[b + 1] - a.off[b];
        s.q = 0;  // constant guess x0
        s.guard_index = n;
        s.active = 1;
        s.status = PITN_NOT_CONVERGED;
        a.st[b] = s;
    }
}

template <int D>
__global__ void batch_finalize_kernel(BatchArgs a, double* out, int* iters_out, int* status_out,
                                      double* res_out, long long* off_out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long k = t0; k < a.M; k += stride) {
        const long long b = seg_of(a.off, a.B, k);
        const IvpState s = a.st[b];
        const long long base = a.off[b];
        if (s.cur == 0 && k - base < s.q && out == a.X0) continue;
        double v[D];
        b_state<D>(a, s, b, base, k - base, v);
#pragma unroll
        for (int i = 0; i < D; ++i) out[k * D + i] = v[i];
    }
    for (long long b = t0; b < a.B; b += stride) {
        const IvpState s = a.st[b];
        iters_out[b] = s.iters;
        status_out[b] = s.status;
        if (res_out) res_out[b] = s.final_res;
    }
    for (long long b = t0; b <= a.B; b += stride) off_out[b] = a.off[b];
}

}  // namespace pitn

namespace pitn_host {

using namespace pitn;

namespace {

// The loop condition of the batch graph: another iteration while an IVP is
// running and at most max_iter + 1 iterations have run (so the device loop
// always ends).
__global__ void batch_loop_kernel(BatchArgs a, cudaGraphConditionalHandle h) {
    const unsigned n = ++a.running[1];
    cudaGraphSetConditional(h, (a.running[0] != 0u && n <= (unsigned)a.max_iter) ? 1u : 0u);
}

// The per-IVP path: a persistent grid of CTAs takes IVPs from the queue
// (longest first) and solves each one whole.  `iterations` reports the
// launch count of the Newton loop (one).
// Pol: void for the FP64 solve, else the reduced-precision scan policy.
template <class Sys, class Pol = void>
int batch_run_ivp(BatchArgs& a, int block, cudaStream_t st, const long long* order, double* out,
                  int* iters_out, int* status_out, double* res_out, long long* off_out, int* iterations) {
    using Kern = void (*)(BatchArgs, const long long*, unsigned long long*);
    Kern kern;
    if constexpr (std::is_void<Pol>::value) {
        kern = batch_ivp_kernel<Sys>;
    } else {
        if (block > Pol::kBatchThreads) return PITN_EUNSUPPORTED;   // the kernel's launch bound
        kern = batch_ivp_mixed_kernel<Sys, Pol>;
    }
    const int eg = (int)std::min<long long>((a.B + 255) / 256, 1024);
    batch_init_kernel<<<eg, 256, 0, st>>>(a);
    count_launch(1);
    // the queue counter: 64 bits at byte 8 of the 16-byte `running` slot
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(a.running + 2);
    if (cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st) != cudaSuccess) return PITN_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0) != cudaSuccess)
        return PITN_ECUDA;
    if (per_sm < 1) return PITN_EUNSUPPORTED;
    const long long grid = std::min<long long>((long long)per_sm * props().multiProcessorCount, a.B);
    auto tok = timed_begin("batch", st);
    kern<<<(unsigned)grid, block, 0, st>>>(a, order, queue);
    timed_end(tok, st);
    count_launch(1);
    if (cudaGetLastError() != cudaSuccess) return PITN_ECUDA;
    *iterations = 1;
    batch_finalize_kernel<Sys::D><<<2048, 256, 0, st>>>(a, out, iters_out, status_out, res_out, off_out);
    count_launch(1);
    if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
    return PITN_OK;
}

template <class Sys>
int batch_run(BatchArgs& a, int block, long long grid, cudaStream_t st, unsigned* h_running,
              double* out, int* iters_out, int* status_out, double* res_out, long long* off_out,
              int* iterations) {
    const int eg = (int)std::min<long long>((a.B + 255) / 256, 1024);
    batch_init_kernel<<<eg, 256, 0, st>>>(a);
    count_launch(1);
    // the whole Newton loop as one CUDA graph: a conditional while node whose
    // body is one iteration (fold, decide, replay, end) and the loop kernel
    // that sets its condition, so the host waits once per solve
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PITN_ECUDA;
    int rc = PITN_OK;
    cudaGraphConditionalHandle cond{};
    cudaGraph_t body = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess ||
        cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
        rc = PITN_ECUDA;
    if (rc == PITN_OK) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) rc = PITN_ECUDA;
        else body = cp.conditional.phGraph_out[0];
    }
    if (rc == PITN_OK &&
        cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        rc = PITN_ECUDA;
    if (rc == PITN_OK) {
        cudaMemsetAsync(a.running, 0, sizeof(unsigned), cs);
        batch_fold_kernel<Sys><<<(unsigned)grid, block, 0, cs>>>(a);
        batch_decide_kernel<<<eg, 256, 0, cs>>>(a);
        batch_replay_kernel<Sys><<<(unsigned)grid, block, 0, cs>>>(a);
        batch_end_kernel<<<eg, 256, 0, cs>>>(a);
        batch_loop_kernel<<<1, 1, 0, cs>>>(a, cond);
        cudaGraph_t captured = nullptr;
        if (cudaStreamEndCapture(cs, &captured) != cudaSuccess) rc = PITN_ECUDA;
    }
    if (rc == PITN_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = PITN_ECUDA;
    // the graph runs on the caller's stream (ordered after the init kernel)
    *iterations = 0;
    if (rc == PITN_OK) {
        auto tok = timed_begin("batch", st);
        if (cudaMemsetAsync(a.running + 1, 0, sizeof(unsigned), st) != cudaSuccess ||
            cudaGraphLaunch(exec, st) != cudaSuccess ||
            cudaMemcpyAsync(h_running, a.running + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = PITN_ECUDA;
        timed_end(tok, st);
        if (rc == PITN_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = PITN_ECUDA;
        if (rc == PITN_OK) {
            *iterations = (int)*h_running;
            count_launch(5 * (int64_t)*iterations);
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc != PITN_OK) { cudaGetLastError(); return rc; }
    batch_finalize_kernel<Sys::D><<<2048, 256, 0, st>>>(a, out, iters_out, status_out, res_out, off_out);
    count_launch(1);
    if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
    return PITN_OK;
}

}  // namespace
}  // namespace pitn_host

using namespace pitn_host;

// step counts of the last batch solve in this process (pitn_batch_work)
static std::atomic<int64_t> g_batch_work[2];

extern "C" int pitn_batch_work(int64_t* evaluated, int64_t* replayed) {
    if (!evaluated || !replayed) return PITN_EINVAL;
    *evaluated = g_batch_work[0].load();
    *replayed = g_batch_work[1].load();
    return PITN_OK;
}

extern "C" int pitn_solve_batch(int system_id, int64_t B, const double* params, const double* x0,
                                const double* h, const int64_t* N, int d, double tol, int max_iter,
                                double* traj_out, int64_t* offsets_out, int32_t* iters_out,
                                int32_t* status_out, double* res_out, const pitn_options* opt) {
    pitn_options o{};
    if (opt) o = *opt;
    if ((system_id != PITN_LORENZ63 && system_id != PITN_VDP && system_id != PITN_LINEAR_OSC) ||
        !system_dim_ok(system_id, d))
        return PITN_EINVAL;
    if (B < 1 || !params || !x0 || !h || !N || !traj_out || !offsets_out || !iters_out || !status_out)
        return PITN_EINVAL;
    if (!std::isfinite(tol) || !(tol >= 0.0) || max_iter < 0 || max_iter > kMaxIter) return PITN_EINVAL;
    if ((o.precision != PITN_PREC_FP64 && o.precision != PITN_PREC_MIXED_FP32 &&
         o.precision != PITN_PREC_FP64_FF) ||
        o.guess || o.res_history || std::isnan(o.guard_B) || o.method != PITN_STEP_EULER)
        return PITN_EINVAL;
    // the reduced-precision scans run on the per-IVP path only
    const bool reduced = o.precision != PITN_PREC_FP64;
    if (o.tile_elems < 0) return PITN_EINVAL;
    if (any_foreign({params, x0, h, N, traj_out, offsets_out, iters_out, status_out, res_out}))
        return PITN_EINVAL;
    const int P = num_params(system_id);

    std::lock_guard<std::recursive_mutex> lk(api_mutex());
    cudaStream_t st = (cudaStream_t)o.stream;
    // lengths and offsets on the host (validated before any device work)
    std::vector<int64_t> hN((size_t)B), hoff((size_t)B + 1);
    if (is_device_ptr(N)) {
        if (cudaMemcpy(hN.data(), N, sizeof(int64_t) * B, cudaMemcpyDeviceToHost) != cudaSuccess)
            return PITN_ECUDA;
    } else {
        std::memcpy(hN.data(), N, sizeof(int64_t) * B);
    }
    std::vector<double> hh((size_t)B);
    if (fetch_to_host(h, (size_t)B, hh.data()) != PITN_OK) return PITN_ECUDA;
    hoff[0] = 0;
    for (int64_t b = 0; b < B; ++b) {
        if (hN[b] < 1 || hN[b] > kMaxSteps) return PITN_EINVAL;
        if (!std::isfinite(hh[b]) || !(hh[b] > 0.0)) return PITN_EINVAL;
        hoff[b + 1] = hoff[b] + hN[b];
        if (hoff[b + 1] > kMaxSteps) return PITN_EINVAL;
    }
    const long long M = hoff[B];

    // launch shape: threads per CTA and steps per thread (autotuned, see tune.cpp)
    int block = 256;
    long long chunk = o.tile_elems > 0 ? o.tile_elems : 32;
    const bool guarded_b = o.guard_B > 0.0 && std::isfinite(o.guard_B);
    char tkey[96];
    std::snprintf(tkey, sizeof(tkey), "batch:%d:%d:%d:%d%s", system_id, d, tune_bucket(M), guarded_b ? 1 : 0,
                  o.precision == PITN_PREC_MIXED_FP32 ? ":f32" : o.precision == PITN_PREC_FP64_FF ? ":ff" : "");
    int tb = 0, tc = 0;
    bool tune_now = false;
    if (reduced && o.tile_elems > 0) return PITN_EINVAL;   // no segmented path to tile
    if (o.tile_elems <= 0 && tune_lookup(tkey, &tb, &tc)) {
        block = tb;
        chunk = tc;
        if (reduced && chunk != 0) return PITN_EUNSUPPORTED;
    } else if (o.tile_elems <= 0 && tune_enabled()) {
        tune_now = true;
    } else if (reduced) {
        block = 128;
        chunk = 0;
    } else if (o.tile_elems <= 0) {
        // untuned default: the per-IVP path when no IVP is longer than one
        // CTA's share of the steps (about four 128-thread CTAs per SM), so
        // longest-first list scheduling keeps every CTA busy to the end
        const long long maxN = *std::max_element(hN.begin(), hN.end());
        const long long ctas = 4LL * props().multiProcessorCount;
        if (maxN * ctas <= M) {
            block = 128;
            chunk = 0;
        }
    }
    // (threads per CTA, steps per thread) of the segmented-scan path; chunk 0:
    // the per-IVP path with that many threads per CTA
    static const int kShapes[][2] = {{256, 8}, {256, 16}, {256, 32}, {256, 64}, {128, 16}, {128, 32},
                                     {512, 0}, {256, 0}, {128, 0}, {64, 0}};
    const long long chunk_g = chunk > 0 ? chunk : 32;   // buffer sizing for the segmented path
    const long long min_chunk = tune_now ? 8 : chunk_g;
    const long long max_threads = (M + min_chunk - 1) / min_chunk + 256;
    const long long grid = (M + (long long)block * chunk_g - 1) / ((long long)block * chunk_g);
    const long long grid_cap = (max_threads + 127) / 128 + 1;  // CTA count bound over all shapes
    const int JN = (system_id == PITN_LORENZ63) ? Lorenz63::JN
                   : (system_id == PITN_VDP ? VanDerPol::JN : LinearOsc::JN);
    const int W = JN + d, E = d * d + d;
    // device buffers: staged inputs | offsets | states | X1 | scratch | agg | texcl
    const bool out_dev = is_device_ptr(traj_out);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o2 = off; off += (bytes + 255) & ~(size_t)255; return o2; };
    const size_t o_par = take(sizeof(double) * P * B), o_x0 = take(sizeof(double) * d * B),
                 o_h = take(sizeof(double) * B), o_off = take(sizeof(long long) * (B + 1)),
                 o_st = take(sizeof(IvpState) * B), o_run = take(16),
                 o_it = take(sizeof(int) * B), o_stat = take(sizeof(int) * B),
                 o_res = take(sizeof(double) * B), o_offo = take(sizeof(long long) * (B + 1)),
                 o_ord = take(sizeof(long long) * B), o_work = take(16),
                 o_out = out_dev ? 0 : take(sizeof(double) * (size_t)M * d);
    char* small = (char*)workspace(off, kSlotStage);
    double* X1 = (double*)workspace(sizeof(double) * (size_t)M * d, kSlotX1);
    double* scratch = (double*)workspace(sizeof(double) * (size_t)M * W, kSlotAux);
    const size_t aggB = sizeof(double) * (size_t)std::max(grid, grid_cap) * E;
    const size_t texB = sizeof(double) * (size_t)std::max(grid * block, max_threads) * E;
    char* aux2 = (char*)workspace(aggB + texB + 512, kSlotAux2);
    unsigned* h_running = (unsigned*)pinned(64);
    if (!small || !X1 || !scratch || !aux2 || !h_running) return PITN_ENOMEM;

    auto put = [&](size_t o2, const void* src, size_t bytes) {
        const cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        return cudaMemcpyAsync(small + o2, src, bytes, kind, st) == cudaSuccess;
    };
    // the per-IVP path's queue order: longest IVP first (list scheduling of
    // unequal jobs on the CTAs), ties in index order
    std::vector<long long> hord((size_t)B);
    for (int64_t b = 0; b < B; ++b) hord[b] = b;
    std::stable_sort(hord.begin(), hord.end(), [&](long long x, long long y) { return hN[x] > hN[y]; });
    if (cudaMemcpyAsync(small + o_ord, hord.data(), sizeof(long long) * B, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return PITN_ECUDA;
    if (!put(o_par, params, sizeof(double) * P * B) || !put(o_x0, x0, sizeof(double) * d * B) ||
        cudaMemcpyAsync(small + o_h, hh.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(small + o_off, hoff.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PITN_ECUDA;

    BatchArgs a{};
    a.params = (const double*)(small + o_par);
    a.x0 = (const double*)(small + o_x0);
    a.h = (const double*)(small + o_h);
    a.off = (const long long*)(small + o_off);
    a.X0 = out_dev ? traj_out : (double*)(small + o_out);
    a.X1 = X1;
    a.scratch = scratch;
    a.agg = (double*)aux2;
    a.texcl = (double*)(aux2 + ((aggB + 255) & ~(size_t)255));
    a.st = (IvpState*)(small + o_st);
    a.running = (unsigned*)(small + o_run);
    a.work = (unsigned long long*)(small + o_work);
    a.B = B;
    a.M = M;
    a.chunk = chunk;
    a.tol = tol;
    a.guarded = (o.guard_B > 0.0 && std::isfinite(o.guard_B)) ? 1 : 0;
    {
        const double cap = a.guarded ? o.guard_B : DBL_MAX;
        std::memcpy(&a.cap_bits, &cap, sizeof(cap));
    }
    a.max_iter = max_iter;

    const bool iters_dev = is_device_ptr(iters_out);
    int* it_d = iters_dev ? iters_out : (int*)(small + o_it);
    int* stat_d = is_device_ptr(status_out) ? status_out : (int*)(small + o_stat);
    double* res_d = res_out ? (is_device_ptr(res_out) ? res_out : (double*)(small + o_res)) : nullptr;
    long long* offo_d = is_device_ptr(offsets_out) ? (long long*)offsets_out : (long long*)(small + o_offo);

    const long long* ord_d = (const long long*)(small + o_ord);
    // a shape with chunk 0 is the per-IVP path with `blk` threads per CTA
    auto run_shape = [&](int blk, long long ch, int* iters_run) -> int {
        if (reduced) {
            if (ch != 0) return PITN_EUNSUPPORTED;
            const bool f32 = o.precision == PITN_PREC_MIXED_FP32;
            switch (system_id) {
            case PITN_LORENZ63:
                return f32 ? batch_run_ivp<Lorenz63, ScanF32>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d,
                                                              iters_run)
                           : batch_run_ivp<Lorenz63, ScanFF>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d,
                                                             iters_run);
            case PITN_VDP:
                return f32 ? batch_run_ivp<VanDerPol, ScanF32>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d,
                                                               iters_run)
                           : batch_run_ivp<VanDerPol, ScanFF>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d,
                                                              iters_run);
            default:
                return f32 ? batch_run_ivp<LinearOsc, ScanF32>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d,
                                                               iters_run)
                           : batch_run_ivp<LinearOsc, ScanFF>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d,
                                                              iters_run);
            }
        }
        if (ch == 0) {
            switch (system_id) {
            case PITN_LORENZ63:
                return batch_run_ivp<Lorenz63>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d, iters_run);
            case PITN_VDP:
                return batch_run_ivp<VanDerPol>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d, iters_run);
            default:
                return batch_run_ivp<LinearOsc>(a, blk, st, ord_d, a.X0, it_d, stat_d, res_d, offo_d, iters_run);
            }
        }
        a.chunk = ch;
        const long long g = (M + (long long)blk * ch - 1) / ((long long)blk * ch);
        switch (system_id) {
        case PITN_LORENZ63:
            return batch_run<Lorenz63>(a, blk, g, st, h_running, a.X0, it_d, stat_d, res_d, offo_d, iters_run);
        case PITN_VDP:
            return batch_run<VanDerPol>(a, blk, g, st, h_running, a.X0, it_d, stat_d, res_d, offo_d, iters_run);
        default:
            return batch_run<LinearOsc>(a, blk, g, st, h_running, a.X0, it_d, stat_d, res_d, offo_d, iters_run);
        }
    };
    if (tune_now) {
        // one untimed solve on each path first: a kernel's first launch also
        // loads its code (lazy module loading), which must not count against
        // the first shape of a path
        {
            int its = 0;
            (void)run_shape(kShapes[0][0], kShapes[0][1], &its);
            (void)run_shape(128, 0, &its);
            if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
        }
        // time each shape on this batch; the whole solve's time decides
        double best = 1e300;
        for (const auto& shp : kShapes) {
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
            int its = 0;
            const int rc1 = run_shape(shp[0], shp[1], &its);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc1 != PITN_OK) continue;
            const double per = ms;
            (void)its;
            if (per < best) {
                best = per;
                block = shp[0];
                chunk = shp[1];
            }
        }
        tune_store(tkey, block, (int)chunk);
    }
    int its_final = 0;
    if (cudaMemsetAsync(a.work, 0, 16, st) != cudaSuccess) return PITN_ECUDA;   // counts of this solve only
    int rc = run_shape(block, chunk, &its_final);
    if (rc != PITN_OK) return rc;
    {
        // step counts of the solve (pitn_batch_work), counted by the kernels
        unsigned long long wk[2] = {0ull, 0ull};
        if (cudaMemcpyAsync(wk, a.work, sizeof(wk), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return PITN_ECUDA;
        g_batch_work[0].store((int64_t)wk[0]);
        g_batch_work[1].store((int64_t)wk[1]);
    }
    // host copies of the outputs given as host memory
    auto get = [&](void* dst, const void* src, size_t bytes) {
        return dst == src || cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    if (!out_dev && !get(traj_out, a.X0, sizeof(double) * (size_t)M * d)) return PITN_ECUDA;
    if (!get(iters_out, it_d, sizeof(int) * B) || !get(status_out, stat_d, sizeof(int) * B) ||
        !get(offsets_out, offo_d, sizeof(long long) * (B + 1)))
        return PITN_ECUDA;
    if (res_out && !get(res_out, res_d, sizeof(double) * B)) return PITN_ECUDA;
    // overall status
    std::vector<int> hs((size_t)B);
    if (cudaMemcpy(hs.data(), stat_d, sizeof(int) * B, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PITN_ECUDA;
    for (int64_t b = 0; b < B; ++b)
        if (hs[b] != PITN_OK) return PITN_NOT_CONVERGED;
    return PITN_OK;
}
