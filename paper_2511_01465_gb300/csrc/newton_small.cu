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
#include <cstring>

#include "common.cuh"
#include "solver.h"
#include "systems.cuh"

namespace pitn {

// Published state of one tile for the look-back.
template <int D>
struct __align__(16) TileSlot {
    unsigned flag;          // (epoch << 2) | 1 (aggregate) or | 2 (inclusive)
    unsigned pad;
    double agg[D * D + D];  // tile aggregate (P row-major, then c)
    double incl[D];         // inclusive prefix vector (state after the tile)
};

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
    long long N;
    double h, tol, cap;
    int guarded;
    int max_iter;
    long long q_init;   // 0: constant guess x0 (buffer contents ignored); N: buffer 0 holds the guess
    double params[4];
    void* tiles;
    long long num_tiles;
    unsigned long long* res_bits;  // [max_iter + 1]  ||r||_inf bits per iteration
    int* nonfinite;                // [max_iter + 1]
    unsigned long long* qenc;      // [max_iter + 1]  max of ~q (0 = no cut)
    unsigned* bar;                 // [2] grid barrier
    int* err;
    SolveRecord* rec;
};

template <int D>
__device__ __forceinline__ void mat_identity(double* P) {
#pragma unroll
    for (int i = 0; i < D * D; ++i) P[i] = (i % (D + 1) == 0) ? 1.0 : 0.0;
}

// (P, c) <- (P2, c2) o (P1, c1) = (P2 P1, P2 c1 + c2)
template <int D>
__device__ __forceinline__ void compose(const double* P2, const double* c2, const double* P1,
                                        const double* c1, double* P, double* c) {
    double tP[D * D], tc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < D; ++l) s = fma(P2[i * D + l], P1[l * D + j], s);
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

// x_k of the current iterate with the guard's lazy fill.
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

template <class Sys, int C>
__global__ void __launch_bounds__(256) newton_small_kernel(SmallArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D;
    Sys sys;
    sys.init(a.params, a.h);

    __shared__ double s_wagg[kMaxWarps][E];   // warp totals -> warp-exclusive prefixes
    __shared__ double s_tile[E];              // tile aggregate
    __shared__ double s_zin[D];               // incoming prefix vector of the tile

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const long long N = a.N;
    const long long TILE = (long long)blockDim.x * C;
    TileSlot<D>* slots = reinterpret_cast<TileSlot<D>*>(a.tiles);

    int cur = 0;
    long long q = a.q_init;       // lazy-fill index of the current iterate
    long long last_cut = N;
    int it = 0, status = PITN_NOT_CONVERGED;
    double final_res = 0.0;
    bool failed = false;

    for (;;) {
        const double* __restrict__ Xc = cur ? a.X1 : a.X0;
        double* __restrict__ Xn = cur ? a.X0 : a.X1;
        const unsigned epoch = (unsigned)it + 1u;
        unsigned long long my_res = 0ull, my_q = 0ull;
        bool my_nf = false;

        for (long long t = blockIdx.x; t < a.num_tiles; t += gridDim.x) {
            const long long base = t * TILE + (long long)threadIdx.x * C;
            // ---- 1. states, residuals, Jacobians ------------------------------
            double xs[C + 1][D];
            double r[C][D], jv[C][JN];
            load_state<D>(Xc, a.x0, base - 1, q, xs[0]);
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const long long k = base + i;
                if (k < N) {
                    load_state<D>(Xc, a.x0, k, q, xs[i + 1]);
                    sys.eval(xs[i], xs[i + 1], r[i], jv[i]);
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        unsigned long long b = (unsigned long long)__double_as_longlong(fabs(r[i][j]));
                        my_res = b > my_res ? b : my_res;
                        my_nf |= !isfinite(r[i][j]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < D; ++j) { xs[i + 1][j] = 0.0; r[i][j] = 0.0; }
#pragma unroll
                    for (int j = 0; j < JN; ++j) jv[i][j] = 0.0;
                }
            }
            // ---- 2. thread aggregate ---------------------------------------
            double P[D * D], c[D];
            mat_identity<D>(P);
#pragma unroll
            for (int j = 0; j < D; ++j) c[j] = 0.0;
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const long long k = base + i;
                if (k >= N) continue;               // identity element
                if (k == 0) {                       // a_0 = (0, -r_0), eq. 3.4
#pragma unroll
                    for (int j = 0; j < D * D; ++j) P[j] = 0.0;
#pragma unroll
                    for (int j = 0; j < D; ++j) c[j] = -r[i][j];
                } else {
                    double tP[D * D], tc[D];
                    sys.jmul(jv[i], P, tP);
                    sys.jvec(jv[i], c, tc);
#pragma unroll
                    for (int j = 0; j < D * D; ++j) P[j] = tP[j];
#pragma unroll
                    for (int j = 0; j < D; ++j) c[j] = tc[j] - r[i][j];
                }
            }
            // ---- 3. warp scan (inclusive), then lane-exclusive ----------------
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                double uP[D * D], uc[D];
#pragma unroll
                for (int j = 0; j < D * D; ++j) uP[j] = __shfl_up_sync(0xffffffffu, P[j], off);
#pragma unroll
                for (int j = 0; j < D; ++j) uc[j] = __shfl_up_sync(0xffffffffu, c[j], off);
                if (lane >= off) compose<D>(P, c, uP, uc, P, c);
            }
            double eP[D * D], ec[D];
#pragma unroll
            for (int j = 0; j < D * D; ++j) eP[j] = __shfl_up_sync(0xffffffffu, P[j], 1);
#pragma unroll
            for (int j = 0; j < D; ++j) ec[j] = __shfl_up_sync(0xffffffffu, c[j], 1);
            if (lane == 0) {
                mat_identity<D>(eP);
#pragma unroll
                for (int j = 0; j < D; ++j) ec[j] = 0.0;
            }
            if (lane == 31) {
#pragma unroll
                for (int j = 0; j < D * D; ++j) s_wagg[warp][j] = P[j];
#pragma unroll
                for (int j = 0; j < D; ++j) s_wagg[warp][D * D + j] = c[j];
            }
            __syncthreads();
            // ---- block level: warp 0 scans the warp totals --------------------
            if (warp == 0) {
                double wP[D * D], wc[D];
                if (lane < nwarps) {
#pragma unroll
                    for (int j = 0; j < D * D; ++j) wP[j] = s_wagg[lane][j];
#pragma unroll
                    for (int j = 0; j < D; ++j) wc[j] = s_wagg[lane][D * D + j];
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
                    for (int j = 0; j < D * D; ++j) s_wagg[lane][j] = xP[j];
#pragma unroll
                    for (int j = 0; j < D; ++j) s_wagg[lane][D * D + j] = xc[j];
                }
                if (lane == nwarps - 1) {
#pragma unroll
                    for (int j = 0; j < D * D; ++j) s_tile[j] = wP[j];
#pragma unroll
                    for (int j = 0; j < D; ++j) s_tile[D * D + j] = wc[j];
                }
            }
            __syncthreads();
            // ---- 4. publish + decoupled look-back (thread 0) ------------------
            if (threadIdx.x == 0) {
                TileSlot<D>* me = slots + t;
                double zin[D];
#pragma unroll
                for (int j = 0; j < D; ++j) zin[j] = 0.0;
                if (t == 0) {
                    // contains element 0, so its aggregate is already inclusive
#pragma unroll
                    for (int j = 0; j < D; ++j) me->incl[j] = s_tile[D * D + j];
                    st_release_u32(&me->flag, (epoch << 2) | 2u);
                } else {
#pragma unroll
                    for (int j = 0; j < E; ++j) me->agg[j] = s_tile[j];
                    st_release_u32(&me->flag, (epoch << 2) | 1u);
                    double Q[D * D], e[D];
                    mat_identity<D>(Q);
#pragma unroll
                    for (int j = 0; j < D; ++j) e[j] = 0.0;
                    long long jt = t - 1;
                    uint64_t t0 = 0;
                    for (;;) {
                        TileSlot<D>* s = slots + jt;
                        unsigned f = ld_acquire_u32(&s->flag);
                        if ((f >> 2) != epoch) {
                            if (t0 == 0) t0 = globaltimer_ns();
                            else if (globaltimer_ns() - t0 > kWaitLimitNs || *(volatile int*)a.err) {
                                raise_error(a.err, PITN_ETIMEOUT);
                                break;
                            }
                            continue;
                        }
                        t0 = 0;
                        if ((f & 3u) == 2u) {
                            double z[D];
#pragma unroll
                            for (int j = 0; j < D; ++j) z[j] = ldcg(&s->incl[j]);
                            apply<D>(Q, e, z, zin);
                            break;
                        }
                        double sP[D * D], sc[D];
#pragma unroll
                        for (int j = 0; j < D * D; ++j) sP[j] = ldcg(&s->agg[j]);
#pragma unroll
                        for (int j = 0; j < D; ++j) sc[j] = ldcg(&s->agg[D * D + j]);
                        compose<D>(Q, e, sP, sc, Q, e);
                        --jt;
                    }
                    double zo[D];
                    apply<D>(s_tile, s_tile + D * D, zin, zo);
#pragma unroll
                    for (int j = 0; j < D; ++j) me->incl[j] = zo[j];
                    st_release_u32(&me->flag, (epoch << 2) | 2u);
                }
#pragma unroll
                for (int j = 0; j < D; ++j) s_zin[j] = zin[j];
            }
            __syncthreads();
            // ---- 5. replay + update ------------------------------------------
            double z[D], zw[D];
            apply<D>(s_wagg[warp], s_wagg[warp] + D * D, s_zin, zw);
            apply<D>(eP, ec, zw, z);
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const long long k = base + i;
                if (k >= N) break;
                if (k == 0) {
#pragma unroll
                    for (int j = 0; j < D; ++j) z[j] = -r[i][j];
                } else {
                    double tz[D];
                    sys.jvec(jv[i], z, tz);
#pragma unroll
                    for (int j = 0; j < D; ++j) z[j] = tz[j] - r[i][j];
                }
                bool bad = false;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    bad |= !(fabs(z[j]) <= a.cap);
                    Xn[k * D + j] = xs[i + 1][j] + z[j];
                }
                if (bad) {
                    unsigned long long e = ~(unsigned long long)k;
                    my_q = e > my_q ? e : my_q;
                }
            }
            __syncthreads();  // shared scratch is reused by the next tile
        }

        // ---- iteration reductions -------------------------------------------
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, my_res, off);
            my_res = o > my_res ? o : my_res;
            o = __shfl_xor_sync(0xffffffffu, my_q, off);
            my_q = o > my_q ? o : my_q;
        }
        bool any_nf = __any_sync(0xffffffffu, my_nf);
        if (lane == 0) {
            atomicMax(a.res_bits + it, my_res);
            if (my_q) atomicMax(a.qenc + it, my_q);
            if (any_nf) atomicOr(a.nonfinite + it, 1);
        }
        if (!grid_barrier(a.bar, a.bar + 1, gridDim.x, a.err)) { failed = true; break; }

        // ---- decision (identical in every CTA) ------------------------------
        const double res = __longlong_as_double((long long)__ldcg(a.res_bits + it));
        const int nf = *(volatile int*)(a.nonfinite + it);
        const unsigned long long qe = __ldcg(a.qenc + it);
        const long long cut = qe ? (long long)(~qe) : N;
        final_res = res;
        if (nf) { status = PITN_NONFINITE; break; }
        if (res <= a.tol) { status = PITN_OK; break; }
        if (it == a.max_iter) { status = PITN_NOT_CONVERGED; break; }
        if (!a.guarded && cut < N) { status = PITN_NONFINITE; break; }
        cur ^= 1;
        q = a.guarded ? cut : N;
        last_cut = cut;
        ++it;
    }
    if (failed) return;

    // ---- write the final iterate (with its fill) to the destination ---------
    const double* Xc = cur ? a.X1 : a.X0;
    const bool same = (Xc == a.out);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
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

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------
struct SmallConfig {
    int block;
    int C;
};

template <class Sys, int C>
static cudaError_t launch_one(SmallArgs& a, int block, cudaStream_t st, int* grid_out) {
    auto kern = newton_small_kernel<Sys, C>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long cap = (long long)per_sm * pitn_host::props().multiProcessorCount;
    int grid = (int)std::min<long long>(a.num_tiles, cap);
    void* args[] = {(void*)&a};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(block), args, 0, st);
    pitn_host::count_launch();
    if (grid_out) *grid_out = grid;
    return e;
}

template <class Sys>
static cudaError_t dispatch_c(SmallArgs& a, SmallConfig cfg, cudaStream_t st) {
    switch (cfg.C) {
    case 2: return launch_one<Sys, 2>(a, cfg.block, st, nullptr);
    case 4: return launch_one<Sys, 4>(a, cfg.block, st, nullptr);
    case 8: return launch_one<Sys, 8>(a, cfg.block, st, nullptr);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pitn

namespace pitn_host {

static size_t tile_slot_bytes(int d) {
    return d == 3 ? sizeof(pitn::TileSlot<3>) : sizeof(pitn::TileSlot<2>);
}

// Default tiling: the largest block that still leaves about two tiles per SM.
void small_default_config(int d, long long N, int* block, int* C) {
    int c = (d == 3) ? 4 : 8;
    int sms = props().multiProcessorCount;
    int b = 256;
    while (b > 32 && (N + (long long)b * c - 1) / ((long long)b * c) < 2LL * sms) b >>= 1;
    *block = b;
    *C = c;
}

int small_solve_full(int system_id, const SolveIO& io, double h, int64_t N, int d, double tol,
                     int max_iter, const pitn_options& o, cudaStream_t st, SolveOutcome* out) {
    using namespace pitn;
    int block = 0, C = 0;
    small_default_config(d, N, &block, &C);
    if (o.tile_elems > 0) {
        if (o.tile_elems != 2 && o.tile_elems != 4 && o.tile_elems != 8) return PITN_EINVAL;
        C = o.tile_elems;
    }
    const long long tile = (long long)block * C;
    const long long num_tiles = (N + tile - 1) / tile;

    double* X1 = (double*)workspace((size_t)N * d * sizeof(double), kSlotX1);
    // control block: tiles | res_bits | qenc | nonfinite | bar | err | record
    size_t off_tiles = 0;
    size_t off_res = off_tiles + (size_t)num_tiles * tile_slot_bytes(d);
    size_t off_q = off_res + sizeof(unsigned long long) * (size_t)(max_iter + 1);
    size_t off_nf = off_q + sizeof(unsigned long long) * (size_t)(max_iter + 1);
    size_t off_bar = (off_nf + sizeof(int) * (size_t)(max_iter + 1) + 15) & ~(size_t)15;
    size_t off_err = off_bar + 16;
    size_t off_rec = off_err + 16;
    size_t total = off_rec + sizeof(SolveRecord);
    char* ctrl = (char*)workspace(total, kSlotCtrl);
    // host mirror: err | record | history
    size_t hbytes = 16 + sizeof(SolveRecord) + sizeof(double) * (size_t)(max_iter + 1);
    char* hbuf = (char*)pinned(hbytes);
    if (!X1 || !ctrl || !hbuf) return PITN_ENOMEM;

    SmallArgs a{};
    a.x0 = io.x0_dev;
    a.X0 = io.traj_dev;
    a.X1 = X1;
    a.out = io.traj_dev;
    a.N = N;
    a.h = h;
    a.tol = tol;
    a.guarded = (o.guard_B > 0.0 && std::isfinite(o.guard_B)) ? 1 : 0;
    a.cap = a.guarded ? o.guard_B : DBL_MAX;
    a.max_iter = max_iter;
    a.q_init = io.have_guess ? N : 0;
    for (int i = 0; i < 4; ++i) a.params[i] = io.params[i];
    a.tiles = ctrl + off_tiles;
    a.num_tiles = num_tiles;
    a.res_bits = (unsigned long long*)(ctrl + off_res);
    a.qenc = (unsigned long long*)(ctrl + off_q);
    a.nonfinite = (int*)(ctrl + off_nf);
    a.bar = (unsigned*)(ctrl + off_bar);
    a.err = (int*)(ctrl + off_err);
    a.rec = (SolveRecord*)(ctrl + off_rec);

    if (cudaMemsetAsync(ctrl, 0, total, st) != cudaSuccess) return PITN_ECUDA;
    SmallConfig cfg{block, C};
    cudaError_t e;
    switch (system_id) {
    case PITN_LORENZ63: e = dispatch_c<Lorenz63>(a, cfg, st); break;
    case PITN_VDP: e = dispatch_c<VanDerPol>(a, cfg, st); break;
    case PITN_LINEAR_OSC: e = dispatch_c<LinearOsc>(a, cfg, st); break;
    default: return PITN_EINVAL;
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

}  // namespace pitn_host
