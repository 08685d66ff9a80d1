// shard.cu -- one shard of a time-sharded Newton solve (one long IVP split
// along time over several GPUs).  Not in the paper, which runs on one GPU;
// its Newton step is the affine recursion of eq. 3.13 solved by prefix sums
// of eq. 3.1 with the operator of eq. 3.3, and an associative scan splits
// across devices exactly as it splits across CTAs: each shard reduces its
// own elements to one aggregate, the aggregates are exchanged, and each
// shard replays its elements from the prefix of the shards before it.
//
// A shard owns the contiguous steps [s, s + n) of the trajectory.  Per Newton
// iteration the host driver (paper_2511_01465_gb300/timeshard.py) calls:
//   pass      residual r_k = x_{k+1} - phi(x_k) (eq. 3.8) of the shard's steps,
//             from the state before the shard (the halo), with ||r||_inf;
//             the elements (J_k, -r_k) (eq. 3.4; a_0 = (0, -r_0) on the shard
//             that holds step 0) folded per thread, scanned per CTA and
//             reduced in a fixed order to the shard aggregate;
//   carry     the incoming correction of shard r: the vector part of the
//             composition of the aggregates of shards 0 .. r-1 applied to 0;
//   update    replay from the incoming correction: dx_{k+1} = J_k dx_k - r_k,
//             x + dx into the next iterate, the shard's first guard cut.
// The guard's fill (reading R8) stays lazy as in the single-GPU kernels:
// local states from q_local on are read as the state before them, and a
// shard wholly beyond the global cut reads every state as its halo, which
// the driver sets to the fill state.  All pointers are device memory of the
// current device; every call blocks until its results are in device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "newton_small.cuh"

namespace pitn {

struct ShardArgs {
    const double* X;        // [n][D] current iterate of the shard
    const double* x_prev;   // [D] state before the shard's first step (halo or fill state)
    double* Xn;             // [n][D] next iterate
    long long n, C;         // steps of the shard, steps per thread
    long long q;            // local lazy fill index (states k >= q read as state q - 1)
    int holds_first;        // the shard holds step 0: its first element is (0, -r_0)
    double h;
    double params[4];
    unsigned long long cap_bits;
    double* scratch;        // [JN + D][C][threads] compact Jacobian and residual per step
    double* tpre;           // [threads][E] exclusive prefix of each thread within its CTA
    double* cagg;           // [G][E] CTA aggregates
    double* cpre;           // [G][E] exclusive prefix of each CTA within the shard
    unsigned long long* res_bits;   // ||r||_inf as bits (NaN above inf)
    unsigned long long* qenc;       // max of ~cut (0: no cut)
    const double* z_in;     // [D] incoming correction (update)
    double* agg_out;        // [E] shard aggregate (pass)
};

template <class Sys>
__global__ void __launch_bounds__(256) shard_pass_kernel(ShardArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D;
    Sys sys;
    sys.init(a.params, a.h);
    __shared__ double s_wex[kMaxWarps][E];
    __shared__ double s_tot[E];
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k0 = min(a.n, gt * a.C), k1 = min(a.n, k0 + a.C);
    auto sidx = [&](long long i, int j) -> long long { return ((long long)j * a.C + i) * nthr + gt; };
    double P[D * D], c[D];
    mat_identity<D>(P);
#pragma unroll
    for (int j = 0; j < D; ++j) c[j] = 0.0;
    unsigned long long my_res = 0ull;
    if (k0 < k1) {
        double xp[D];
        load_state<D>(a.X, a.x_prev, k0 - 1, a.q, xp);
        for (long long k = k0; k < k1; ++k) {
            double x[D], r[D], jv[JN];
            load_state<D>(a.X, a.x_prev, k, a.q, x);
            sys.eval(xp, x, r, jv);
#pragma unroll
            for (int j = 0; j < JN; ++j) a.scratch[sidx(k - k0, j)] = jv[j];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                a.scratch[sidx(k - k0, JN + j)] = r[j];
                const unsigned long long b = abs_bits(r[j]);
                my_res = b > my_res ? b : my_res;
            }
            if (a.holds_first && k == 0) {   // a_0 = (0, -r_0), eq. 3.4
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
        }
    }
    double eP[D * D], ec[D];
    block_scan<D>(P, c, eP, ec, s_wex, s_tot);
    {
        // exclusive prefix of this thread: the warps before it, then the lanes before it
        double tP[D * D], tc[D];
        compose<D>(eP, ec, s_wex[threadIdx.x >> 5], s_wex[threadIdx.x >> 5] + D * D, tP, tc);
#pragma unroll
        for (int j = 0; j < D * D; ++j) a.tpre[gt * E + j] = tP[j];
#pragma unroll
        for (int j = 0; j < D; ++j) a.tpre[gt * E + D * D + j] = tc[j];
    }
    if (threadIdx.x < E) a.cagg[(size_t)blockIdx.x * E + threadIdx.x] = s_tot[threadIdx.x];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, my_res, off);
        my_res = o > my_res ? o : my_res;
    }
    if ((threadIdx.x & 31) == 0 && my_res) atomicMax(a.res_bits, my_res);
}

// One thread: the CTA aggregates composed in order into the shard aggregate,
// each CTA's exclusive prefix on the way.
template <int D>
__global__ void shard_reduce_kernel(ShardArgs a, int G) {
    constexpr int E = D * D + D;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double P[D * D], c[D];
    mat_identity<D>(P);
#pragma unroll
    for (int j = 0; j < D; ++j) c[j] = 0.0;
    for (int b = 0; b < G; ++b) {
#pragma unroll
        for (int j = 0; j < D * D; ++j) a.cpre[(size_t)b * E + j] = P[j];
#pragma unroll
        for (int j = 0; j < D; ++j) a.cpre[(size_t)b * E + D * D + j] = c[j];
        compose<D>(a.cagg + (size_t)b * E, a.cagg + (size_t)b * E + D * D, P, c, P, c);
    }
#pragma unroll
    for (int j = 0; j < D * D; ++j) a.agg_out[j] = P[j];
#pragma unroll
    for (int j = 0; j < D; ++j) a.agg_out[D * D + j] = c[j];
}

// One thread: the incoming correction of shard r from the gathered shard
// aggregates [R][E], composed in shard order from the zero correction.
template <int D>
__global__ void shard_carry_kernel(const double* __restrict__ aggs, long long r, double* __restrict__ z_out) {
    constexpr int E = D * D + D;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double z[D], t[D];
#pragma unroll
    for (int j = 0; j < D; ++j) z[j] = 0.0;
    for (long long i = 0; i < r; ++i) {
        apply<D>(aggs + i * E, aggs + i * E + D * D, z, t);
#pragma unroll
        for (int j = 0; j < D; ++j) z[j] = t[j];
    }
#pragma unroll
    for (int j = 0; j < D; ++j) z_out[j] = z[j];
}

template <class Sys>
__global__ void __launch_bounds__(256) shard_update_kernel(ShardArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D;
    Sys sys;
    sys.init(a.params, a.h);
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k0 = min(a.n, gt * a.C), k1 = min(a.n, k0 + a.C);
    auto sidx = [&](long long i, int j) -> long long { return ((long long)j * a.C + i) * nthr + gt; };
    double zin[D], zc[D], z[D];
#pragma unroll
    for (int j = 0; j < D; ++j) zin[j] = a.z_in[j];
    apply<D>(a.cpre + (size_t)blockIdx.x * E, a.cpre + (size_t)blockIdx.x * E + D * D, zin, zc);
    apply<D>(a.tpre + gt * E, a.tpre + gt * E + D * D, zc, z);
    for (long long k = k0; k < k1; ++k) {
        double jv[JN], r[D], x[D];
#pragma unroll
        for (int j = 0; j < JN; ++j) jv[j] = a.scratch[sidx(k - k0, j)];
#pragma unroll
        for (int j = 0; j < D; ++j) r[j] = a.scratch[sidx(k - k0, JN + j)];
        load_state<D>(a.X, a.x_prev, k, a.q, x);
        if (a.holds_first && k == 0) {
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
            a.Xn[k * D + j] = x[j] + z[j];
            const unsigned long long b = abs_bits(z[j]);
            zb = b > zb ? b : zb;
        }
        if (zb > a.cap_bits) {   // first correction beyond the bound (or not finite): stop here
            atomicMax(a.qenc, ~(unsigned long long)k);
            break;
        }
    }
}

template <int D>
__global__ void shard_finalize_kernel(const double* __restrict__ X, const double* __restrict__ x_prev,
                                      long long n, long long q, double* __restrict__ out) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double v[D];
        load_state<D>(X, x_prev, k, q, v);
#pragma unroll
        for (int j = 0; j < D; ++j) out[k * D + j] = v[j];
    }
}

}  // namespace pitn

// ---------------------------------------------------------------------------
// Host side: the plan and the C ABI.
// ---------------------------------------------------------------------------
struct pitn_shard {
    int sys, d, E, JN;
    long long n, C, nthr;
    int grid, block;
    pitn::ShardArgs a;
    double* buf;                 // one allocation: scratch | tpre | cagg | cpre | control
    cudaStream_t st;
    bool passed;                 // a pass has run since the last update
    cudaError_t (*pass)(const pitn::ShardArgs&, int, int, cudaStream_t);
    cudaError_t (*update)(const pitn::ShardArgs&, int, int, cudaStream_t);
};

namespace {

template <class Sys>
cudaError_t launch_pass(const pitn::ShardArgs& a, int grid, int block, cudaStream_t st) {
    pitn::shard_pass_kernel<Sys><<<grid, block, 0, st>>>(a);
    pitn::shard_reduce_kernel<Sys::D><<<1, 32, 0, st>>>(a, grid);
    pitn_host::count_launch(2);
    return cudaGetLastError();
}

template <class Sys>
cudaError_t launch_update(const pitn::ShardArgs& a, int grid, int block, cudaStream_t st) {
    pitn::shard_update_kernel<Sys><<<grid, block, 0, st>>>(a);
    pitn_host::count_launch(1);
    return cudaGetLastError();
}

bool all_device(std::initializer_list<const void*> ptrs) {
    for (const void* p : ptrs)
        if (!p || !pitn_host::is_device_ptr(p) || pitn_host::is_foreign_device_ptr(p)) return false;
    return true;
}

}  // namespace

extern "C" {

int pitn_shard_create(int system_id, const double* params, double h, int64_t n, int d, double guard_B,
                      void* stream, pitn_shard** out) {
    using namespace pitn;
    using namespace pitn_host;
    if (!out) return PITN_EINVAL;
    *out = nullptr;
    if (system_id != PITN_LORENZ63 && system_id != PITN_VDP && system_id != PITN_LINEAR_OSC) return PITN_EINVAL;
    if (!system_dim_ok(system_id, d) || !params || n < 1 || n > kMaxSteps) return PITN_EINVAL;
    if (!std::isfinite(h) || !(h > 0.0) || std::isnan(guard_B)) return PITN_EINVAL;
    if (any_foreign({params})) return PITN_EINVAL;
    pitn_shard* s = new (std::nothrow) pitn_shard{};
    if (!s) return PITN_ENOMEM;
    s->sys = system_id;
    s->d = d;
    s->E = d * d + d;
    s->st = (cudaStream_t)stream;
    s->n = n;
    switch (system_id) {
    case PITN_LORENZ63:
        s->JN = Lorenz63::JN; s->pass = &launch_pass<Lorenz63>; s->update = &launch_update<Lorenz63>; break;
    case PITN_VDP:
        s->JN = VanDerPol::JN; s->pass = &launch_pass<VanDerPol>; s->update = &launch_update<VanDerPol>; break;
    default:
        s->JN = LinearOsc::JN; s->pass = &launch_pass<LinearOsc>; s->update = &launch_update<LinearOsc>; break;
    }
    // about 8 steps per thread, 256-thread CTAs (no grid-wide wait: any grid)
    s->block = 256;
    const long long threads = std::max<long long>(1LL, ((long long)n + 7) / 8);
    s->grid = (int)std::min<long long>((threads + s->block - 1) / s->block, 1LL << 20);
    s->nthr = (long long)s->grid * s->block;
    s->C = (n + s->nthr - 1) / s->nthr;
    const size_t n_scr = (size_t)(s->JN + d) * s->C * s->nthr;
    const size_t n_tpre = (size_t)s->nthr * s->E;
    const size_t n_cagg = (size_t)s->grid * s->E;
    const size_t total = n_scr + n_tpre + 2 * n_cagg + 4;
    if (cudaMalloc(&s->buf, total * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return PITN_ENOMEM;
    }
    ShardArgs& a = s->a;
    a.n = n;
    a.C = s->C;
    a.h = h;
    const int P = num_params(system_id);
    double hp[4] = {0, 0, 0, 0};
    if (fetch_to_host(params, (size_t)P, hp) != PITN_OK) {
        cudaFree(s->buf);
        delete s;
        return PITN_ECUDA;
    }
    for (int i = 0; i < 4; ++i) a.params[i] = hp[i];
    const bool guarded = guard_B > 0.0 && std::isfinite(guard_B);
    const double cap = guarded ? guard_B : DBL_MAX;
    std::memcpy(&a.cap_bits, &cap, sizeof(cap));
    a.scratch = s->buf;
    a.tpre = a.scratch + n_scr;
    a.cagg = a.tpre + n_tpre;
    a.cpre = a.cagg + n_cagg;
    a.res_bits = reinterpret_cast<unsigned long long*>(a.cpre + n_cagg);
    a.qenc = a.res_bits + 1;
    *out = s;
    return PITN_OK;
}

int pitn_shard_pass(pitn_shard* s, const double* x_prev, int holds_first, const double* X, int64_t q_local,
                    double* agg_out, int64_t* res_bits_out) {
    if (!s || q_local < 0 || q_local > s->n) return PITN_EINVAL;
    if (!all_device({x_prev, X, agg_out, res_bits_out})) return PITN_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(pitn_host::api_mutex());
    pitn::ShardArgs& a = s->a;
    a.X = X;
    a.x_prev = x_prev;
    a.q = q_local;
    a.holds_first = holds_first ? 1 : 0;
    a.agg_out = agg_out;
    if (cudaMemsetAsync(a.res_bits, 0, 2 * sizeof(unsigned long long), s->st) != cudaSuccess) return PITN_ECUDA;
    if (s->pass(a, s->grid, s->block, s->st) != cudaSuccess) return PITN_ECUDA;
    if (cudaMemcpyAsync(res_bits_out, a.res_bits, sizeof(int64_t), cudaMemcpyDeviceToDevice, s->st) != cudaSuccess)
        return PITN_ECUDA;
    if (cudaStreamSynchronize(s->st) != cudaSuccess) return PITN_ECUDA;
    s->passed = true;
    return PITN_OK;
}

int pitn_shard_carry(pitn_shard* s, int64_t r, const double* aggs, double* z_out) {
    if (!s || r < 0) return PITN_EINVAL;
    if (!all_device({z_out}) || (r > 0 && !all_device({aggs}))) return PITN_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(pitn_host::api_mutex());
    switch (s->d) {
    case 2: pitn::shard_carry_kernel<2><<<1, 32, 0, s->st>>>(aggs, r, z_out); break;
    default: pitn::shard_carry_kernel<3><<<1, 32, 0, s->st>>>(aggs, r, z_out); break;
    }
    pitn_host::count_launch(1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s->st) != cudaSuccess) return PITN_ECUDA;
    return PITN_OK;
}

int pitn_shard_update(pitn_shard* s, const double* z_in, double* Xn, int64_t* cut_out) {
    if (!s || !s->passed) return PITN_EINVAL;
    if (!all_device({z_in, Xn, cut_out})) return PITN_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(pitn_host::api_mutex());
    pitn::ShardArgs& a = s->a;
    a.z_in = z_in;
    a.Xn = Xn;
    if (cudaMemsetAsync(a.qenc, 0, sizeof(unsigned long long), s->st) != cudaSuccess) return PITN_ECUDA;
    if (s->update(a, s->grid, s->block, s->st) != cudaSuccess) return PITN_ECUDA;
    unsigned long long qe = 0;
    if (cudaMemcpyAsync(&qe, a.qenc, sizeof(qe), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess)
        return PITN_ECUDA;
    const int64_t cut = qe ? (int64_t)~qe : (int64_t)s->n;
    if (cudaMemcpyAsync(cut_out, &cut, sizeof(cut), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess)
        return PITN_ECUDA;
    s->passed = false;
    return PITN_OK;
}

int pitn_shard_finalize(pitn_shard* s, const double* X, const double* x_prev, int64_t q_local, double* out) {
    if (!s || q_local < 0 || q_local > s->n) return PITN_EINVAL;
    if (!all_device({X, x_prev, out})) return PITN_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(pitn_host::api_mutex());
    switch (s->d) {
    case 2: pitn::shard_finalize_kernel<2><<<256, 256, 0, s->st>>>(X, x_prev, s->n, q_local, out); break;
    default: pitn::shard_finalize_kernel<3><<<256, 256, 0, s->st>>>(X, x_prev, s->n, q_local, out); break;
    }
    pitn_host::count_launch(1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s->st) != cudaSuccess) return PITN_ECUDA;
    return PITN_OK;
}

int pitn_shard_destroy(pitn_shard* s) {
    if (!s) return PITN_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(pitn_host::api_mutex());
    cudaStreamSynchronize(s->st);
    cudaFree(s->buf);
    delete s;
    return PITN_OK;
}

}  // extern "C"
