// adjoint.cu -- gradients of a loss of converged trajectories with respect to
// x0 and the ODE parameters (pitn_backward).
//
// For x_{n+1} = phi(x_n) and a loss L(x_1..x_N) with G_n = dL/dx_n, the
// adjoint states satisfy the reverse-time affine recursion
//     lambda_N = G_N,   lambda_n = J_n^T lambda_{n+1} + G_n,   J_n = dphi/dx(x_n),
// the transposed form of the Newton-step recursion of eq. 3.13.  It is
// solved as an affine scan in reversed step order over the elements
// (J_n^T, G_n); the element of the last step of every IVP has matrix 0, so
// the concatenated IVPs segment themselves exactly as in the forward batch.
// Then
//     dL/dx0 = J_0^T lambda_1,   dL/dp = sum_{n=0}^{N-1} (dphi/dp(x_n))^T lambda_{n+1}.
// Kernels: A (reverse fold + block scan: one aggregate per CTA span of
// ckpt_every steps, the scan's checkpoints, and each thread's exclusive
// prefix), C (incoming prefix from the checkpoints back to the IVP's last
// step, replay, lambda per step), R (one CTA per IVP: the parameter and x0
// gradients summed in a fixed order, so results are deterministic).  The
// Jacobians are recomputed from the trajectory, never stored.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "solver.h"
#include "systems.cuh"

namespace pitn {

struct AdjArgs {
    const double* params;  // [B][P]
    const double* x0;      // [B][D]
    const double* h;       // [B]
    const long long* off;  // [B+1]
    const double* traj;    // [M][D]
    const double* gtraj;   // [M][D] or null
    const double* gN;      // [B][D] or null
    double* lam;           // [M][D]
    double* agg;           // [G][E]
    double* texcl;         // [threads][E]
    long long B, M, chunk;
};

__device__ __forceinline__ long long a_seg(const long long* __restrict__ off, long long B, long long k) {
    long long lo = 0, hi = B;
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (off[mid] <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int D>
__device__ __forceinline__ void a_identity(double* P) {
#pragma unroll
    for (int i = 0; i < D * D; ++i) P[i] = (i % (D + 1) == 0) ? 1.0 : 0.0;
}
template <int D>
__device__ __forceinline__ void a_compose(const double* P2, const double* c2, const double* P1,
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
__device__ __forceinline__ void a_apply(const double* P, const double* c, const double* v, double* o) {
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

// G_n for the step at global index k of IVP b (last step adds grad_xN).
template <int D>
__device__ __forceinline__ void a_g(const AdjArgs& a, long long b, long long k, bool last, double* g) {
#pragma unroll
    for (int i = 0; i < D; ++i) g[i] = a.gtraj ? a.gtraj[k * D + i] : 0.0;
    if (last && a.gN) {
#pragma unroll
        for (int i = 0; i < D; ++i) g[i] += a.gN[b * D + i];
    }
}

// ---- A: reverse fold + block scan ------------------------------------------
template <class Sys>
__global__ void __launch_bounds__(256) adj_fold_kernel(AdjArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D;
    __shared__ double s_w[8][E];
    __shared__ double s_tot[E];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long v0 = gt * a.chunk, v1 = min(a.M, v0 + a.chunk);
    double P[D * D], c[D];
    a_identity<D>(P);
#pragma unroll
    for (int i = 0; i < D; ++i) c[i] = 0.0;
    long long b = -1;
    Sys sys;
    for (long long v = v0; v < v1; ++v) {
        const long long k = a.M - 1 - v;
        if (b < 0 || k < a.off[b]) {
            b = (b < 0) ? a_seg(a.off, a.B, k) : b - 1;
            while (a.off[b] > k) --b;
            sys.init(a.params + b * Sys::P, a.h[b]);
        }
        const bool last = (k == a.off[b + 1] - 1);
        double g[D];
        a_g<D>(a, b, k, last, g);
        if (last) {
#pragma unroll
            for (int i = 0; i < D * D; ++i) P[i] = 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i) c[i] = g[i];
        } else {
            double jv[JN], J[D * D], JT[D * D];
            sys.jac(a.traj + k * D, jv);
            sys.jfull(jv, J);
#pragma unroll
            for (int r = 0; r < D; ++r)
#pragma unroll
                for (int q = 0; q < D; ++q) JT[r * D + q] = J[q * D + r];
            a_compose<D>(JT, g, P, c, P, c);
        }
    }
    // block scan (same fixed order as the forward kernels)
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        double uP[D * D], uc[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) uP[i] = __shfl_up_sync(0xffffffffu, P[i], off);
#pragma unroll
        for (int i = 0; i < D; ++i) uc[i] = __shfl_up_sync(0xffffffffu, c[i], off);
        if (lane >= off) a_compose<D>(P, c, uP, uc, P, c);
    }
    double eP[D * D], ec[D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) eP[i] = __shfl_up_sync(0xffffffffu, P[i], 1);
#pragma unroll
    for (int i = 0; i < D; ++i) ec[i] = __shfl_up_sync(0xffffffffu, c[i], 1);
    if (lane == 0) {
        a_identity<D>(eP);
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
            a_identity<D>(wP);
#pragma unroll
            for (int i = 0; i < D; ++i) wc[i] = 0.0;
        }
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) {
            double uP[D * D], uc[D];
#pragma unroll
            for (int i = 0; i < D * D; ++i) uP[i] = __shfl_up_sync(0xffffffffu, wP[i], off);
#pragma unroll
            for (int i = 0; i < D; ++i) uc[i] = __shfl_up_sync(0xffffffffu, wc[i], off);
            if (lane >= off) a_compose<D>(wP, wc, uP, uc, wP, wc);
        }
        double xP[D * D], xc[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) xP[i] = __shfl_up_sync(0xffffffffu, wP[i], 1);
#pragma unroll
        for (int i = 0; i < D; ++i) xc[i] = __shfl_up_sync(0xffffffffu, wc[i], 1);
        __syncwarp();
        if (lane < nwarps) {
            if (lane == 0) {
                a_identity<D>(xP);
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
    double tP[D * D], tc[D];
    a_compose<D>(eP, ec, s_w[warp], s_w[warp] + D * D, tP, tc);
    double* te = a.texcl + (size_t)gt * E;
#pragma unroll
    for (int i = 0; i < D * D; ++i) te[i] = tP[i];
#pragma unroll
    for (int i = 0; i < D; ++i) te[D * D + i] = tc[i];
    if (threadIdx.x < E) a.agg[(size_t)blockIdx.x * E + threadIdx.x] = s_tot[threadIdx.x];
}

// ---- C: replay, lambda per step ----------------------------------------------
template <class Sys>
__global__ void __launch_bounds__(256) adj_replay_kernel(AdjArgs a) {
    constexpr int D = Sys::D, JN = Sys::JN, E = D * D + D;
    __shared__ double s_zin[D];
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long v0 = gt * a.chunk, v1 = min(a.M, v0 + a.chunk);
    const long long span = (long long)blockDim.x * a.chunk;
    if (threadIdx.x == 0) {
        double z[D];
#pragma unroll
        for (int i = 0; i < D; ++i) z[i] = 0.0;
        const long long vf = (long long)blockIdx.x * span;
        if (vf < a.M && blockIdx.x > 0) {
            const long long kf = a.M - 1 - vf;
            const long long b0 = a_seg(a.off, a.B, kf);
            const long long vhead = a.M - a.off[b0 + 1];  // virtual index of the IVP's last step
            if (vhead < vf) {
                for (long long cc = vhead / span; cc < blockIdx.x; ++cc) {
                    const double* g = a.agg + (size_t)cc * E;
                    double t[D];
                    a_apply<D>(g, g + D * D, z, t);
#pragma unroll
                    for (int i = 0; i < D; ++i) z[i] = t[i];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) s_zin[i] = z[i];
    }
    __syncthreads();
    if (v0 >= v1) return;
    double z[D];
    {
        const double* te = a.texcl + (size_t)gt * E;
        double tP[D * D], tc[D], zi[D];
#pragma unroll
        for (int i = 0; i < D * D; ++i) tP[i] = te[i];
#pragma unroll
        for (int i = 0; i < D; ++i) { tc[i] = te[D * D + i]; zi[i] = s_zin[i]; }
        a_apply<D>(tP, tc, zi, z);
    }
    long long b = -1;
    Sys sys;
    for (long long v = v0; v < v1; ++v) {
        const long long k = a.M - 1 - v;
        if (b < 0 || k < a.off[b]) {
            b = (b < 0) ? a_seg(a.off, a.B, k) : b - 1;
            while (a.off[b] > k) --b;
            sys.init(a.params + b * Sys::P, a.h[b]);
        }
        const bool last = (k == a.off[b + 1] - 1);
        double g[D];
        a_g<D>(a, b, k, last, g);
        if (last) {
#pragma unroll
            for (int i = 0; i < D; ++i) z[i] = g[i];
        } else {
            double jv[JN], t[D];
            sys.jac(a.traj + k * D, jv);
            sys.jtvec(jv, z, t);
#pragma unroll
            for (int i = 0; i < D; ++i) z[i] = t[i] + g[i];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) a.lam[k * D + i] = z[i];
    }
}

// ---- R: per-IVP gradients (fixed summation order) ---------------------------
template <class Sys>
__global__ void __launch_bounds__(256) adj_reduce_kernel(AdjArgs a, double* gx0, double* gp) {
    constexpr int D = Sys::D, JN = Sys::JN, P = Sys::P;
    __shared__ double s_red[256][P];
    const long long b = blockIdx.x;
    const long long base = a.off[b], n = a.off[b + 1] - base;
    Sys sys;
    sys.init(a.params + b * P, a.h[b]);
    double acc[P];
#pragma unroll
    for (int i = 0; i < P; ++i) acc[i] = 0.0;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
        // term (dphi/dp(x_j))^T lambda_{j+1}; x_j is x0 for j = 0
        const double* xj = (j == 0) ? a.x0 + b * D : a.traj + (base + j - 1) * D;
        sys.vjp_param(xj, a.lam + (base + j) * D, acc);
    }
#pragma unroll
    for (int i = 0; i < P; ++i) s_red[threadIdx.x][i] = acc[i];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int i = 0; i < P; ++i) s_red[threadIdx.x][i] += s_red[threadIdx.x + w][i];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < P; ++i) gp[b * P + i] = s_red[0][i];
        double jv[JN], t[D];
        sys.jac(a.x0 + b * D, jv);
        sys.jtvec(jv, a.lam + base * D, t);
#pragma unroll
        for (int i = 0; i < D; ++i) gx0[b * D + i] = t[i];
    }
}

}  // namespace pitn

namespace pitn_host {
using namespace pitn;
namespace {

template <class Sys>
int adj_run(AdjArgs& a, int block, long long grid, cudaStream_t st, double* gx0, double* gp) {
    auto tok = timed_begin("adjoint", st);
    adj_fold_kernel<Sys><<<(unsigned)grid, block, 0, st>>>(a);
    adj_replay_kernel<Sys><<<(unsigned)grid, block, 0, st>>>(a);
    adj_reduce_kernel<Sys><<<(unsigned)a.B, 256, 0, st>>>(a, gx0, gp);
    timed_end(tok, st);
    count_launch(3);
    if (cudaGetLastError() != cudaSuccess) return PITN_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? PITN_OK : PITN_ECUDA;
}

}  // namespace
}  // namespace pitn_host

using namespace pitn_host;

extern "C" int pitn_backward(int system_id, int64_t B, const double* params, const double* x0,
                             const double* h, const int64_t* N, int d, const double* traj,
                             const double* grad_traj, const double* grad_xN, int ckpt_every,
                             double* grad_x0_out, double* grad_params_out, const pitn_options* opt) {
    pitn_options o{};
    if (opt) o = *opt;
    if ((system_id != PITN_LORENZ63 && system_id != PITN_VDP && system_id != PITN_LINEAR_OSC) ||
        !system_dim_ok(system_id, d))
        return PITN_EINVAL;
    if (B < 1 || !params || !x0 || !h || !N || !traj || !grad_x0_out || !grad_params_out) return PITN_EINVAL;
    if (ckpt_every < 0) return PITN_EINVAL;
    if (any_foreign({params, x0, h, N, traj, grad_traj, grad_xN, grad_x0_out, grad_params_out}))
        return PITN_EINVAL;
    if (o.method != PITN_STEP_EULER) return PITN_EUNSUPPORTED;
    const int P = num_params(system_id);
    std::lock_guard<std::recursive_mutex> lk(api_mutex());
    cudaStream_t st = (cudaStream_t)o.stream;
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
        if (hN[b] < 1 || !std::isfinite(hh[b]) || !(hh[b] > 0.0)) return PITN_EINVAL;
        hoff[b + 1] = hoff[b] + hN[b];
        if (hoff[b + 1] > kMaxSteps) return PITN_EINVAL;
    }
    const long long M = hoff[B];
    const int block = 256;
    const int ck = ckpt_every > 0 ? ckpt_every : 1024;
    const long long chunk = std::max(1, ck / block);
    const long long grid = (M + (long long)block * chunk - 1) / ((long long)block * chunk);
    const int E = d * d + d;

    // device copies of the inputs given as host memory, outputs, lambda, checkpoints
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o2 = off; off += (bytes + 255) & ~(size_t)255; return o2; };
    const size_t o_par = take(sizeof(double) * P * B), o_x0 = take(sizeof(double) * d * B),
                 o_h = take(sizeof(double) * B), o_off = take(sizeof(long long) * (B + 1)),
                 o_gN = take(sizeof(double) * d * B), o_gx0 = take(sizeof(double) * d * B),
                 o_gp = take(sizeof(double) * P * B), o_agg = take(sizeof(double) * grid * E),
                 o_tr = is_device_ptr(traj) ? 0 : take(sizeof(double) * (size_t)M * d),
                 o_gt = (grad_traj && !is_device_ptr(grad_traj)) ? take(sizeof(double) * (size_t)M * d) : 0;
    char* small = (char*)workspace(off, kSlotStage);
    double* lam = (double*)workspace(sizeof(double) * (size_t)M * d, kSlotX1);
    double* texcl = (double*)workspace(sizeof(double) * (size_t)grid * block * E, kSlotAux);
    if (!small || !lam || !texcl) return PITN_ENOMEM;
    auto put = [&](size_t o2, const void* src, size_t bytes) -> const double* {
        if (is_device_ptr(src)) return (const double*)src;
        if (cudaMemcpyAsync(small + o2, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
        return (const double*)(small + o2);
    };
    AdjArgs a{};
    a.params = put(o_par, params, sizeof(double) * P * B);
    a.x0 = put(o_x0, x0, sizeof(double) * d * B);
    if (cudaMemcpyAsync(small + o_h, hh.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(small + o_off, hoff.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PITN_ECUDA;
    a.h = (const double*)(small + o_h);
    a.off = (const long long*)(small + o_off);
    a.traj = put(o_tr, traj, sizeof(double) * (size_t)M * d);
    a.gtraj = grad_traj ? put(o_gt, grad_traj, sizeof(double) * (size_t)M * d) : nullptr;
    a.gN = grad_xN ? put(o_gN, grad_xN, sizeof(double) * d * B) : nullptr;
    if (!a.params || !a.x0 || !a.traj || (grad_traj && !a.gtraj) || (grad_xN && !a.gN)) return PITN_ECUDA;
    a.lam = lam;
    a.agg = (double*)(small + o_agg);
    a.texcl = texcl;
    a.B = B;
    a.M = M;
    a.chunk = chunk;
    const bool gx_dev = is_device_ptr(grad_x0_out), gp_dev = is_device_ptr(grad_params_out);
    double* gx0 = gx_dev ? grad_x0_out : (double*)(small + o_gx0);
    double* gp = gp_dev ? grad_params_out : (double*)(small + o_gp);
    int rc;
    switch (system_id) {
    case PITN_LORENZ63: rc = adj_run<Lorenz63>(a, block, grid, st, gx0, gp); break;
    case PITN_VDP: rc = adj_run<VanDerPol>(a, block, grid, st, gx0, gp); break;
    default: rc = adj_run<LinearOsc>(a, block, grid, st, gx0, gp); break;
    }
    if (rc != PITN_OK) return rc;
    if (!gx_dev && cudaMemcpy(grad_x0_out, gx0, sizeof(double) * d * B, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PITN_ECUDA;
    if (!gp_dev && cudaMemcpy(grad_params_out, gp, sizeof(double) * P * B, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PITN_ECUDA;
    return PITN_OK;
}
