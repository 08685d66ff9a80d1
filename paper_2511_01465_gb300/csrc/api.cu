// api.cu -- the extern "C" boundary: argument validation, host/device
// staging, the per-device scratch cache and dispatch to the kernels.
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "solver.h"

namespace pitn_host {

namespace {
std::recursive_mutex g_mu;  // one solve at a time per process (shared scratch)
std::atomic<int64_t> g_launches{0};

struct DevCache {
    void* ptr[kSlots] = {};
    size_t bytes[kSlots] = {};
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
};
std::map<int, DevCache> g_cache;
// failure injection (pitn_debug_inject): allocations still to refuse, and
// the in-kernel wait limits
std::atomic<int64_t> g_fail_allocs{0};
WaitLimits g_waits;
std::map<int, cudaDeviceProp> g_props;

// kernel timing
std::atomic<int> g_timing{0};
struct Pending {
    cudaEvent_t e0, e1;
    std::string name;
};
std::vector<Pending> g_pending;
std::map<std::string, std::pair<double, int64_t>> g_times;
std::mutex g_tmu;
}  // namespace

TimedToken timed_begin(const char* name, cudaStream_t st) {
    TimedToken t;
    if (!g_timing.load()) return t;
    cudaEvent_t e0;
    if (cudaEventCreate(&e0) != cudaSuccess) return t;
    cudaEventRecord(e0, st);
    t.e0 = (void*)e0;
    t.name = name;
    return t;
}

void timed_end(const TimedToken& t, cudaStream_t st) {
    if (!t.e0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy((cudaEvent_t)t.e0);
        return;
    }
    cudaEventRecord(e1, st);
    std::lock_guard<std::mutex> lk(g_tmu);
    g_pending.push_back(Pending{(cudaEvent_t)t.e0, e1, t.name});
}

static void resolve_timing() {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            auto& v = g_times[p.name];
            v.first += ms;
            v.second += 1;
        }
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    g_pending.clear();
}

const WaitLimits& wait_limits() { return g_waits; }

void* workspace(size_t bytes, int slot) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    DevCache& c = g_cache[dev];
    if (bytes == 0) bytes = 256;
    if (c.bytes[slot] < bytes) {
        if (g_fail_allocs.load() > 0 && g_fail_allocs.fetch_sub(1) > 0) return nullptr;  // injected
        if (c.ptr[slot]) cudaFree(c.ptr[slot]);
        c.ptr[slot] = nullptr;
        c.bytes[slot] = 0;
        size_t want = bytes + bytes / 8;  // some headroom against regrowth
        if (cudaMalloc(&c.ptr[slot], want) != cudaSuccess) {
            cudaGetLastError();
            if (cudaMalloc(&c.ptr[slot], bytes) != cudaSuccess) {
                cudaGetLastError();
                c.ptr[slot] = nullptr;
                return nullptr;
            }
            want = bytes;
        }
        c.bytes[slot] = want;
    }
    return c.ptr[slot];
}

void* pinned(size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    DevCache& c = g_cache[dev];
    if (c.pinned_bytes < bytes) {
        if (c.pinned) cudaFreeHost(c.pinned);
        c.pinned = nullptr;
        c.pinned_bytes = 0;
        if (cudaMallocHost(&c.pinned, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        c.pinned_bytes = bytes;
    }
    return c.pinned;
}

void release_all() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    auto it = g_cache.find(dev);
    if (it == g_cache.end()) return;
    for (int s = 0; s < kSlots; ++s)
        if (it->second.ptr[s]) cudaFree(it->second.ptr[s]);
    if (it->second.pinned) cudaFreeHost(it->second.pinned);
    g_cache.erase(it);
}

void count_launch(int64_t n) { g_launches.fetch_add(n); }

const cudaDeviceProp& props() {
    int dev = 0;
    cudaGetDevice(&dev);
    auto it = g_props.find(dev);
    if (it == g_props.end()) {
        cudaDeviceProp p{};
        cudaGetDeviceProperties(&p, dev);
        it = g_props.emplace(dev, p).first;
    }
    return it->second;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device memory that belongs to a GPU other than the current one.  The
// kernels run on the current device and would load or store through such a
// pointer as a peer access (or fault), so the entry points refuse it.
// Managed memory migrates to whichever device touches it and is accepted.
bool is_foreign_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (attr.type != cudaMemoryTypeDevice) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return true;
    return attr.device != dev;
}

bool any_foreign(std::initializer_list<const void*> ptrs) {
    for (const void* p : ptrs)
        if (is_foreign_device_ptr(p)) return true;
    return false;
}

int system_dim_ok(int sys, int d) {
    switch (sys) {
    case PITN_LORENZ63: return d == 3;
    case PITN_VDP: return d == 2;
    case PITN_LINEAR_OSC: return d == 2;
    case PITN_FKPP: return d >= 3 && d <= kFkppMaxD;
    case PITN_LOGISTIC: return d == 1;
    case PITN_DAHLQUIST: return d == 1;
    case PITN_ROBERTSON: return d == 3;
    default: return 0;
    }
}

int num_params(int sys) {
    switch (sys) {
    case PITN_LORENZ63: return 3;
    case PITN_VDP: return 1;
    case PITN_LINEAR_OSC: return 2;
    case PITN_FKPP: return 1;
    case PITN_LOGISTIC: return 2;
    case PITN_DAHLQUIST: return 1;
    case PITN_ROBERTSON: return 3;
    default: return -1;
    }
}

// Copies n doubles from a host-or-device pointer to host memory.
int fetch_to_host(const double* src, size_t n, double* dst) {
    if (is_device_ptr(src)) {
        if (cudaMemcpy(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return PITN_ECUDA;
    } else {
        std::memcpy(dst, src, n * sizeof(double));
    }
    return PITN_OK;
}

std::recursive_mutex& api_mutex() { return g_mu; }

int stage_inputs(int system_id, const double* params, const double* x0, int64_t N, int d,
                 double* traj_out, const double* guess, cudaStream_t st, SolveIO* io) {
    const int P = num_params(system_id);
    for (int i = 0; i < kMaxParams; ++i) io->params[i] = 0.0;
    if (fetch_to_host(params, (size_t)P, io->params) != PITN_OK) return PITN_ECUDA;
    const size_t nd = (size_t)N * d;
    const bool traj_dev = is_device_ptr(traj_out);
    const bool x0_dev = is_device_ptr(x0);
    // stage slot: [trajectory (host case)] [x0 (host case)]
    size_t need = (traj_dev ? 0 : nd * sizeof(double)) + 64 + (size_t)d * sizeof(double);
    char* stage = (char*)workspace(need, kSlotStage);
    if (!stage) return PITN_ENOMEM;
    io->traj_is_host = !traj_dev;
    io->traj_dev = traj_dev ? traj_out : (double*)stage;
    double* x0_stage = (double*)(stage + (traj_dev ? 0 : ((nd * sizeof(double) + 63) & ~(size_t)63)));
    if (x0_dev) {
        io->x0_dev = x0;
    } else {
        if (cudaMemcpyAsync(x0_stage, x0, (size_t)d * sizeof(double), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return PITN_ECUDA;
        io->x0_dev = x0_stage;
    }
    io->have_guess = guess != nullptr;
    if (guess) {
        cudaMemcpyKind kind = is_device_ptr(guess) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (cudaMemcpyAsync(io->traj_dev, guess, nd * sizeof(double), kind, st) != cudaSuccess)
            return PITN_ECUDA;
    }
    return PITN_OK;
}

int finish_outputs(const SolveIO& io, int64_t N, int d, double* traj_out, cudaStream_t st) {
    if (!io.traj_is_host) return PITN_OK;
    if (cudaMemcpyAsync(traj_out, io.traj_dev, (size_t)N * d * sizeof(double),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PITN_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PITN_ECUDA;
    return PITN_OK;
}

}  // namespace pitn_host

using namespace pitn_host;

extern "C" {

int pitn_num_params(int system_id) { return num_params(system_id); }

const char* pitn_status_string(int code) {
    switch (code) {
    case PITN_OK: return "converged: ||h||_inf <= tol";
    case PITN_NOT_CONVERGED: return "not converged within max_iter Newton updates";
    case PITN_NONFINITE: return "non-finite residual or Newton correction";
    case PITN_EINVAL: return "invalid argument";
    case PITN_ENOMEM: return "out of memory";
    case PITN_ECUDA: return "CUDA runtime error";
    case PITN_ETIMEOUT: return "in-kernel wait timed out";
    case PITN_EUNSUPPORTED: return "unsupported request";
    default: return "unknown code";
    }
}

int pitn_release_workspace(void) {
    std::lock_guard<std::recursive_mutex> lk(api_mutex());
    release_all();
    return PITN_OK;
}

int64_t pitn_launch_count(void) { return g_launches.load(); }

int pitn_debug_inject(int what, int64_t value) {
    std::lock_guard<std::recursive_mutex> lk(api_mutex());
    switch (what) {
    case PITN_DEBUG_RESET:
        g_fail_allocs.store(0);
        g_waits = WaitLimits{};
        return PITN_OK;
    case PITN_DEBUG_FAIL_ALLOCS:
        if (value < 0) return PITN_EINVAL;
        g_fail_allocs.store(value);
        return PITN_OK;
    case PITN_DEBUG_GRID_WAIT_NS:
        g_waits.grid_ns = value > 0 ? (uint64_t)value : WaitLimits{}.grid_ns;
        return PITN_OK;
    case PITN_DEBUG_LOAD_POLLS:
        g_waits.load_polls = value >= 0 ? (uint64_t)value : WaitLimits{}.load_polls;
        return PITN_OK;
    case PITN_DEBUG_MMA_POLLS:
        g_waits.mma_polls = value >= 0 ? (uint64_t)value : WaitLimits{}.mma_polls;
        return PITN_OK;
    default:
        return PITN_EINVAL;
    }
}

int pitn_timing_enable(int on) {
    resolve_timing();
    g_timing.store(on ? 1 : 0);
    return PITN_OK;
}

int pitn_timing_reset(void) {
    resolve_timing();
    std::lock_guard<std::mutex> lk(g_tmu);
    g_times.clear();
    return PITN_OK;
}

int pitn_timing_get(const char* kernel, double* total_ms, int64_t* launches) {
    if (!kernel || !total_ms || !launches) return PITN_EINVAL;
    resolve_timing();
    std::lock_guard<std::mutex> lk(g_tmu);
    auto it = g_times.find(kernel);
    if (it == g_times.end()) {
        *total_ms = 0.0;
        *launches = 0;
    } else {
        *total_ms = it->second.first;
        *launches = it->second.second;
    }
    return PITN_OK;
}

int pitn_solve(int system_id, const double* params, const double* x0, double h, int64_t N, int d,
               double tol, int max_iter, double* traj_out) {
    return pitn_solve_ex(system_id, params, x0, h, N, d, tol, max_iter, traj_out, nullptr, nullptr);
}

int pitn_solve_ex(int system_id, const double* params, const double* x0, double h, int64_t N,
                  int d, double tol, int max_iter, double* traj_out, const pitn_options* opt,
                  pitn_result* result) {
    pitn_options o{};
    if (opt) o = *opt;
    // ---- validation (host, before any device work) ----
    if (!system_dim_ok(system_id, d)) return PITN_EINVAL;
    if (!params || !x0 || !traj_out) return PITN_EINVAL;
    if (N < 1 || N > kMaxSteps) return PITN_EINVAL;
    if (!std::isfinite(h) || !(h > 0.0)) return PITN_EINVAL;
    if (!std::isfinite(tol) || !(tol >= 0.0)) return PITN_EINVAL;
    if (max_iter < 0 || max_iter > kMaxIter) return PITN_EINVAL;
    if (std::isnan(o.guard_B)) return PITN_EINVAL;
    if (o.precision != PITN_PREC_FP64 && o.precision != PITN_PREC_MIXED_BF16 &&
        o.precision != PITN_PREC_MIXED_FP32 && o.precision != PITN_PREC_FP64_FF &&
        o.precision != PITN_PREC_MIXED_TF32)
        return PITN_EINVAL;
    if (o.precision == PITN_PREC_MIXED_TF32 && system_id != PITN_FKPP) return PITN_EINVAL;
    if (o.precision == PITN_PREC_FP64_FF &&
        !(((system_id == PITN_VDP || system_id == PITN_LINEAR_OSC || system_id == PITN_LORENZ63) &&
           o.method == PITN_STEP_EULER) ||
          (system_id == PITN_VDP && o.method == PITN_STEP_RK4) ||
          ((system_id == PITN_ROBERTSON || system_id == PITN_DAHLQUIST || system_id == PITN_VDP ||
            system_id == PITN_LOGISTIC) &&
           (o.method == PITN_STEP_BACKWARD_EULER || o.method == PITN_STEP_TRAPEZOID))))
        return PITN_EINVAL;
    if (o.precision == PITN_PREC_MIXED_BF16 && system_id != PITN_FKPP) return PITN_EINVAL;
    if (o.precision == PITN_PREC_MIXED_FP32 &&
        !(((system_id == PITN_LORENZ63 || system_id == PITN_VDP || system_id == PITN_LINEAR_OSC) &&
           o.method == PITN_STEP_EULER) ||
          (system_id == PITN_VDP && o.method == PITN_STEP_RK4) ||
          ((system_id == PITN_ROBERTSON || system_id == PITN_DAHLQUIST || system_id == PITN_VDP ||
            system_id == PITN_LOGISTIC) &&
           (o.method == PITN_STEP_BACKWARD_EULER || o.method == PITN_STEP_TRAPEZOID))))
        return PITN_EINVAL;
    if (o.tile_elems < 0) return PITN_EINVAL;
    if (o.method < PITN_STEP_EULER || o.method > PITN_STEP_TRAPEZOID) return PITN_EINVAL;
    if (any_foreign({params, x0, traj_out, o.guess})) return PITN_EINVAL;
    if (o.method == PITN_STEP_RK4 && system_id != PITN_VDP && system_id != PITN_LOGISTIC)
        return PITN_EUNSUPPORTED;
    if ((o.method == PITN_STEP_BACKWARD_EULER || o.method == PITN_STEP_TRAPEZOID) &&
        system_id != PITN_DAHLQUIST && system_id != PITN_ROBERTSON && system_id != PITN_VDP &&
        system_id != PITN_LOGISTIC)
        return PITN_EUNSUPPORTED;

    std::lock_guard<std::recursive_mutex> lk(api_mutex());
    cudaStream_t st = (cudaStream_t)o.stream;
    SolveIO io{};
    int rc = stage_inputs(system_id, params, x0, N, d, traj_out, o.guess, st, &io);
    if (rc != PITN_OK) return rc;

    SolveOutcome out{};
    if (system_id == PITN_FKPP) {
        rc = fkpp_solve(io, h, N, d, tol, max_iter, o, st, &out);
    } else {
        rc = small_solve_full(system_id, io, h, N, d, tol, max_iter, o, st, &out);
    }
    if (rc != PITN_OK) return rc;
    rc = finish_outputs(io, N, d, traj_out, st);
    if (rc != PITN_OK) return rc;
    if (o.res_history) {
        for (int k = 0; k <= out.iters && k <= max_iter; ++k) o.res_history[k] = out.history[k];
    }
    if (o.cut_history) {
        for (int k = 0; k <= max_iter; ++k)
            o.cut_history[k] = (size_t)k < out.cuts.size() ? (int64_t)out.cuts[k] : (int64_t)-1;
    }
    if (result) {
        result->iters = out.iters;
        result->status = out.status;
        result->final_res = out.final_res;
        result->guard_index = out.guard_index;
    }
    return out.status;
}

}  // extern "C"
