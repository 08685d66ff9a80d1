// solver.h -- internal interfaces between the C ABI layer (api.cu) and the
// kernel families (newton_small.cu, fkpp.cu, batch.cu, adjoint.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>
#include <mutex>
#include <vector>

#include "pitn.h"

namespace pitn_host {

// Scratch slots of the per-device cache.
enum : int {
    kSlotStage = 0,  // host-staged inputs/outputs
    kSlotX1 = 1,     // second trajectory buffer
    kSlotCtrl = 2,   // tile descriptors, per-iteration reductions, barrier words
    kSlotAux = 3,    // kernel-family specific (aggregates, checkpoints)
    kSlotAux2 = 4,
    kSlots = 5
};

constexpr int64_t kMaxSteps = (int64_t)1 << 34;  // per call
constexpr int kMaxIter = 1 << 20;
constexpr int kMaxParams = 4;
constexpr int kFkppMaxD = 128;

// Limits of the in-kernel waits (pitn_debug_inject changes them for tests of
// the timeout paths): a grid barrier gives up after grid_ns nanoseconds, an
// mbarrier wait for bulk loads after load_polls polls and one for the
// tensor cores after mma_polls polls.
struct WaitLimits {
    uint64_t grid_ns = 2000000000ull;   // 2 s
    uint64_t load_polls = 1ull << 26;
    uint64_t mma_polls = 1ull << 26;
};
const WaitLimits& wait_limits();

void* workspace(size_t bytes, int slot);
void* pinned(size_t bytes);
void release_all();
void count_launch(int64_t n);
const cudaDeviceProp& props();
bool is_device_ptr(const void* p);
bool is_foreign_device_ptr(const void* p);
bool any_foreign(std::initializer_list<const void*> ptrs);
int system_dim_ok(int sys, int d);
int num_params(int sys);
int fetch_to_host(const double* src, size_t n, double* dst);
std::recursive_mutex& api_mutex();

// Optional per-kernel timing (CUDA events on the launching stream).
// timed_begin returns a token to pass to timed_end; both are no-ops while
// timing is disabled.
struct TimedToken {
    void* e0 = nullptr;
    const char* name = nullptr;
};
TimedToken timed_begin(const char* name, cudaStream_t st);
void timed_end(const TimedToken& t, cudaStream_t st);

// Inputs of one single-IVP solve, resident on the device.
struct SolveIO {
    double params[kMaxParams];  // host copy of the parameters
    const double* x0_dev;       // x0 on the device
    double* traj_dev;           // device buffer that receives the trajectory
    bool traj_is_host;          // traj_out was host memory (copy back at the end)
    bool have_guess;            // traj_dev already holds the initial guess
};

struct SolveOutcome {
    int iters = 0;
    int status = PITN_NOT_CONVERGED;
    double final_res = 0.0;
    int64_t guard_index = 0;
    std::vector<double> history;  // ||h||_inf per residual evaluation
    std::vector<long long> cuts;  // guard cut q of every Newton step computed
};

int stage_inputs(int system_id, const double* params, const double* x0, int64_t N, int d,
                 double* traj_out, const double* guess, cudaStream_t st, SolveIO* io);
int finish_outputs(const SolveIO& io, int64_t N, int d, double* traj_out, cudaStream_t st);

// Autotuner: launch shapes cached per key (workload class and size bucket),
// optionally persisted in the file named by PITN_TUNE_CACHE.
bool tune_enabled();
bool tune_lookup(const char* key, int* a, int* b);
void tune_store(const char* key, int a, int b);
int tune_bucket(long long n);  // floor(log2 n)

// Small-state systems (d = 2, 3): one persistent cooperative kernel per solve.
int small_solve_full(int system_id, const SolveIO& io, double h, int64_t N, int d, double tol,
                     int max_iter, const pitn_options& o, cudaStream_t st, SolveOutcome* out);
void small_default_config(int d, long long N, int* block, int* C);

// Fisher-KPP method-of-lines systems (d >= 3).
int fkpp_solve(const SolveIO& io, double h, int64_t N, int d, double tol, int max_iter,
               const pitn_options& o, cudaStream_t st, SolveOutcome* out);

}  // namespace pitn_host
