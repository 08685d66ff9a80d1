// compose_tc.cuh -- dense delta-form compose of two 128x128 affine elements
// on the 5th-generation tensor cores (tcgen05, TMEM accumulator).
//
//   (I + S2, b2) o (I + S1, b1) = (I + S, b),
//   S = S2 + S1 + S2 S1,   b = b2 + b1 + S2 b1                       (eq. 3.3)
//
// Both FP32 inputs arrive in shared memory by bulk copies (TMA, completion
// counted on one mbarrier per input, so that S2's conversion starts while S1
// is still in flight); S2 S1 is then one M = N = K = 128 product: BF16
// operands converted into the canonical K-major core-matrix layout (8 rows x
// 16 bytes per core matrix, no swizzle), eight tcgen05.mma (K = 16 each)
// issued by one thread into a 128-lane x 128-column FP32 accumulator in TMEM,
// completion signalled through another mbarrier, and read back with
// tcgen05.ld: TMEM lane m is row m of the product, so thread m of the CTA
// owns row m in the epilogue, which adds S2 + S1 (FP32, summed in shared
// memory while the product runs) and stores column-major (coalesced across
// the warp).  The vector part uses the same BF16 rows of S2 with FP32
// accumulation, also while the product runs.
// Matrices are column-major FP32 (S[col][row]), 128 x 128.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace pitn {
namespace tc {

constexpr int kDim = 128;
constexpr uint32_t kCoreBytes = 128;             // 8 rows x 16 bytes
constexpr uint32_t kGroupBytes = 16 * kCoreBytes;  // one 8-row group spans K = 128 (16 cores)
constexpr uint32_t kTileBytes = 16 * kGroupBytes;  // 128 rows
constexpr uint64_t kSpinLimit = 1ull << 26;       // default bound of an mbarrier wait (polls)

// Outcome of one compose.
enum : int {
    kTcOk = 0,        // done
    kTcTimedOut = 1,  // a wait gave up; nothing is in flight any more (TMEM may be freed)
    kTcStuck = 2      // a wait gave up and a copy or the product may still be in flight:
                      // the CTA must not free its TMEM or reuse its shared memory
};

// byte offset of element (row, k) in the K-major core-matrix layout
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)((row >> 3) * kGroupBytes + (k >> 3) * kCoreBytes + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading byte offset (next
// core matrix along K), stride byte offset (next 8-row group), version 1,
// no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kCoreBytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kGroupBytes >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major,
// N = 128, M = 128
__device__ __forceinline__ uint32_t make_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kDim >> 3) << 17) |
           ((uint32_t)(kDim >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_addr(dst_smem)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_addr(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}
// bounded wait for the phase with the given parity (at most `polls` polls);
// false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint64_t polls = kSpinLimit) {
    const uint32_t a = smem_addr(mbar);
    for (uint64_t i = 0; i < polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
}
// bulk copy global -> shared (16 B-aligned addresses, size a multiple of 16),
// completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(sdst)), "l"(gsrc), "r"(bytes), "r"(smem_addr(mbar)) : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared memory of one compose: the FP32 inputs, the BF16 A and B tiles, the
// mbarriers (loads, MMA) and the TMEM address.
struct __align__(1024) ComposeSmem {
    uint8_t A[kTileBytes];     // S2 (rows m, K-major)
    uint8_t B[kTileBytes];     // S1 (rows n = columns of S1, K-major)
    float S2f[kDim * kDim];    // S2 column-major, as loaded
    float S1f[kDim * kDim];    // S1 column-major, as loaded
    float b1[kDim];
    uint64_t mbar;             // MMA completion
    uint64_t mbar_ld;          // bulk copies of S2
    uint64_t mbar_ld2;         // bulk copies of S1
    uint32_t tmem;
};
constexpr uint32_t kMatBytes = kDim * kDim * sizeof(float);
constexpr uint32_t kLoadChunk = 16384;  // bytes per bulk copy

// mbarrier set-up of a compose's shared memory (one thread), made visible to
// the async proxy; the caller synchronises the CTA afterwards
template <class Sm>
__device__ __forceinline__ void init_barriers(Sm& sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.mbar, 1);
        mbar_init(&sm.mbar_ld, 1);
        mbar_init(&sm.mbar_ld2, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// After a copy wait gave up: wait (default bound) for both inputs' copies,
// CTA-wide, before the shared memory they write is released or reused.
__device__ __forceinline__ int drain_loads(ComposeSmem& sm, uint32_t phase) {
    const bool drained =
        __syncthreads_and((mbar_wait(&sm.mbar_ld, phase) && mbar_wait(&sm.mbar_ld2, phase)) ? 1 : 0) != 0;
    return drained ? kTcTimedOut : kTcStuck;
}

// One compose by a CTA of 128 or 256 threads (with 256, two threads share a
// row in the epilogue, each taking 64 columns); every thread of the CTA
// calls it.  Returns kTcOk, or kTcTimedOut / kTcStuck when a wait gave up
// (then nothing is written).  `phase` is the parity of this CTA's MMA
// completions so far (and of its bulk loads: bulk loads only in the CTA's
// first compose).  bulk = false reads the inputs with L2 loads instead, for
// inputs that other CTAs of the same launch wrote (ordered by the caller's
// acquire).  load_polls and mma_polls bound the first wait for the copies and
// for the product; a wait that gives up is followed by a second one with the
// default bound for the operation already in flight, and every decision is
// taken CTA-wide (the TMEM loads are warp-collective).
__device__ __forceinline__ int compose_tc(ComposeSmem& sm, const float* __restrict__ S2,
                                          const float* __restrict__ b2, const float* __restrict__ S1,
                                          const float* __restrict__ b1, float* __restrict__ So,
                                          float* __restrict__ bo, uint32_t phase, bool bulk = true,
                                          uint64_t load_polls = kSpinLimit, uint64_t mma_polls = kSpinLimit) {
    const int tid = threadIdx.x, warp = tid >> 5;
    if (bulk) {
        // each input by its own bulk copies and mbarrier; b1 by plain loads meanwhile
        if (tid == 0) {
            mbar_expect_tx(&sm.mbar_ld, kMatBytes);
            mbar_expect_tx(&sm.mbar_ld2, kMatBytes);
            for (uint32_t o = 0; o < kMatBytes; o += kLoadChunk)
                bulk_load(reinterpret_cast<uint8_t*>(sm.S2f) + o, reinterpret_cast<const uint8_t*>(S2) + o,
                          kLoadChunk, &sm.mbar_ld);
            for (uint32_t o = 0; o < kMatBytes; o += kLoadChunk)
                bulk_load(reinterpret_cast<uint8_t*>(sm.S1f) + o, reinterpret_cast<const uint8_t*>(S1) + o,
                          kLoadChunk, &sm.mbar_ld2);
        }
        if (tid < kDim) sm.b1[tid] = __ldcg(b1 + tid);
        if (__syncthreads_and(mbar_wait(&sm.mbar_ld, phase, load_polls) ? 1 : 0) == 0) return drain_loads(sm, phase);
    } else {
        // 16-byte asynchronous copies through L2, all in flight at once: S2
        // in the first commit group, S1 in the second
        const float4* s2 = reinterpret_cast<const float4*>(S2);
        const float4* s1 = reinterpret_cast<const float4*>(S1);
        float4* d2 = reinterpret_cast<float4*>(sm.S2f);
        float4* d1 = reinterpret_cast<float4*>(sm.S1f);
        for (int i = tid; i < kDim * kDim / 4; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                         :: "r"(smem_addr(d2 + i)), "l"(s2 + i) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int i = tid; i < kDim * kDim / 4; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                         :: "r"(smem_addr(d1 + i)), "l"(s1 + i) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (tid < kDim) sm.b1[tid] = __ldcg(b1 + tid);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
    }
    // A(m, k) = S2[m][k] = S2 column-major [k][m]: thread gathers 8 consecutive
    // k of one row m (conflict-free across the warp) into one 16-byte core row
    for (int idx = tid; idx < kDim * (kDim / 8); idx += blockDim.x) {
        const int m = idx % kDim, kc = (idx / kDim) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = sm.S2f[(kc + j) * kDim + m];
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]), h1 = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]), h3 = __floats2bfloat162_rn(v[6], v[7]);
        uint4 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&h0);
        pk.y = *reinterpret_cast<uint32_t*>(&h1);
        pk.z = *reinterpret_cast<uint32_t*>(&h2);
        pk.w = *reinterpret_cast<uint32_t*>(&h3);
        *reinterpret_cast<uint4*>(sm.A + core_off(m, kc)) = pk;
    }
    if (bulk) {
        if (__syncthreads_and(mbar_wait(&sm.mbar_ld2, phase, load_polls) ? 1 : 0) == 0)
            return drain_loads(sm, phase);
    } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
    }
    // B(n, k) = S1[k][n] = S1 column-major [n][k]: 8 consecutive k of one n are
    // 32 contiguous bytes.  Consecutive threads take consecutive n, and chunk
    // j + (n mod 8) of it: the 16-byte stores of 8 lanes fill one 128-byte
    // core matrix row set (no bank conflicts), the loads meet at most 2-way.
    for (int idx = tid; idx < kDim * (kDim / 8); idx += blockDim.x) {
        const int n = idx & (kDim - 1), kc = (((idx >> 7) + (n & 7)) & (kDim / 8 - 1)) * 8;
        const float4 lo = *reinterpret_cast<const float4*>(sm.S1f + n * kDim + kc);
        const float4 hi = *reinterpret_cast<const float4*>(sm.S1f + n * kDim + kc + 4);
        __nv_bfloat162 h0 = __floats2bfloat162_rn(lo.x, lo.y), h1 = __floats2bfloat162_rn(lo.z, lo.w);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(hi.x, hi.y), h3 = __floats2bfloat162_rn(hi.z, hi.w);
        uint4 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&h0);
        pk.y = *reinterpret_cast<uint32_t*>(&h1);
        pk.z = *reinterpret_cast<uint32_t*>(&h2);
        pk.w = *reinterpret_cast<uint32_t*>(&h3);
        *reinterpret_cast<uint4*>(sm.B + core_off(n, kc)) = pk;
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
        const uint32_t a0 = smem_addr(sm.A), b0 = smem_addr(sm.B), idesc = make_idesc();
#pragma unroll
        for (int s = 0; s < kDim / 16; ++s)
            mma_bf16(sm.tmem, make_desc(a0 + s * 2 * kCoreBytes), make_desc(b0 + s * 2 * kCoreBytes), idesc,
                     s > 0 ? 1u : 0u);
        mma_commit(&sm.mbar);
    }
    // while the product runs (it reads only the A and B tiles): the vector
    // part b = b2 + b1 + S2 b1 from the staged BF16 rows of S2 (the same
    // operand the product uses), FP32 accumulation, kept in a register until
    // the product is known to be done (threads 0 .. 127); and S1f <- S1 + S2
    // for the epilogue (the other threads; with 128 threads, all of them
    // after the vector part)
    const int m = tid & (kDim - 1);
    float bvec = 0.f;
    if (tid < kDim) {
        float sacc = __ldcg(b2 + m) + sm.b1[m];
#pragma unroll 4
        for (int kc = 0; kc < kDim; kc += 8) {
            const uint4 pk = *reinterpret_cast<const uint4*>(sm.A + core_off(m, kc));
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&pk);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 f = __bfloat1622float2(h[j]);
                sacc = fmaf(f.x, sm.b1[kc + 2 * j], sacc);
                sacc = fmaf(f.y, sm.b1[kc + 2 * j + 1], sacc);
            }
        }
        bvec = sacc;
    }
    {
        const int nadd = blockDim.x > kDim ? blockDim.x - kDim : blockDim.x;
        const int t0 = blockDim.x > kDim ? tid - kDim : tid;
        if (t0 >= 0) {
            float4* s1 = reinterpret_cast<float4*>(sm.S1f);
            const float4* s2 = reinterpret_cast<const float4*>(sm.S2f);
            for (int i = t0; i < kDim * kDim / 4; i += nadd) {
                float4 x = s2[i];
                const float4 y = s1[i];
                x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
                s1[i] = x;
            }
        }
    }
    const bool done = __syncthreads_and(mbar_wait(&sm.mbar, phase, mma_polls) ? 1 : 0) != 0;
    if (!done) {
        // the product is in flight: no TMEM load, and no return (after which
        // the caller frees the TMEM) before its commit has arrived
        const bool drained = __syncthreads_and(mbar_wait(&sm.mbar, phase) ? 1 : 0) != 0;
        fence_after();
        return drained ? kTcTimedOut : kTcStuck;
    }
    fence_after();
    // epilogue: thread owns row m (TMEM lane m; a warp reaches the lane
    // quarter warp % 4) and a range of columns, and stores column-major
    // (coalesced across the warp)
    const int halves = blockDim.x / kDim;  // 1 or 2
    const int cols = kDim / halves, c0 = (tid / kDim) * cols;
    const uint32_t trow = sm.tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
    for (int c = c0; c < c0 + cols; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const size_t off = (size_t)(c + j) * kDim + m;
            So[off] = sm.S1f[off] + v[j];
        }
    }
    if (tid < kDim) bo[m] = bvec;
    fence_before();
    __syncthreads();
    return kTcOk;
}

// ---------------------------------------------------------------------------
// The same compose with TF32 operands (tcgen05.mma kind::tf32).  The FP32
// aggregates are the operands as they stand: a 32-bit container per element,
// of which the tensor core uses the TF32 part (10 explicit mantissa bits
// against BF16's 7), accumulating in FP32.  Core matrices of the canonical
// K-major layout hold 8 rows x 4 elements (16 bytes per row); one MMA takes
// K = 8, so K = 128 is 16 MMAs.  S1 arrives column-major by asynchronous
// copies into a staging tile, from which its operand tile is built in shared
// memory; S2's operand tile is gathered from L2 meanwhile (its rows are
// strided in memory).  The epilogue takes S2 from its operand tile and S1
// from the staging tile; the vector part uses the FP32 rows of S2 while the
// product runs.
// ---------------------------------------------------------------------------
constexpr uint32_t kGroupBytes32 = 32 * kCoreBytes;      // one 8-row group spans K = 128 (32 cores)
constexpr uint32_t kTileBytes32 = 16 * kGroupBytes32;    // 128 rows, 64 KB

__device__ __forceinline__ uint32_t core_off32(int row, int k) {
    return (uint32_t)((row >> 3) * kGroupBytes32 + (k >> 2) * kCoreBytes + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t make_desc32(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kCoreBytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kGroupBytes32 >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::tf32: D = F32, A = B = TF32 (format 2),
// both K-major, N = 128, M = 128
__device__ __forceinline__ uint32_t make_idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kDim >> 3) << 17) | ((uint32_t)(kDim >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

struct __align__(1024) ComposeSmem32 {
    uint8_t A[kTileBytes32];   // S2 (rows m, K-major), FP32 bits
    uint8_t B[kTileBytes32];   // S1 (rows n = columns of S1, K-major), FP32 bits
    float S1f[kDim * kDim];    // S1 column-major as loaded; the result tile in the epilogue
    float b1[kDim];
    uint64_t mbar;             // MMA completion
    uint64_t mbar_ld, mbar_ld2;  // unused (kept so both layouts share the set-up code)
    uint32_t tmem;
};

// One TF32 compose by a CTA of 128 or 256 threads; every thread calls it.
// Inputs by L2 loads (the caller orders them after their writers); returns
// kTcOk, or kTcTimedOut / kTcStuck as compose_tc (then nothing is written).
__device__ __forceinline__ int compose_tc32(ComposeSmem32& sm, const float* __restrict__ S2,
                                            const float* __restrict__ b2, const float* __restrict__ S1,
                                            const float* __restrict__ b1, float* __restrict__ So,
                                            float* __restrict__ bo, uint32_t phase,
                                            uint64_t mma_polls = kSpinLimit) {
    const int tid = threadIdx.x, warp = tid >> 5;
    // S1 (column-major, contiguous) into the staging tile: 16-byte
    // asynchronous copies through L2, all in flight while A is gathered
    {
        const float4* s1 = reinterpret_cast<const float4*>(S1);
        float4* d1 = reinterpret_cast<float4*>(sm.S1f);
        for (int i = tid; i < kDim * kDim / 4; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                         :: "r"(smem_addr(d1 + i)), "l"(s1 + i) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    if (tid < kDim) sm.b1[tid] = __ldcg(b1 + tid);
    // A(m, k) = S2[m][k], stored column-major at k * 128 + m: thread (m, kq)
    // gathers k = 4 kq .. 4 kq + 3 (four coalesced warp loads) into one
    // 16-byte core row; lanes run over m, so a phase of 8 lanes fills one
    // 128-byte core matrix (no bank conflicts)
    // (kU core rows per thread and batch: all their loads are issued before
    // any of their stores, so that many L2 requests are in flight at once)
    constexpr int kU = 8;
    constexpr int kRows = kDim * (kDim / 4);
    for (int base = tid; base < kRows; base += kU * blockDim.x) {
        float4 v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < kRows) {
                const int m = idx & (kDim - 1), k = (idx >> 7) * 4;
                v[u].x = __ldcg(S2 + (size_t)k * kDim + m);
                v[u].y = __ldcg(S2 + (size_t)(k + 1) * kDim + m);
                v[u].z = __ldcg(S2 + (size_t)(k + 2) * kDim + m);
                v[u].w = __ldcg(S2 + (size_t)(k + 3) * kDim + m);
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < kRows) *reinterpret_cast<float4*>(sm.A + core_off32(idx & (kDim - 1), (idx >> 7) * 4)) = v[u];
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // B(n, k) = S1[k][n] = S1f[n * 128 + k]: 4 consecutive k of one n are 16
    // contiguous bytes.  Consecutive threads take consecutive n and k group
    // j + (n mod 8): the 8 lanes of a phase store into one 128-byte core
    // matrix and load from 8 distinct bank groups (no conflicts either way).
    for (int idx = tid; idx < kRows; idx += blockDim.x) {
        const int n = idx & (kDim - 1), k = (((idx >> 7) + (n & 7)) & (kDim / 4 - 1)) * 4;
        *reinterpret_cast<float4*>(sm.B + core_off32(n, k)) = *reinterpret_cast<const float4*>(sm.S1f + n * kDim + k);
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
        const uint32_t a0 = smem_addr(sm.A), b0 = smem_addr(sm.B), idesc = make_idesc_tf32();
#pragma unroll
        for (int s = 0; s < kDim / 8; ++s)
            mma_tf32(sm.tmem, make_desc32(a0 + s * 2 * kCoreBytes), make_desc32(b0 + s * 2 * kCoreBytes), idesc,
                     s > 0 ? 1u : 0u);
        mma_commit(&sm.mbar);
    }
    // while the product runs: the vector part from the FP32 rows of S2 in the
    // A tile, FP32 accumulation, kept in a register until the product is done
    const int m = tid & (kDim - 1);
    float bvec = 0.f;
    if (tid < kDim) {
        float sacc = __ldcg(b2 + m) + sm.b1[m];
#pragma unroll 4
        for (int kc = 0; kc < kDim; kc += 4) {
            const float4 a = *reinterpret_cast<const float4*>(sm.A + core_off32(m, kc));
            sacc = fmaf(a.x, sm.b1[kc], sacc);
            sacc = fmaf(a.y, sm.b1[kc + 1], sacc);
            sacc = fmaf(a.z, sm.b1[kc + 2], sacc);
            sacc = fmaf(a.w, sm.b1[kc + 3], sacc);
        }
        bvec = sacc;
    }
    const bool done = __syncthreads_and(mbar_wait(&sm.mbar, phase, mma_polls) ? 1 : 0) != 0;
    if (!done) {
        const bool drained = __syncthreads_and(mbar_wait(&sm.mbar, phase) ? 1 : 0) != 0;
        fence_after();
        return drained ? kTcTimedOut : kTcStuck;
    }
    fence_after();
    // epilogue: row m, a range of columns; S2 (m, c..c+3) is one 16-byte core
    // row of the A tile, S1 (m, c) the staging tile's column c; stores
    // column-major (coalesced across the warp)
    const int halves = blockDim.x / kDim;  // 1 or 2
    const int cols = kDim / halves, c0 = (tid / kDim) * cols;
    const uint32_t trow = sm.tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
    for (int c = c0; c < c0 + cols; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = *reinterpret_cast<const float4*>(sm.A + core_off32(m, c + 4 * q));
            const float s2[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * q + e;
                const size_t off = (size_t)(c + j) * kDim + m;
                So[off] = s2[e] + sm.S1f[off] + v[j];
            }
        }
    }
    if (tid < kDim) bo[m] = bvec;
    fence_before();
    __syncthreads();
    return kTcOk;
}

}  // namespace tc
}  // namespace pitn
