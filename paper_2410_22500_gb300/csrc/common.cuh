// Shared internals of libfhr (not part of the public ABI).
#pragma once

#include <algorithm>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "fhr.h"

// Per-context launch accounting: every kernel launch is counted; with
// profiling on, launches of the timed kernel families are bracketed by CUDA
// events on the context's stream (read back by fhr_profile_read).
enum FhrTimer { TM_NORMALISE = 0, TM_NMF_PASS, TM_NMF_REDUCE, TM_NMF_UPDATE, TM_PROJ_FWD, TM_MBIR_UPDATE,
                TM_PROJ_BWD, TM_EXPAND, TM_NNDSVD_PASS, TM_FBP_FILTER, TM_MLP_FORWARD, TM_FMD, TM_COUNT };

struct fhr_ctx {
    int device;
    cudaStream_t stream;
    int sm_count;
    int max_smem_optin;
    char err[512];
    long long launches;
    int prof_on;
    struct {
        cudaEvent_t *ev;       // pairs (start, stop)
        int used, cap;
    } tm[TM_COUNT];
    // host I/O of the pipeline: copy streams and the events that order them
    int io_ready;
    cudaStream_t io_h2d, io_d2h;
    cudaEvent_t ev_in_ready, ev_in_free, ev_out_ready, ev_out_free;
};

namespace fhr {

// ------------------------------------------------------------------ errors
fhr_status set_error(fhr_ctx *ctx, fhr_status code, const char *fmt, ...);

#define FHR_ARG(cond, ...)                                        \
    do {                                                          \
        if (!(cond)) return ::fhr::set_error(ctx, FHR_ERR_ARG, __VA_ARGS__); \
    } while (0)

#define FHR_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::fhr::set_error(ctx, FHR_ERR_CUDA, "%s: %s (%s:%d)", #call,        \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);        \
    } while (0)

#define FHR_LAUNCHED()                                                                  \
    do {                                                                                \
        ++ctx->launches;                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return ::fhr::set_error(ctx, FHR_ERR_CUDA, "launch failed: %s (%s:%d)",    \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);        \
    } while (0)

// Bracket one launch with the context's timer `id` when profiling is on.
#define FHR_TIMED(id, launch)                                               \
    do {                                                                    \
        cudaEvent_t *ev_ = ::fhr::timer_begin(ctx, (id));                   \
        launch;                                                             \
        if (ev_) cudaEventRecord(ev_[1], ctx->stream);                      \
        FHR_LAUNCHED();                                                     \
    } while (0)

#define FHR_TRY(expr)                  \
    do {                               \
        fhr_status s_ = (expr);        \
        if (s_ != FHR_OK) return s_;   \
    } while (0)

cudaEvent_t *timer_begin(fhr_ctx *ctx, int id);

static inline bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }
static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// Linear carve-out of a caller workspace in 256-byte aligned pieces.
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t n) {
        off = round_up(off, 256);
        T *p = base ? (T *)(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
    size_t size() const { return round_up(off, 256); }
};

// The first 256 bytes of every workspace hold the device status word.
constexpr size_t kStatusBytes = 256;

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void report(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded waits give up after this long and report FHR_ERR_TIMEOUT.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ float bf16_to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// -------- mbarrier / bulk-copy wrappers (PTX, sm_90+)
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000000;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false after kWaitLimitNs.
// The clock is read only every 64 polls so a short wait costs few instructions.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t n = 1;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 63u) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
}

// 1-D bulk copy global -> shared, completion counted on an mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Hint: bring [src, src + bytes) into L2 (no completion tracking; bytes % 16 == 0).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Ordinary-precision helpers
__device__ __forceinline__ float4 ld_nc_f4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

}  // namespace fhr
