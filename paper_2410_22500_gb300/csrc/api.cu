// Context management, errors and the workspace status word.
#include <stdarg.h>
#include <stdlib.h>

#include "common.cuh"

namespace fhr {
fhr_status set_error(fhr_ctx *ctx, fhr_status code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}
// Start event of a fresh (start, stop) pair for timer `id`, recorded now;
// NULL when profiling is off or no event could be created.
cudaEvent_t *timer_begin(fhr_ctx *ctx, int id) {
    if (!ctx->prof_on || id < 0 || id >= TM_COUNT) return nullptr;
    auto &t = ctx->tm[id];
    if (t.used == t.cap) {
        const int ncap = t.cap ? 2 * t.cap : 64;
        cudaEvent_t *nev = (cudaEvent_t *)realloc(t.ev, sizeof(cudaEvent_t) * 2 * ncap);
        if (!nev) return nullptr;
        for (int i = 2 * t.cap; i < 2 * ncap; ++i)
            if (cudaEventCreate(&nev[i]) != cudaSuccess) {
                t.ev = nev;
                return nullptr;
            }
        t.ev = nev;
        t.cap = ncap;
    }
    cudaEvent_t *e = &t.ev[2 * t.used++];
    cudaEventRecord(e[0], ctx->stream);
    return e;
}

static const char *kTimerNames[TM_COUNT] = {"normalise", "nmf_pass", "nmf_reduce", "nmf_update", "proj_fwd",
                                            "mbir_update", "proj_bwd", "expand", "nndsvd_pass", "fbp_filter",
                                            "mlp_forward", "fmd"};

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_profile_enable(fhr_ctx *ctx, int enable) {
    if (!ctx) return FHR_ERR_ARG;
    ctx->prof_on = enable ? 1 : 0;
    ctx->launches = 0;
    for (int i = 0; i < TM_COUNT; ++i) ctx->tm[i].used = 0;
    return FHR_OK;
}

extern "C" fhr_status fhr_profile_read(fhr_ctx *ctx, const char *name, long long *launches, double *ms) {
    if (!ctx) return FHR_ERR_ARG;
    if (!name) {
        if (launches) *launches = ctx->launches;
        if (ms) *ms = 0.0;
        return FHR_OK;
    }
    for (int i = 0; i < TM_COUNT; ++i) {
        if (strcmp(name, kTimerNames[i]) != 0) continue;
        auto &t = ctx->tm[i];
        double total = 0.0;
        for (int j = 0; j < t.used; ++j) {
            FHR_CUDA(cudaEventSynchronize(t.ev[2 * j + 1]));
            float e = 0.f;
            FHR_CUDA(cudaEventElapsedTime(&e, t.ev[2 * j], t.ev[2 * j + 1]));
            total += e;
        }
        if (launches) *launches = t.used;
        if (ms) *ms = total;
        return FHR_OK;
    }
    return set_error(ctx, FHR_ERR_ARG, "unknown timer '%s'", name);
}

extern "C" fhr_status fhr_create(fhr_ctx **out, int device, void *stream) {
    fhr_ctx *ctx = nullptr;
    if (!out) return FHR_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return FHR_ERR_ARG;
    ctx = (fhr_ctx *)calloc(1, sizeof(fhr_ctx));
    if (!ctx) return FHR_ERR_ARG;
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        free(ctx);
        return FHR_ERR_CUDA;
    }
    if (prop.major < 10) {
        free(ctx);
        return FHR_ERR_UNSUPPORTED;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
    *out = ctx;
    return FHR_OK;
}

extern "C" void fhr_destroy(fhr_ctx *ctx) {
    if (!ctx) return;
    if (ctx->io_ready) {
        cudaStreamSynchronize(ctx->io_h2d);
        cudaStreamSynchronize(ctx->io_d2h);
        cudaEventDestroy(ctx->ev_in_ready);
        cudaEventDestroy(ctx->ev_in_free);
        cudaEventDestroy(ctx->ev_out_ready);
        cudaEventDestroy(ctx->ev_out_free);
        cudaStreamDestroy(ctx->io_h2d);
        cudaStreamDestroy(ctx->io_d2h);
    }
    for (int i = 0; i < TM_COUNT; ++i) {
        for (int j = 0; j < 2 * ctx->tm[i].cap; ++j) cudaEventDestroy(ctx->tm[i].ev[j]);
        free(ctx->tm[i].ev);
    }
    free(ctx);
}

extern "C" fhr_status fhr_set_stream(fhr_ctx *ctx, void *stream) {
    if (!ctx) return FHR_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return FHR_OK;
}

extern "C" const char *fhr_last_error(const fhr_ctx *ctx) { return ctx ? ctx->err : "null context"; }

extern "C" const char *fhr_version(void) { return "libfhr 0.1 (sm_103a)"; }

extern "C" fhr_status fhr_io_join(fhr_ctx *ctx) {
    if (!ctx) return FHR_ERR_ARG;
    if (!ctx->io_ready) return FHR_OK;
    FHR_CUDA(cudaSetDevice(ctx->device));
    FHR_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_out_free, 0));
    return FHR_OK;
}

extern "C" fhr_status fhr_workspace_status(fhr_ctx *ctx, void *ws) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_ARG(ws, "workspace is null");
    FHR_CUDA(cudaSetDevice(ctx->device));
    if (ctx->io_ready) FHR_CUDA(cudaStreamSynchronize(ctx->io_d2h));
    int st = 0;
    FHR_CUDA(cudaMemcpyAsync(&st, ws, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    FHR_CUDA(cudaStreamSynchronize(ctx->stream));
    if (st != 0) {
        FHR_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), ctx->stream));
        return set_error(ctx, st, "device reported status %d", st);
    }
    return FHR_OK;
}
