// fhr_decompose_static: the subspace decomposition without a caller workspace.
//
// Some callers cannot hand the library a workspace.  A plugin that has to
// keep a fixed C signature has no argument to pass one.  A host framework
// may own every byte of device memory through its own allocator.  And in a
// latency-critical loop, a cudaMalloc (which may synchronise the whole device)
// is not allowed.  For them this entry point runs the same kernels as
// fhr_decompose.  Their scratch lives in one file-scope __device__ array of
// kStaticWorkspaceBytes.  Every GPU that loads the library keeps that array
// until the process exits.  Nothing here calls cudaMalloc, cudaFree or any
// other allocating routine.
#include <mutex>

#include "common.cuh"

namespace fhr {

// Upper bound of the scratch this entry point can use.
constexpr size_t kStaticWorkspaceBytes = 32u << 20;

static __device__ __align__(256) unsigned char g_static_ws[kStaticWorkspaceBytes];

// Device address of g_static_ws per device ordinal, looked up once per device.
constexpr int kMaxDevices = 64;
static void *g_static_ptr[kMaxDevices];
static std::mutex g_static_mu;

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_decompose_static(fhr_ctx *ctx, const fhr_nmf_params *prm, const void *P, float *D,
                                           float *W, double *obj) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_ARG(ctx->device >= 0 && ctx->device < kMaxDevices, "device ordinal out of range");
    size_t need = 0;
    FHR_TRY(fhr_decompose_workspace_size(ctx, prm, &need));
    if (need > kStaticWorkspaceBytes)
        return set_error(ctx, FHR_ERR_ARG,
                         "fhr_decompose_static: this problem needs %zu bytes of scratch, above the fixed %zu-byte "
                         "static workspace; use fhr_decompose with a caller workspace",
                         need, kStaticWorkspaceBytes);
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[ctx->device]) {
            // the host-side name of the array is not a device address: ask the
            // runtime for it, with this context's device current
            FHR_CUDA(cudaSetDevice(ctx->device));
            void *p = nullptr;
            FHR_CUDA(cudaGetSymbolAddress(&p, g_static_ws));
            g_static_ptr[ctx->device] = p;
        }
        ws = g_static_ptr[ctx->device];
    }
    // event timers would create driver objects; keep them off for this call
    const int prof = ctx->prof_on;
    ctx->prof_on = 0;
    const fhr_status st = fhr_decompose(ctx, prm, P, D, W, obj, ws, kStaticWorkspaceBytes);
    ctx->prof_on = prof;
    return st;
}

// The status word at the start of the static array: bounded waits that
// expired (FHR_ERR_TIMEOUT) and non-finite objectives (FHR_ERR_NONFINITE)
// of the static calls land there, as they land in a caller workspace for
// fhr_decompose.  Before the first static call on a device there is nothing
// to report.
extern "C" fhr_status fhr_decompose_static_status(fhr_ctx *ctx) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_ARG(ctx->device >= 0 && ctx->device < kMaxDevices, "device ordinal out of range");
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        ws = g_static_ptr[ctx->device];
    }
    if (!ws) return FHR_OK;
    return fhr_workspace_status(ctx, ws);
}
