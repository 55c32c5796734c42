// Filtered back-projection of the subspace sinograms: the paper's faster
// variant of the reconstruction step ("FHR with FBP", Sec. V / Table II).
//   q[v][c][w] = (pi / Nv) sum_c' h[c - c'] p[v][c'][w]   (ramp filter along the
//                detector, band-limited Ram-Lak samples at unit bin spacing)
//   x = A^T q                                           (strip-area back-projector)
// The filter is one block per (view, 32 values of w): the view's slab of p and
// the filter taps sit in shared memory; each thread owns one w and a stride of
// bins, so the reads of p are shared-memory broadcasts along c' and the writes
// of q are coalesced along w.
#include <math.h>

#include "proj.cuh"

namespace fhr {

constexpr int kFbpW = 32;        // values of w per block
constexpr int kFbpCG = 8;        // bin groups per block (threads = kFbpW * kFbpCG)
constexpr int kFbpMaxNc = 1024;  // shared slab limit: Nc * kFbpW floats + taps

// h[n] for n = -(Nc-1) .. Nc-1, scaled by pi / Nv
__device__ __forceinline__ float ramp_tap(int n, double scale) {
    if (n == 0) return (float)(0.25 * scale);
    if (n & 1) return (float)(-scale / (3.141592653589793 * 3.141592653589793 * (double)n * (double)n));
    return 0.f;
}

__global__ void __launch_bounds__(kFbpW * kFbpCG) fbp_filter_kernel(const float *__restrict__ p, float *__restrict__ q,
                                                                    int Nc, int Wl, double scale) {
    extern __shared__ float sh[];
    float *slab = sh;                        // [Nc][kFbpW]
    float *taps = sh + (size_t)Nc * kFbpW;   // [2 Nc - 1], taps[n + Nc - 1] = h[n]
    const int v = blockIdx.x;
    const int w0 = blockIdx.y * kFbpW;
    const int tid = threadIdx.x;
    const int lw = tid % kFbpW, cg = tid / kFbpW;
    const int w = w0 + lw;
    const float *pv = p + (size_t)v * Nc * Wl;
    for (int i = tid; i < Nc * kFbpW; i += blockDim.x) {
        const int c = i / kFbpW, ww = w0 + i % kFbpW;
        slab[i] = ww < Wl ? pv[(size_t)c * Wl + ww] : 0.f;
    }
    for (int i = tid; i < 2 * Nc - 1; i += blockDim.x) taps[i] = ramp_tap(i - (Nc - 1), scale);
    __syncthreads();
    if (w >= Wl) return;
    float *qv = q + (size_t)v * Nc * Wl;
    for (int c = cg; c < Nc; c += kFbpCG) {
        // h[0] term, then the odd offsets d = c - c' (even ones vanish)
        float acc = taps[Nc - 1] * slab[c * kFbpW + lw];
        for (int c2 = (c & 1) ? 0 : 1; c2 < Nc; c2 += 2) acc = fmaf(taps[c - c2 + Nc - 1], slab[c2 * kFbpW + lw], acc);
        qv[(size_t)c * Wl + w] = acc;
    }
}

struct FbpWs {
    int *status;
    ProjTables t;
    float *q;
};

static size_t carve_fbp(void *base, const fhr_geom *g, int Wl, FbpWs *w) {
    Carve c(base);
    FbpWs t;
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    proj_tables_carve(c, g->N, g->Nc, g->Nv, &t.t);
    t.q = c.take<float>((size_t)g->Nv * g->Nc * Wl);
    if (w) *w = t;
    return c.size();
}

static fhr_status check_fbp(fhr_ctx *ctx, const fhr_geom *g, int Wl) {
    FHR_TRY(check_geom(ctx, g, Wl));
    FHR_ARG(g->Nc <= kFbpMaxNc, "Nc must be <= %d for the ramp filter", kFbpMaxNc);
    return FHR_OK;
}

size_t fbp_ws_bytes(const fhr_geom *g, int Wl) { return carve_fbp(nullptr, g, Wl, nullptr); }

fhr_status fbp_impl(fhr_ctx *ctx, const fhr_geom *g, int Wl, const float *sino, float *xs, void *ws,
                    size_t ws_bytes) {
    FHR_TRY(check_fbp(ctx, g, Wl));
    FHR_ARG(sino && xs && ws, "null pointer argument");
    FHR_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
    FHR_ARG(Wl % 4 != 0 || aligned(xs, 16), "xs must be 16-byte aligned");
    FbpWs w;
    const size_t need = carve_fbp(ws, g, Wl, &w);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    FHR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    FHR_CUDA(cudaMemsetAsync(w.status, 0, kStatusBytes, st));
    FHR_TRY(proj_build_tables(ctx, g, w.t));
    const size_t smem = sizeof(float) * ((size_t)g->Nc * kFbpW + 2 * g->Nc);
    if (smem > 48 * 1024)
        FHR_CUDA(cudaFuncSetAttribute(fbp_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 grid((unsigned)g->Nv, (unsigned)cdiv(Wl, kFbpW));
    const double scale = 3.141592653589793 / (double)g->Nv;
    FHR_TIMED(TM_FBP_FILTER, (fbp_filter_kernel<<<grid, kFbpW * kFbpCG, smem, st>>>(sino, w.q, g->Nc, Wl, scale)));
    FHR_TRY(proj_backward(ctx, g, w.t, Wl, w.q, xs));
    return FHR_OK;
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_fbp_workspace_size(fhr_ctx *ctx, const fhr_geom *g, int Wl, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_fbp(ctx, g, Wl));
    FHR_ARG(bytes, "bytes is null");
    *bytes = fbp_ws_bytes(g, Wl);
    return FHR_OK;
}

extern "C" fhr_status fhr_fbp(fhr_ctx *ctx, const fhr_geom *g, int Wl, const float *sino, float *xs, void *ws,
                              size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    return fbp_impl(ctx, g, Wl, sino, xs, ws, ws_bytes);
}
