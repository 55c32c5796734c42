// Algorithm 1 end to end on one stream: normalise -> decompose -> reconstruct
// -> expand, with optional host input/output staged through the workspace.
#include "common.cuh"

namespace fhr {
fhr_status reconstruct_impl(fhr_ctx *ctx, const fhr_geom *g, const fhr_mbir_params *p, const float *sino, float *xs,
                            void *ws, size_t ws_bytes);
size_t reconstruct_ws_bytes(const fhr_geom *g, int K);
fhr_status fbp_impl(fhr_ctx *ctx, const fhr_geom *g, int Wl, const float *sino, float *xs, void *ws,
                    size_t ws_bytes);
size_t fbp_ws_bytes(const fhr_geom *g, int Wl);
fhr_status expand_impl(fhr_ctx *ctx, int N, int Nr, int K, int Nk, int k0, int k1, const float *xs, const float *D,
                       int dt, void *xh);

// Copy streams of the host-I/O form, created on first use.
static fhr_status io_init(fhr_ctx *ctx) {
    if (ctx->io_ready) return FHR_OK;
    FHR_CUDA(cudaStreamCreateWithFlags(&ctx->io_h2d, cudaStreamNonBlocking));
    FHR_CUDA(cudaStreamCreateWithFlags(&ctx->io_d2h, cudaStreamNonBlocking));
    cudaEvent_t *evs[4] = {&ctx->ev_in_ready, &ctx->ev_in_free, &ctx->ev_out_ready, &ctx->ev_out_free};
    for (cudaEvent_t *e : evs) FHR_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    ctx->io_ready = 1;
    return FHR_OK;
}

struct PipeWs {
    int *status;
    uint16_t *y, *y0;
    void *P;
    float *W, *xs, *b;
    void *xh;
    void *nmf_ws, *mbir_ws;
    size_t nmf_bytes, mbir_bytes;
};

// the nested calls keep their own status words; fold them into the pipeline's
__global__ void gather_status(int *status, const int *a, const int *b) {
    if (threadIdx.x == 0) {
        if (*a) report(status, *a);
        if (*b) report(status, *b);
    }
}

static fhr_status pipe_check(fhr_ctx *ctx, const fhr_pipeline_params *p) {
    FHR_ARG(p, "params is null");
    const fhr_norm_params &n = p->norm;
    FHR_ARG(p->nmf.Np == (int64_t)n.Nv * n.Nr * n.Nc, "nmf.Np != Nv*Nr*Nc");
    FHR_ARG(p->nmf.Nk == n.Nk && p->nmf.ldP == n.ldP && p->nmf.p_dtype == n.p_dtype, "norm and nmf disagree");
    FHR_ARG(p->geom.Nr == n.Nr && p->geom.Nc == n.Nc && p->geom.Nv == n.Nv, "geometry and counts disagree");
    FHR_ARG(p->mbir.K == p->nmf.K, "mbir.K != nmf.K");
    FHR_ARG(p->nmf.init == FHR_INIT_NNDSVD || p->nmf.init == FHR_INIT_CLUSTER || p->nmf.init == FHR_INIT_LEARNED,
            "the pipeline starts the decomposition from NNDSVD, the clustering start or the learned start");
    FHR_ARG(p->xh_dtype == FHR_F32 || p->xh_dtype == FHR_BF16, "bad xh_dtype");
    FHR_ARG(p->recon == FHR_RECON_MBIR || p->recon == FHR_RECON_FBP, "bad recon");
    return FHR_OK;
}

static fhr_status pipe_carve(fhr_ctx *ctx, const fhr_pipeline_params *p, void *base, PipeWs *w, size_t *total) {
    const fhr_norm_params &n = p->norm;
    const int K = p->nmf.K;
    Carve c(base);
    PipeWs t;
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    const size_t ny = (size_t)n.Nv * n.Nr * n.Nc * n.Nk, ny0 = (size_t)n.Nr * n.Nc * n.Nk;
    const size_t nxh = (size_t)n.Nr * p->geom.N * p->geom.N * n.Nk;
    t.y = p->host_io ? c.take<uint16_t>(ny) : nullptr;
    t.y0 = p->host_io ? c.take<uint16_t>(ny0) : nullptr;
    t.xh = p->host_io ? (void *)c.take<char>(nxh * (p->xh_dtype == FHR_BF16 ? 2 : 4)) : nullptr;
    t.P = c.take<char>((size_t)p->nmf.Np * n.ldP * (n.p_dtype == FHR_BF16 ? 2 : 4));
    t.W = c.take<float>((size_t)p->nmf.Np * K);
    t.b = c.take<float>((size_t)n.Nv * n.Nk);
    t.xs = c.take<float>((size_t)p->geom.N * p->geom.N * n.Nr * K);
    FHR_TRY(fhr_decompose_workspace_size(ctx, &p->nmf, &t.nmf_bytes));
    t.nmf_ws = c.take<char>(t.nmf_bytes);
    t.mbir_bytes = p->recon == FHR_RECON_FBP ? fbp_ws_bytes(&p->geom, p->geom.Nr * K)
                                             : reconstruct_ws_bytes(&p->geom, K);
    t.mbir_ws = c.take<char>(t.mbir_bytes);
    if (w) *w = t;
    *total = c.size();
    return FHR_OK;
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_pipeline_workspace_size(fhr_ctx *ctx, const fhr_pipeline_params *p, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(pipe_check(ctx, p));
    FHR_ARG(bytes, "bytes is null");
    FHR_CUDA(cudaSetDevice(ctx->device));
    return pipe_carve(ctx, p, nullptr, nullptr, bytes);
}

extern "C" fhr_status fhr_pipeline(fhr_ctx *ctx, const fhr_pipeline_params *p, const uint16_t *y, const uint16_t *y0,
                                   const uint8_t *bg, const uint8_t *dead, float *D_out, void *xh, double *obj,
                                   void *ws, size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(pipe_check(ctx, p));
    FHR_ARG(y && y0 && D_out && xh && ws, "null pointer argument");
    FHR_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
    FHR_CUDA(cudaSetDevice(ctx->device));
    PipeWs w;
    size_t need = 0;
    FHR_TRY(pipe_carve(ctx, p, ws, &w, &need));
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    cudaStream_t st = ctx->stream;
    const fhr_norm_params &n = p->norm;
    const int K = p->nmf.K;
    FHR_CUDA(cudaMemsetAsync(w.status, 0, kStatusBytes, st));
    const uint16_t *yd = y, *y0d = y0;
    const size_t ny = (size_t)n.Nv * n.Nr * n.Nc * n.Nk, ny0 = (size_t)n.Nr * n.Nc * n.Nk;
    if (p->host_io) {
        // Host I/O runs on two copy streams, so consecutive calls overlap: this
        // call's input copy waits only until the previous call has normalised its
        // staged counts, and its output copy runs behind the next call's compute.
        FHR_TRY(io_init(ctx));
        FHR_CUDA(cudaStreamWaitEvent(ctx->io_h2d, ctx->ev_in_free, 0));
        FHR_CUDA(cudaMemcpyAsync(w.y, y, ny * 2, cudaMemcpyHostToDevice, ctx->io_h2d));
        FHR_CUDA(cudaMemcpyAsync(w.y0, y0, ny0 * 2, cudaMemcpyHostToDevice, ctx->io_h2d));
        FHR_CUDA(cudaEventRecord(ctx->ev_in_ready, ctx->io_h2d));
        FHR_CUDA(cudaStreamWaitEvent(st, ctx->ev_in_ready, 0));
        yd = w.y;
        y0d = w.y0;
    }
    FHR_TRY(fhr_normalise(ctx, &n, yd, y0d, bg, dead, bg ? w.b : nullptr, w.P));
    if (p->host_io) FHR_CUDA(cudaEventRecord(ctx->ev_in_free, st));
    FHR_TRY(fhr_decompose(ctx, &p->nmf, w.P, D_out, w.W, obj, w.nmf_ws, w.nmf_bytes));
    const size_t nxs = (size_t)p->geom.N * p->geom.N * n.Nr * K;
    FHR_CUDA(cudaMemsetAsync(w.xs, 0, nxs * sizeof(float), st));
    if (p->recon == FHR_RECON_FBP)
        FHR_TRY(fbp_impl(ctx, &p->geom, n.Nr * K, w.W, w.xs, w.mbir_ws, w.mbir_bytes));
    else
        FHR_TRY(reconstruct_impl(ctx, &p->geom, &p->mbir, w.W, w.xs, w.mbir_ws, w.mbir_bytes));
    void *xo = p->host_io ? w.xh : xh;
    // the staged output is reused once the previous call's output copy is done
    if (p->host_io) FHR_CUDA(cudaStreamWaitEvent(st, ctx->ev_out_free, 0));
    FHR_TRY(expand_impl(ctx, p->geom.N, n.Nr, K, n.Nk, 0, 0, w.xs, D_out, p->xh_dtype, xo));
    gather_status<<<1, 32, 0, st>>>(w.status, (const int *)w.nmf_ws, (const int *)w.mbir_ws);
    FHR_LAUNCHED();
    if (p->host_io) {
        const size_t nxh = (size_t)n.Nr * p->geom.N * p->geom.N * n.Nk * (p->xh_dtype == FHR_BF16 ? 2 : 4);
        FHR_CUDA(cudaEventRecord(ctx->ev_out_ready, st));
        FHR_CUDA(cudaStreamWaitEvent(ctx->io_d2h, ctx->ev_out_ready, 0));
        FHR_CUDA(cudaMemcpyAsync(xh, w.xh, nxh, cudaMemcpyDeviceToHost, ctx->io_d2h));
        FHR_CUDA(cudaEventRecord(ctx->ev_out_free, ctx->io_d2h));
    }
    return FHR_OK;
}
