// MBIR of the subspace sinograms, Eq. (recon), by separable quadratic
// surrogates (SQS) with the qGGMRF prior.  All Nr slices and K channels are
// one vector of Wl = Nr*K values per pixel, so each iteration is
//   1. e = V - A z                 (forward gather, residual fused)
//   2. x+ = max(0, z - g / d)      (backward gather fused with the prior's
//                                   gradient and surrogate curvature)
// with g = -A^T e / sv^2 + beta sum_n b_n rho'(z - z_n),
//      d = (A^T A 1) / sv^2 + beta sum_n 2 b_n rho'(z - z_n)/(z - z_n),
// and optional momentum z <- max(0, x+ + a_t (x+ - x)).
#include <math.h>

#include "proj_tma.cuh"

namespace fhr {

__device__ __forceinline__ void chan_from_sigmas(MbirChan *c, int j, float sv, float sx, float T, float p) {
    c->sv[j] = sv;
    c->sx[j] = sx;
    c->inv_sv2[j] = 1.f / (sv * sv);
    c->c0[j] = (float)(1.0 / (pow((double)T, 2.0 - (double)p) * (double)sx * (double)sx));
    c->inv_tsx[j] = 1.f / (T * sx);
}

__global__ void mbir_set_chan(SigmaArgs s, int K, float T, float p, MbirChan *out) {
    const int j = threadIdx.x;
    if (j < K) chan_from_sigmas(out, j, s.sv[j], s.sx[j], T, p);
}

// Per-channel sum and sum of squares of the sinogram [rows][K]; the last block
// turns them into sigma_v = rms 10^(-snr/20), sigma_x = 0.2 mean / Nc.
__global__ void mbir_sigma_kernel(const float *sino, int64_t rows, int K, double *part, unsigned *counter,
                                  float snr_db, int Nc, float T, float p, MbirChan *out) {
    __shared__ double sh[2 * kMbirMaxK][33];
    __shared__ bool last;
    float s1[kMbirMaxK], s2[kMbirMaxK];
    for (int j = 0; j < K; ++j) s1[j] = s2[j] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < K; ++j) {
            const float v = sino[i * K + j];
            s1[j] += v;
            s2[j] = fmaf(v, v, s2[j]);
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < 2 * K; ++j) {
        double v = j < K ? (double)s1[j] : (double)s2[j - K];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[j][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[threadIdx.x][w];
        part[(size_t)blockIdx.x * 2 * K + threadIdx.x] = a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < K) {
        const int j = threadIdx.x;
        double a1 = 0.0, a2 = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            a1 += part[(size_t)b * 2 * K + j];
            a2 += part[(size_t)b * 2 * K + K + j];
        }
        const double rms = sqrt(a2 / (double)rows), mean = a1 / (double)rows;
        float sv = 1.f, sx = 1.f;
        if (rms > 0.0 && mean > 0.0) {
            sv = (float)(rms * pow(10.0, -(double)snr_db / 20.0));
            sx = (float)(0.2 * mean / (double)Nc);
        }
        chan_from_sigmas(out, j, sv, sx, T, p);
    }
    if (threadIdx.x == 0) *counter = 0u;
}

__global__ void fill_kernel(float *x, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

template <int VW, int G>
__global__ void __launch_bounds__(kUpdateThreads, kUpdateMinBlocks) mbir_update_kernel(const float *__restrict__ e, const float *__restrict__ z,
                                                           const float *__restrict__ xprev, float *__restrict__ xnew,
                                                           float *__restrict__ znext, ProjTables t,
                                                           const float *__restrict__ dA, const MbirChan *__restrict__ chp,
                                                           MbirPrior pr, float mom_a, int N, int Nc, int Nv, int Nr,
                                                           int K, int Wl, int Wc) {
    const GatherIdx gi = gather_idx<VW, G>(N * N, Wl, Wc);
    if (!gi.ok) return;
    mbir_update_at<VW, G>(e, z, xprev, xnew, znext, t, dA, chp, pr, mom_a, N, Nc, Nv, Nr, K, Wl, gi.item, gi.w0, gi.gs);
}

struct MbirWs {
    int *status;
    ProjTables t;
    MbirChan *chan;
    double *sig_part;
    unsigned *counter;
    float *dA, *e, *buf[4];
};


static size_t carve_mbir(void *base, const fhr_geom *g, int K, MbirWs *w) {
    Carve c(base);
    MbirWs t;
    const int Wl = g->Nr * K;
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    t.counter = c.take<unsigned>(4);
    t.chan = c.take<MbirChan>(1);
    t.sig_part = c.take<double>((size_t)kSigBlocks * 2 * kMbirMaxK);
    proj_tables_carve(c, g->N, g->Nc, g->Nv, &t.t);
    t.dA = c.take<float>((size_t)g->N * g->N);
    t.e = c.take<float>((size_t)g->Nv * g->Nc * Wl);
    for (int i = 0; i < 4; ++i) t.buf[i] = c.take<float>((size_t)g->N * g->N * Wl);
    if (w) *w = t;
    return c.size();
}

static fhr_status check_mbir(fhr_ctx *ctx, const fhr_geom *g, const fhr_mbir_params *p) {
    FHR_ARG(p, "params is null");
    FHR_ARG(p->K >= 1 && p->K <= kMbirMaxK, "K must be 1..8");
    FHR_TRY(check_geom(ctx, g, g ? g->Nr * p->K : 1));
    FHR_ARG(p->iters >= 0, "iters < 0");
    if (p->q != 2.f) return set_error(ctx, FHR_ERR_UNSUPPORTED, "only q = 2 is implemented");
    FHR_ARG(p->p >= 1.f && p->p <= 2.f, "p must be in [1, 2]");
    FHR_ARG(p->T > 0.f, "T must be positive");
    FHR_ARG(p->beta >= 0.f, "beta must be >= 0");
    return FHR_OK;
}

template <int VW, int G>
static fhr_status launch_update_g(fhr_ctx *ctx, const fhr_geom *g, const GatherShape &s, const MbirWs &w,
                                  const float *z, const float *xp, float *xn, float *zn, const MbirPrior &pr, float a,
                                  int K, int Wl) {
    FHR_TIMED(TM_MBIR_UPDATE, (mbir_update_kernel<VW, G><<<s.blocks(g->N * g->N, Wl), s.threads, 0, ctx->stream>>>(
                                  w.e, z, xp, xn, zn, w.t, w.dA, w.chan, pr, a, g->N, g->Nc, g->Nv, g->Nr, K, Wl,
                                  s.wc)));
    return FHR_OK;
}

static fhr_status launch_update(fhr_ctx *ctx, const fhr_geom *g, const MbirWs &w, const float *z, const float *xp,
                                float *xn, float *zn, const MbirPrior &pr, float a, int K, int Wl) {
    if (tma_gathers_ok(g, Wl)) {
        TmaUpdate u;
        u.z = z;
        u.xprev = xp;
        u.znext = zn;
        u.dA = w.dA;
        u.chp = w.chan;
        u.pr = pr;
        u.mom_a = a;
        u.Nr = g->Nr;
        u.K = K;
        return tma_backward(ctx, g, w.t, Wl, w.e, xn, &u, w.status);
    }
    const GatherShape s = gather_shape(Wl, gather_slab_values(g), kGatherMaxGBwd, kUpdateThreads);
    if (s.vw == 4 && s.g == 2) return launch_update_g<4, 2>(ctx, g, s, w, z, xp, xn, zn, pr, a, K, Wl);
    if (s.vw == 4) return launch_update_g<4, 1>(ctx, g, s, w, z, xp, xn, zn, pr, a, K, Wl);
    return launch_update_g<1, 1>(ctx, g, s, w, z, xp, xn, zn, pr, a, K, Wl);
}

fhr_status reconstruct_impl(fhr_ctx *ctx, const fhr_geom *g, const fhr_mbir_params *p, const float *sino, float *xs,
                            void *ws, size_t ws_bytes) {
    FHR_TRY(check_mbir(ctx, g, p));
    FHR_ARG(sino && xs && ws, "null pointer argument");
    FHR_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
    const int K = p->K, Wl = g->Nr * K;
    FHR_ARG(Wl % 4 != 0 || (aligned(sino, 16) && aligned(xs, 16)), "sino and xs must be 16-byte aligned");
    MbirWs w;
    const size_t need = carve_mbir(ws, g, K, &w);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    FHR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    FHR_CUDA(cudaMemsetAsync(w.status, 0, kStatusBytes, st));
    FHR_CUDA(cudaMemsetAsync(w.counter, 0, 4 * sizeof(unsigned), st));
    FHR_TRY(proj_build_tables(ctx, g, w.t));

    // per-channel sigmas
    if (p->sigma_v && p->sigma_x) {
        SigmaArgs s;
        for (int j = 0; j < kMbirMaxK; ++j) {
            s.sv[j] = j < K ? p->sigma_v[j] : 1.f;
            s.sx[j] = j < K ? p->sigma_x[j] : 1.f;
            if (j < K) FHR_ARG(s.sv[j] > 0.f && s.sx[j] > 0.f, "sigmas must be positive");
        }
        mbir_set_chan<<<1, 32, 0, st>>>(s, K, p->T, p->p, w.chan);
    } else {
        const int64_t rows = (int64_t)g->Nv * g->Nc * g->Nr;
        mbir_sigma_kernel<<<kSigBlocks, 256, 0, st>>>(sino, rows, K, w.sig_part, w.counter, p->snr_db, g->Nc, p->T,
                                                      p->p, w.chan);
    }
    FHR_LAUNCHED();

    // SQS data-term curvature A^T A 1 (one value per pixel)
    const int64_t nx = (int64_t)g->N * g->N * Wl;
    fill_kernel<<<ctx->sm_count * 4, 256, 0, st>>>(w.buf[0], (int64_t)g->N * g->N, 1.f);
    FHR_LAUNCHED();
    FHR_TRY(proj_forward(ctx, g, w.t, 1, w.buf[0], w.e, nullptr));
    FHR_TRY(proj_backward(ctx, g, w.t, 1, w.e, w.dA));

    MbirPrior pr;
    pr.p = p->p;
    pr.T = p->T;
    pr.e = 2.f - p->p;
    pr.c1 = (2.f - p->p) / p->p;
    pr.beta = p->beta;
    const double r2 = 1.0 / sqrt(2.0);
    const double z = 4.0 + 4.0 * r2 + (g->Nr > 1 ? 2.0 : 0.0);
    pr.b_edge = (float)(1.0 / z);
    pr.b_diag = (float)(r2 / z);
    pr.b_slice = (float)(1.0 / z);

    if (p->iters == 0) return FHR_OK;
    const size_t xbytes = (size_t)nx * sizeof(float);
    float *X0 = w.buf[0], *Z0 = w.buf[1], *X1 = w.buf[2], *Z1 = w.buf[3];
    FHR_CUDA(cudaMemcpyAsync(X0, xs, xbytes, cudaMemcpyDeviceToDevice, st));
    if (p->momentum) FHR_CUDA(cudaMemcpyAsync(Z0, xs, xbytes, cudaMemcpyDeviceToDevice, st));
    else Z0 = X0;
    double tk = 1.0;
    for (int it = 0; it < p->iters; ++it) {
        FHR_TRY(proj_forward(ctx, g, w.t, Wl, Z0, w.e, sino, w.status));
        float a = 0.f;
        if (p->momentum) {
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
            a = (float)((tk - 1.0) / tn);
            tk = tn;
            FHR_TRY(launch_update(ctx, g, w, Z0, X0, X1, Z1, pr, a, K, Wl));
            std::swap(X0, X1);
            std::swap(Z0, Z1);
        } else {
            FHR_TRY(launch_update(ctx, g, w, Z0, nullptr, X1, nullptr, pr, 0.f, K, Wl));
            std::swap(X0, X1);
            Z0 = X0;
        }
    }
    FHR_CUDA(cudaMemcpyAsync(xs, X0, xbytes, cudaMemcpyDeviceToDevice, st));
    return FHR_OK;
}

size_t reconstruct_ws_bytes(const fhr_geom *g, int K) { return carve_mbir(nullptr, g, K, nullptr); }

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_reconstruct_workspace_size(fhr_ctx *ctx, const fhr_geom *g, const fhr_mbir_params *p,
                                                     size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_mbir(ctx, g, p));
    FHR_ARG(bytes, "bytes is null");
    *bytes = carve_mbir(nullptr, g, p->K, nullptr);
    return FHR_OK;
}

extern "C" fhr_status fhr_reconstruct(fhr_ctx *ctx, const fhr_geom *g, const fhr_mbir_params *p, const float *sino,
                                      float *xs, void *ws, size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    return reconstruct_impl(ctx, g, p, sino, xs, ws, ws_bytes);
}
