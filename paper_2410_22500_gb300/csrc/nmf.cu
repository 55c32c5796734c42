// Subspace decomposition (Sec. III, Eq. sub_extract_solve): fast-HALS NMF.
//
// Per iteration three launches: the fused pass over P (V half-step and the
// two contractions), a deterministic FP64 reduction of the per-CTA partials,
// and the D half-step with column normalisation and the objective.  The
// column scaling of V is applied lazily by the next pass (state.wscale).
#include "nmf_internal.h"

namespace fhr {

constexpr int kUpdThreads = 64;

struct NmfWs {
    int *status;
    float *Qpart, *Gpart, *ssqpart;
    double *Q64, *GW64, *ssq64, *D64, *Bpart, *objscratch;
    unsigned int *counter;
    NmfState *state;     // [2]
};

static size_t carve_nmf(void *base, int64_t Np, int Nk, int K, int grid, int iters, NmfWs *w) {
    Carve c(base);
    NmfWs t;
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    t.counter = c.take<unsigned int>(4);
    t.state = c.take<NmfState>(2);
    t.Qpart = c.take<float>((size_t)grid * Nk * K);
    t.Gpart = c.take<float>((size_t)grid * K * K);
    t.ssqpart = c.take<float>((size_t)grid);
    t.Q64 = c.take<double>((size_t)Nk * K);
    t.GW64 = c.take<double>((size_t)K * K);
    t.ssq64 = c.take<double>(1);
    t.D64 = c.take<double>((size_t)Nk * K);
    const int nb = (int)cdiv(Nk, kUpdThreads);
    t.Bpart = c.take<double>((size_t)nb * (K + 1 + K * (K + 1) / 2));
    t.objscratch = c.take<double>((size_t)(iters > 0 ? iters : 1));
    (void)Np;
    if (w) *w = t;
    return c.size();
}

// ---------------------------------------------------------------- kernels
// GIVEN start: D64 = D0, unit state (no normalisation before the first V step).
__global__ void nmf_init_given(const float *D0, int Nk, int K, double *D64, NmfState *st) {
    __shared__ double g[kMaxK * kMaxK];
    const int tid = threadIdx.x;
    for (int i = tid; i < Nk * K; i += blockDim.x) D64[i] = (double)D0[i];
    // G = D0^T D0: thread (pair, slice) partial dot products, fixed order
    const int npair = K * K;
    const int nsl = blockDim.x / npair;   // >= 1 since blockDim >= 64 >= K*K
    __shared__ double part[256];
    const int pair = tid % npair, sl = tid / npair;
    double acc = 0.0;
    if (sl < nsl) {
        const int s = pair / K, t = pair % K;
        for (int k = sl; k < Nk; k += nsl) acc += (double)D0[k * K + s] * (double)D0[k * K + t];
    }
    part[tid] = acc;
    __syncthreads();
    if (tid < npair) {
        double a = 0.0;
        for (int j = 0; j < nsl; ++j) a += part[j * npair + tid];
        g[tid] = a;
    }
    __syncthreads();
    if (tid < kMaxK * kMaxK) {
        const int s = tid / kMaxK, t = tid % kMaxK;
        st->G[tid] = (s < K && t < K) ? (float)g[s * K + t] : 0.f;
    }
    if (tid < kMaxK) {
        st->invn[tid] = 1.0;
        st->wscale[tid] = 1.f;
        const double d = tid < K ? g[tid * K + tid] : 0.0;
        st->Gdiag[tid] = (float)d;
        st->invdiag[tid] = d != 0.0 ? (float)(1.0 / d) : 0.f;
    }
}

// Q64[k][s] = sum over CTAs of Qpart (FP64, fixed order).  The last block also
// reduces the K x K Gram partials and ||P||^2.
__global__ void nmf_reduce(const float *Qpart, const float *Gpart, const float *ssqpart, int grid, int nval,
                           int K, double *Q64, double *GW64, double *ssq64, int want_ssq) {
    __shared__ double part[8][33];
    const int tid = threadIdx.x;
    const int lane = tid & 31, ch = tid >> 5;   // 8 chunks over the CTA partials
    if (blockIdx.x == gridDim.x - 1) {
        // Gram and ||P||^2: nsmall = K*K + 1 values
        const int nsmall = K * K + (want_ssq ? 1 : 0);
        for (int v0 = 0; v0 < nsmall; v0 += 32) {
            const int v = v0 + lane;
            double acc = 0.0;
            if (v < nsmall)
                for (int g = ch; g < grid; g += 8)
                    acc += (double)(v < K * K ? Gpart[(size_t)g * K * K + v] : ssqpart[g]);
            part[ch][lane] = acc;
            __syncthreads();
            if (ch == 0 && v < nsmall) {
                double a = 0.0;
                for (int j = 0; j < 8; ++j) a += part[j][lane];
                if (v < K * K) GW64[v] = a;
                else *ssq64 = a;
            }
            __syncthreads();
        }
        return;
    }
    const int v = blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (v < nval)
        for (int g = ch; g < grid; g += 8) acc += (double)Qpart[(size_t)g * nval + v];
    part[ch][lane] = acc;
    __syncthreads();
    if (ch == 0 && v < nval) {
        double a = 0.0;
        for (int j = 0; j < 8; ++j) a += part[j][lane];
        Q64[v] = a;
    }
}

// D half-step of fast HALS for bin k (one thread per bin), FP64:
//   d_ks <- max(0, d_ks + (Q_ks - sum_t d_kt GW_ts) / GW_ss)
// then the last block normalises the columns, evaluates the objective and
// publishes the state for the next pass.  Per-bin contributions to the column
// norms, <D, Q> and D^T D (upper triangle) are summed in fixed order: through
// shared memory inside a block, over blocks in the last block.
constexpr int kUpdNV = kMaxK + 1 + kMaxK * (kMaxK + 1) / 2;   // values reduced per bin (max)

__global__ void nmf_update_d(const double *Q64, const double *GW64, const double *ssq64, double *D64, int Nk,
                             int K, const NmfState *st_in, NmfState *st_out, double *Bpart,
                             unsigned int *counter, double *obj, int *status) {
    __shared__ double gw[kMaxK * kMaxK];
    __shared__ double invh[kMaxK];
    __shared__ double vals[kUpdThreads][kUpdNV + 1];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int k = blockIdx.x * blockDim.x + tid;
    const int nv = K + 1 + K * (K + 1) / 2;
    if (tid < K * K) gw[tid] = GW64[tid];
    __syncthreads();
    if (tid < K) invh[tid] = gw[tid * K + tid] != 0.0 ? 1.0 / gw[tid * K + tid] : 0.0;
    __syncthreads();
    double d[kMaxK], q[kMaxK];
#pragma unroll
    for (int s = 0; s < kMaxK; ++s) d[s] = q[s] = 0.0;
    if (k < Nk) {
        for (int s = 0; s < K; ++s) {
            d[s] = D64[(size_t)k * K + s] * st_in->invn[s];
            q[s] = Q64[(size_t)k * K + s];
        }
        for (int s = 0; s < K; ++s) {
            if (invh[s] == 0.0) continue;
            double g = q[s];
            for (int t = 0; t < K; ++t) g -= d[t] * gw[t * K + s];
            d[s] = fmax(0.0, d[s] + g * invh[s]);
        }
        for (int s = 0; s < K; ++s) D64[(size_t)k * K + s] = d[s];
    }
    // this bin's contributions: d_s^2 (K), <d, q> (1), d_s d_t for t >= s
    {
        double *v = vals[tid];
        double dq = 0.0;
        for (int s = 0; s < K; ++s) {
            v[s] = d[s] * d[s];
            dq += d[s] * q[s];
        }
        v[K] = dq;
        int o = K + 1;
        for (int s = 0; s < K; ++s)
            for (int t = s; t < K; ++t) v[o++] = d[s] * d[t];
    }
    __syncthreads();
    if (tid < nv) {
        double a = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) a += vals[i][tid];
        Bpart[(size_t)blockIdx.x * nv + tid] = a;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double tot[kUpdNV];
    if (tid < nv) {
        double a = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) a += Bpart[(size_t)b * nv + tid];
        tot[tid] = a;
    }
    __syncthreads();
    // The state from the totals, one thread per entry (an FP64 warp instruction
    // costs about the same with one active lane as with 32, so no serial chains).
    __shared__ double sdtd[kMaxK * kMaxK], sinvn[kMaxK];
    if (tid < K * K) {   // D^T D from the packed upper triangle
        const int s = tid / K, t = tid % K;
        const int lo = s < t ? s : t, hi = s < t ? t : s;
        sdtd[tid] = tot[K + 1 + lo * K - lo * (lo - 1) / 2 + (hi - lo)];
    }
    if (tid < kMaxK) {   // column norms: D is normalised, V scaled by the norms
        const double n = tid < K ? sqrt(tot[tid]) : 0.0;
        const double in = n > 0.0 ? 1.0 / n : 1.0;
        sinvn[tid] = in;
        st_out->invn[tid] = in;
        st_out->wscale[tid] = n > 0.0 ? (float)n : 1.f;
    }
    __syncthreads();
    if (tid < kMaxK * kMaxK) {   // Gram of the normalised D for the next pass
        const int s = tid / kMaxK, t = tid % kMaxK;
        const double gd = (s < K && t < K) ? sdtd[s * K + t] * sinvn[s] * sinvn[t] : 0.0;
        st_out->G[tid] = (float)gd;
        if (s == t) {
            st_out->Gdiag[s] = (float)gd;
            st_out->invdiag[s] = gd != 0.0 ? (float)(1.0 / gd) : 0.f;
        }
    }
    if (tid < 32) {   // objective ||P||^2 - 2 <D, Q> + <D^T D, G_W>, fixed-order tree
        double v = 0.0;
        for (int i = tid; i < K * K; i += 32) v += sdtd[i] * gw[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tid == 0) {
            const double f = *ssq64 - 2.0 * tot[K] + v;
            *obj = f;
            if (!isfinite(f)) report(status, FHR_ERR_NONFINITE);
            *counter = 0u;
        }
    }
}

// Learned start: D0 from `sweeps` HALS D half-steps from D = 0 with Q = P^T W0
// and G_W = W0^T W0 fixed (no further passes over P).  One thread per bin.
__global__ void nmf_d_from_q(const double *Q64, const double *GW64, int Nk, int K, int sweeps, float *D) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nk) return;
    double d[kMaxK], q[kMaxK], gw[kMaxK * kMaxK];
    for (int s = 0; s < K; ++s) {
        d[s] = 0.0;
        q[s] = Q64[(size_t)k * K + s];
    }
    for (int i = 0; i < K * K; ++i) gw[i] = GW64[i];
    for (int it = 0; it < sweeps; ++it)
        for (int s = 0; s < K; ++s) {
            const double h = gw[s * K + s];
            if (h == 0.0) continue;
            double g = q[s];
            for (int t = 0; t < K; ++t) g -= d[t] * gw[t * K + s];
            d[s] = fmax(0.0, d[s] + g / h);
        }
    for (int s = 0; s < K; ++s) D[(size_t)k * K + s] = (float)d[s];
}

// Final outputs: D = D64 * invn, W *= wscale.
__global__ void nmf_finalize(const double *D64, const NmfState *st, int Nk, int K, float *D, float *W, int64_t Np) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0; i < (int64_t)Nk * K; i += stride) D[i] = (float)(D64[i] * st->invn[i % K]);
    for (int64_t i = i0; i < Np * K; i += stride) W[i] *= st->wscale[i % K];
}

// ---------------------------------------------------------------- host
fhr_status cluster_check(fhr_ctx *ctx, const fhr_nmf_params *p);

static fhr_status check_nmf(fhr_ctx *ctx, const fhr_nmf_params *p) {
    FHR_ARG(p, "params is null");
    FHR_ARG(p->Np > 0 && p->Nk > 0, "Np and Nk must be positive");
    FHR_ARG(p->K >= 1 && p->K <= kMaxK, "K must be 1..8");
    FHR_ARG(p->ldP >= p->Nk, "ldP < Nk");
    FHR_ARG(p->p_dtype == FHR_F32 || p->p_dtype == FHR_BF16, "bad p_dtype");
    FHR_ARG(p->ldP % (p->p_dtype == FHR_BF16 ? 8 : 4) == 0, "ldP must be a multiple of 16 bytes");
    FHR_ARG(p->iters >= 0, "iters < 0");
    FHR_ARG(p->K <= p->Nk && (int64_t)p->K <= p->Np, "K > min(Nk, Np)");
    if (p->init != FHR_INIT_GIVEN && p->init != FHR_INIT_NNDSVD && p->init != FHR_INIT_LEARNED &&
        p->init != FHR_INIT_CLUSTER)
        return set_error(ctx, FHR_ERR_ARG, "unknown init %d", p->init);
    if (p->init == FHR_INIT_CLUSTER) FHR_TRY(cluster_check(ctx, p));
    if (p->init == FHR_INIT_LEARNED) {
        FHR_ARG(p->mlp && p->mlp_params, "FHR_INIT_LEARNED needs mlp and mlp_params");
        FHR_ARG(p->mlp->K == p->K && p->mlp->Nk == p->Nk && p->mlp->ldx == p->ldP && p->mlp->x_dtype == p->p_dtype,
                "the warm-start network does not match the problem (K, Nk, ldP, p_dtype)");
    }
    return FHR_OK;
}

fhr_status nndsvd_ws_size(fhr_ctx *ctx, const fhr_nmf_params *p, size_t *bytes);
size_t cluster_ws_bytes(const fhr_nmf_params *p);
fhr_status cluster_run(fhr_ctx *ctx, const fhr_nmf_params *p, const void *P, float *D, void *region);
size_t mlp_ws_bytes(const fhr_mlp_dims *d, int train);
fhr_status mlp_forward_impl(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *prm, int64_t M, const void *X, float *Y,
                            void *ws, size_t ws_bytes);
fhr_status nndsvd_run(fhr_ctx *ctx, const fhr_nmf_params *p, const void *P, float *D, float *W, void *region,
                      int *status);

// Total decomposition workspace: the iteration buffers, then the
// initialisation's own region (NNDSVD, clustering or learned start).
static fhr_status decompose_ws(fhr_ctx *ctx, const fhr_nmf_params *p, const PassConfig &cfg, void *base, NmfWs *w,
                               size_t *total, void **nn_region) {
    size_t a = carve_nmf(base, p->Np, p->Nk, p->K, cfg.grid, p->iters, w);
    size_t b = 0;
    if (p->init == FHR_INIT_NNDSVD) FHR_TRY(nndsvd_ws_size(ctx, p, &b));
    if (p->init == FHR_INIT_LEARNED) b = mlp_ws_bytes(p->mlp, 0);
    if (p->init == FHR_INIT_CLUSTER) b = cluster_ws_bytes(p);
    if (nn_region) *nn_region = base ? (void *)((char *)base + a) : nullptr;
    *total = a + b;
    return FHR_OK;
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_decompose_workspace_size(fhr_ctx *ctx, const fhr_nmf_params *p, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_nmf(ctx, p));
    FHR_ARG(bytes, "bytes is null");
    FHR_CUDA(cudaSetDevice(ctx->device));
    PassConfig cfg;
    FHR_TRY(pass_config(ctx, p->K, p->Nk, p->ldP, p->p_dtype, &cfg));
    return decompose_ws(ctx, p, cfg, nullptr, nullptr, bytes, nullptr);
}

extern "C" fhr_status fhr_decompose(fhr_ctx *ctx, const fhr_nmf_params *p, const void *P, float *D, float *W,
                                    double *obj, void *ws, size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_nmf(ctx, p));
    FHR_ARG(P && D && W && ws, "null pointer argument");
    FHR_ARG(aligned(P, 16) && aligned(W, 16), "P and W must be 16-byte aligned");
    FHR_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
    FHR_CUDA(cudaSetDevice(ctx->device));
    PassConfig cfg;
    FHR_TRY(pass_config(ctx, p->K, p->Nk, p->ldP, p->p_dtype, &cfg));
    NmfWs w;
    size_t need = 0;
    void *nn_region = nullptr;
    FHR_TRY(decompose_ws(ctx, p, cfg, ws, &w, &need, &nn_region));
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    cudaStream_t st = ctx->stream;
    FHR_CUDA(cudaMemsetAsync(w.status, 0, kStatusBytes, st));
    FHR_CUDA(cudaMemsetAsync(w.counter, 0, 4 * sizeof(unsigned int), st));
    const int K = p->K, Nk = p->Nk;

    if (p->init == FHR_INIT_NNDSVD) FHR_TRY(nndsvd_run(ctx, p, P, D, W, nn_region, w.status));
    PassArgs a;
    if (p->init == FHR_INIT_LEARNED) {
        FHR_TRY(mlp_forward_impl(ctx, p->mlp, p->mlp_params, p->Np, P, W, nn_region, mlp_ws_bytes(p->mlp, 0)));
        // unit state, then one pass with W0 fixed for Q = P^T W0, G_W = W0^T W0
        nmf_init_given<<<1, 256, 0, st>>>(D, Nk, K, w.D64, &w.state[0]);
        FHR_LAUNCHED();
        a.P = P; a.Np = p->Np; a.Nk = Nk; a.ldP = p->ldP; a.D64 = w.D64; a.st = &w.state[0]; a.W = W;
        a.Qpart = w.Qpart; a.Gpart = w.Gpart; a.ssqpart = w.ssqpart; a.status = w.status;
        a.mode = PASS_GIVEN_W; a.want_ssq = 0;
        FHR_TRY(launch_pass(ctx, cfg, a));
        nmf_reduce<<<(unsigned)cdiv(Nk * K, 32) + 1, 256, 0, st>>>(w.Qpart, w.Gpart, w.ssqpart, cfg.grid, Nk * K, K,
                                                                    w.Q64, w.GW64, w.ssq64, 0);
        FHR_LAUNCHED();
        nmf_d_from_q<<<(unsigned)cdiv(Nk, 128), 128, 0, st>>>(w.Q64, w.GW64, Nk, K, 10, D);
        FHR_LAUNCHED();
    }
    if (p->init == FHR_INIT_CLUSTER) {
        // D0 = k-means centres; W0 = one HALS V half-step from V = 0
        FHR_TRY(cluster_run(ctx, p, P, D, nn_region));
        FHR_CUDA(cudaMemsetAsync(W, 0, sizeof(float) * (size_t)p->Np * K, st));
        nmf_init_given<<<1, 256, 0, st>>>(D, Nk, K, w.D64, &w.state[0]);
        FHR_LAUNCHED();
        a.P = P; a.Np = p->Np; a.Nk = Nk; a.ldP = p->ldP; a.D64 = w.D64; a.st = &w.state[0]; a.W = W;
        a.Qpart = w.Qpart; a.Gpart = w.Gpart; a.ssqpart = w.ssqpart; a.status = w.status;
        a.mode = PASS_HALS; a.want_ssq = 0;
        FHR_TRY(launch_pass(ctx, cfg, a));
    }
    nmf_init_given<<<1, 256, 0, st>>>(D, Nk, K, w.D64, &w.state[0]);
    FHR_LAUNCHED();

    a.P = P;
    a.Np = p->Np;
    a.Nk = Nk;
    a.ldP = p->ldP;
    a.D64 = w.D64;
    a.W = W;
    a.Qpart = w.Qpart;
    a.Gpart = w.Gpart;
    a.ssqpart = w.ssqpart;
    a.status = w.status;
    a.mode = PASS_HALS;
    a.want_ssq = 1;
    const int nval = Nk * K;
    const int nred = (int)cdiv(nval, 32) + 1;
    const int nupd = (int)cdiv(Nk, kUpdThreads);
    for (int t = 0; t < p->iters; ++t) {
        a.st = &w.state[t & 1];
        a.want_ssq = t == 0;   // ||P||^2 once; later iterations reuse it
        FHR_TRY(launch_pass(ctx, cfg, a));
        FHR_TIMED(TM_NMF_REDUCE, (nmf_reduce<<<nred, 256, 0, st>>>(w.Qpart, w.Gpart, w.ssqpart, cfg.grid, nval, K,
                                                                   w.Q64, w.GW64, w.ssq64, a.want_ssq)));
        FHR_TIMED(TM_NMF_UPDATE,
                  (nmf_update_d<<<nupd, kUpdThreads, 0, st>>>(w.Q64, w.GW64, w.ssq64, w.D64, Nk, K, &w.state[t & 1],
                                                              &w.state[(t + 1) & 1], w.Bpart, w.counter,
                                                              obj ? obj + t : w.objscratch + t, w.status)));
    }
    nmf_finalize<<<ctx->sm_count * 4, 256, 0, st>>>(w.D64, &w.state[p->iters & 1], Nk, K, D, W, p->Np);
    FHR_LAUNCHED();
    return FHR_OK;
}
