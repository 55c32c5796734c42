// Clustering start for the NMF (the library's added "clustering-initialised"
// mode; Sec. III itself starts from NNDSVD).  On a strided pixel sample:
// k-means++ seeding drawn from splitmix64 uniforms, a fixed number of Lloyd
// iterations, then D0 = the centres.  Distances, running sums and means are
// FP64, so the assignment decisions are those of an FP64 evaluation up to
// summation order.  All reductions run in a fixed order.
#include <cuda_bf16.h>

#include "nmf_internal.h"

namespace fhr {

constexpr int kKmChunks = 64;       // sample chunks of the centre sums
constexpr int kKmAccThreads = 128;
constexpr int kKmPickThreads = 1024;
constexpr int64_t kKmMaxSamples = 1 << 20;
constexpr int64_t kKmDefaultSamples = 32768;
constexpr int kKmDefaultIters = 20;

template <typename T>
__device__ __forceinline__ double ld64(const T *p);
template <>
__device__ __forceinline__ double ld64<float>(const float *p) { return (double)__ldg(p); }
template <>
__device__ __forceinline__ double ld64<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return (double)__bfloat162float(*p);
}

// sample i -> pixel floor(i * Np / S); i < S <= 2^20 and Np < 2^40 keep the product in range
__device__ __forceinline__ int64_t km_row(int64_t i, int64_t Np, int64_t S) {
    return (int64_t)(((uint64_t)i * (uint64_t)Np) / (uint64_t)S);
}

__device__ __forceinline__ double warp_sum64(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// dmin[i] = min(dmin[i], |x_i - c|^2) (first: = |x_i - c|^2); one warp per sample
template <typename T>
__global__ void km_dist(const T *P, int64_t Np, int ldP, int Nk, int64_t S, const double *c, double *dmin,
                        int first) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < S; i += nw) {
        const T *x = P + km_row(i, Np, S) * ldP;
        double s = 0.0;
        for (int k = lane; k < Nk; k += 32) {
            const double d = ld64(x + k) - c[k];
            s = fma(d, d, s);
        }
        s = warp_sum64(s);
        if (lane == 0) dmin[i] = (first || s < dmin[i]) ? s : dmin[i];
    }
}

// Seed m: m = 0 -> sample floor(u S); else the first sample whose running sum
// of dmin exceeds u * sum(dmin).  Copies that sample into C[m].
template <typename T>
__global__ void __launch_bounds__(kKmPickThreads) km_pick(const double *dmin, int64_t S, double u, int m,
                                                          const T *P, int64_t Np, int ldP, int Nk, double *C) {
    __shared__ double csum[kKmPickThreads];
    __shared__ int64_t pick;
    const int tid = threadIdx.x;
    const int64_t per = (S + kKmPickThreads - 1) / kKmPickThreads;
    if (m > 0) {
        const int64_t lo = min(S, (int64_t)tid * per), hi = min(S, lo + per);
        double a = 0.0;
        for (int64_t i = lo; i < hi; ++i) a += dmin[i];
        csum[tid] = a;
    }
    __syncthreads();
    if (tid == 0) {
        int64_t pk = (int64_t)(u * (double)S);
        if (m > 0) {
            double tot = 0.0;
            for (int t = 0; t < kKmPickThreads; ++t) tot += csum[t];
            if (tot > 0.0) {
                const double target = u * tot;
                double run = 0.0;
                pk = -1;
                for (int t = 0; t < kKmPickThreads && pk < 0; ++t) {
                    if (run + csum[t] > target) {
                        const int64_t lo = min(S, (int64_t)t * per), hi = min(S, lo + per);
                        for (int64_t i = lo; i < hi; ++i) {
                            run += dmin[i];
                            if (run > target) {
                                pk = i;
                                break;
                            }
                        }
                    } else {
                        run += csum[t];
                    }
                }
                if (pk < 0)   // rounding: the last sample with a positive distance
                    for (int64_t i = S - 1; i >= 0; --i)
                        if (dmin[i] > 0.0) {
                            pk = i;
                            break;
                        }
            }
        }
        pick = pk < 0 ? 0 : (pk >= S ? S - 1 : pk);
    }
    __syncthreads();
    const T *x = P + km_row(pick, Np, S) * ldP;
    for (int k = tid; k < Nk; k += kKmPickThreads) C[(size_t)m * Nk + k] = ld64(x + k);
}

// lab[i] = argmin_m |x_i - C[m]|^2 (lowest m on ties); one warp per sample
template <typename T>
__global__ void km_assign(const T *P, int64_t Np, int ldP, int Nk, int64_t S, int K, const double *C, int *lab) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < S; i += nw) {
        const T *x = P + km_row(i, Np, S) * ldP;
        double s[kMaxK];
#pragma unroll
        for (int m = 0; m < kMaxK; ++m) s[m] = 0.0;
        for (int k = lane; k < Nk; k += 32) {
            const double xv = ld64(x + k);
#pragma unroll
            for (int m = 0; m < kMaxK; ++m)
                if (m < K) {
                    const double d = xv - C[(size_t)m * Nk + k];
                    s[m] = fma(d, d, s[m]);
                }
        }
        int best = 0;
        double bd = 0.0;
#pragma unroll
        for (int m = 0; m < kMaxK; ++m)
            if (m < K) {
                const double v = warp_sum64(s[m]);
                if (m == 0 || v < bd) {
                    bd = v;
                    best = m;
                }
            }
        if (lane == 0) lab[i] = best;
    }
}

// Per-chunk centre sums: part[chunk][m][k] = sum of x_i[k] over the chunk's
// samples with label m (in sample order); cnt[chunk][m] their count.
template <typename T>
__global__ void __launch_bounds__(kKmAccThreads) km_accum(const T *P, int64_t Np, int ldP, int Nk, int64_t S, int K,
                                                          const int *lab, double *part, long long *cnt) {
    const int k = blockIdx.x * kKmAccThreads + threadIdx.x;
    const int chunk = blockIdx.y;
    const int64_t per = (S + kKmChunks - 1) / kKmChunks;
    const int64_t lo = min(S, (int64_t)chunk * per), hi = min(S, lo + per);
    const bool counter = blockIdx.x == 0 && threadIdx.x == 0;
    double acc[kMaxK];
    long long c[kMaxK];
#pragma unroll
    for (int m = 0; m < kMaxK; ++m) {
        acc[m] = 0.0;
        c[m] = 0;
    }
    for (int64_t i = lo; i < hi; ++i) {
        const int l = lab[i];
        const double x = k < Nk ? ld64(P + km_row(i, Np, S) * ldP + k) : 0.0;
#pragma unroll
        for (int m = 0; m < kMaxK; ++m)
            if (m == l) {
                acc[m] += x;
                c[m] += 1;
            }
    }
    for (int m = 0; m < K; ++m) {
        if (k < Nk) part[((size_t)chunk * K + m) * Nk + k] = acc[m];
        if (counter) cnt[chunk * K + m] = c[m];
    }
}

// C[m][k] = (sum over chunks) / count, unchanged for an empty cluster
__global__ void km_update(const double *part, const long long *cnt, int K, int Nk, double *C) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * Nk) return;
    const int m = idx / Nk, k = idx % Nk;
    long long n = 0;
    double s = 0.0;
    for (int ch = 0; ch < kKmChunks; ++ch) {
        n += cnt[ch * K + m];
        s += part[((size_t)ch * K + m) * Nk + k];
    }
    if (n > 0) C[idx] = s / (double)n;
}

__global__ void km_to_d(const double *C, int K, int Nk, float *D) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * Nk) return;
    const int k = idx / K, m = idx % K;
    D[idx] = (float)C[(size_t)m * Nk + k];
}

// ---------------------------------------------------------------- host
static uint64_t splitmix64_host(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int64_t km_samples(const fhr_nmf_params *p) {
    const int64_t want = p->kmeans_samples > 0 ? p->kmeans_samples : kKmDefaultSamples;
    return std::min<int64_t>(p->Np, want);
}

struct KmWs {
    double *C, *dmin, *part;
    int *lab;
    long long *cnt;
};

static size_t carve_km(void *base, int64_t S, int K, int Nk, KmWs *w) {
    Carve c(base);
    KmWs t;
    t.C = c.take<double>((size_t)K * Nk);
    t.dmin = c.take<double>((size_t)S);
    t.lab = c.take<int>((size_t)S);
    t.part = c.take<double>((size_t)kKmChunks * K * Nk);
    t.cnt = c.take<long long>((size_t)kKmChunks * K);
    if (w) *w = t;
    return c.size();
}

fhr_status cluster_check(fhr_ctx *ctx, const fhr_nmf_params *p) {
    FHR_ARG(p->kmeans_samples >= 0 && p->kmeans_samples <= kKmMaxSamples, "kmeans_samples must be 0..%lld",
            (long long)kKmMaxSamples);
    FHR_ARG(p->kmeans_iters >= 0, "kmeans_iters < 0");
    FHR_ARG(km_samples(p) >= p->K, "fewer pixel samples than clusters");
    FHR_ARG(p->Np < ((int64_t)1 << 40), "Np too large for the clustering start");
    return FHR_OK;
}

size_t cluster_ws_bytes(const fhr_nmf_params *p) { return carve_km(nullptr, km_samples(p), p->K, p->Nk, nullptr); }

template <typename T>
static fhr_status cluster_run_t(fhr_ctx *ctx, const fhr_nmf_params *p, const T *P, float *D, void *region) {
    const int64_t S = km_samples(p);
    const int K = p->K, Nk = p->Nk, ldP = p->ldP;
    const int64_t Np = p->Np;
    const int iters = p->kmeans_iters > 0 ? p->kmeans_iters : kKmDefaultIters;
    KmWs w;
    carve_km(region, S, K, Nk, &w);
    cudaStream_t st = ctx->stream;
    const unsigned wgrid = (unsigned)std::min<int64_t>(cdiv(S, 8), (int64_t)ctx->sm_count * 8);
    uint64_t state = p->seed;
    for (int m = 0; m < K; ++m) {
        const double u = (double)(splitmix64_host(&state) >> 11) * 0x1.0p-53;
        if (m > 0) {
            km_dist<T><<<wgrid, 256, 0, st>>>(P, Np, ldP, Nk, S, w.C + (size_t)(m - 1) * Nk, w.dmin, m == 1);
            FHR_LAUNCHED();
        }
        km_pick<T><<<1, kKmPickThreads, 0, st>>>(w.dmin, S, u, m, P, Np, ldP, Nk, w.C);
        FHR_LAUNCHED();
    }
    const dim3 agrid((unsigned)cdiv(Nk, kKmAccThreads), kKmChunks);
    const unsigned ugrid = (unsigned)cdiv(K * Nk, 256);
    for (int it = 0; it < iters; ++it) {
        km_assign<T><<<wgrid, 256, 0, st>>>(P, Np, ldP, Nk, S, K, w.C, w.lab);
        FHR_LAUNCHED();
        km_accum<T><<<agrid, kKmAccThreads, 0, st>>>(P, Np, ldP, Nk, S, K, w.lab, w.part, w.cnt);
        FHR_LAUNCHED();
        km_update<<<ugrid, 256, 0, st>>>(w.part, w.cnt, K, Nk, w.C);
        FHR_LAUNCHED();
    }
    km_to_d<<<ugrid, 256, 0, st>>>(w.C, K, Nk, D);
    FHR_LAUNCHED();
    return FHR_OK;
}

fhr_status cluster_run(fhr_ctx *ctx, const fhr_nmf_params *p, const void *P, float *D, void *region) {
    if (p->p_dtype == FHR_BF16)
        return cluster_run_t(ctx, p, static_cast<const __nv_bfloat16 *>(P), D, region);
    return cluster_run_t(ctx, p, static_cast<const float *>(P), D, region);
}

}  // namespace fhr
