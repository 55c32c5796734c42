// Learned warm start: a 3-layer MLP (Nk -> H1 -> H2 -> K, GELU, GELU,
// softplus) mapping a pixel's spectrum to K nonnegative subspace
// coefficients, with hand-written forward, backward and AdamW kernels.
// Not in the paper: an added form that starts the fast-HALS iterations of
// Sec. III closer to their end point.
//
// Every layer is one tiled GEMM with a fused epilogue (bias + activation, or
// the activation's derivative); weight gradients are split-K GEMMs over the
// pixel dimension with a fixed-order reduction of the splits.  Arithmetic is
// FP32 (FP32 accumulation); with weights_bf16 the weights and the hidden
// activations that feed the next layer are rounded to bf16.
#include <math.h>

#include "common.cuh"
#include "mlp_tc.h"

namespace fhr {

enum GemmEpi { EPI_STORE = 0, EPI_BIAS_GELU, EPI_BIAS_SOFTPLUS, EPI_GELU_BACK };

struct GemmArgs {
    int M, N, Kd;
    const void *A;
    int64_t sai, sak;   // A(i, k) = A[i * sai + k * sak]
    const void *B;
    int64_t sbk, sbj;   // B(k, j) = B[k * sbk + j * sbj]
    float *C;           // C[i * ldc + j] (+ split * split_stride)
    int64_t ldc, split_stride;
    void *C2;           // activation output (EPI_BIAS_GELU), f32 or bf16
    int c2_bf16;
    int64_t ldc2;
    const float *bias;
    const float *Z;     // pre-activation for EPI_GELU_BACK
    int64_t ldz;
    int kchunk;         // contraction range per grid.z slice
};

template <typename T>
__device__ __forceinline__ float ld_as_f32(const void *p, int64_t i);
template <>
__device__ __forceinline__ float ld_as_f32<float>(const void *p, int64_t i) {
    return __ldg(reinterpret_cast<const float *>(p) + i);
}
template <>
__device__ __forceinline__ float ld_as_f32<__nv_bfloat16>(const void *p, int64_t i) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d_f(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}
__device__ __forceinline__ float softplus_f(float z) { return z > 20.f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigmoid_f(float z) { return 1.f / (1.f + expf(-z)); }

constexpr int GBM = 64, GBN = 64, GBK = 16;

template <typename TA, typename TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
    __shared__ __align__(16) float As[GBK][GBM];
    __shared__ __align__(16) float Bs[GBK][GBN];
    const int tid = threadIdx.x;
    const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
    const int kbeg = blockIdx.z * g.kchunk;
    const int kend = min(g.Kd, kbeg + g.kchunk);
    const int ty = tid / 16, tx = tid % 16;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const bool a_kfast = g.sak == 1;
    const bool b_jfast = g.sbj == 1;
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int i, k;
            if (a_kfast) {
                i = tid / 4;
                k = (tid % 4) * 4 + e;
            } else {
                k = tid / 16;
                i = (tid % 16) * 4 + e;
            }
            const int gi = i0 + i, gk = k0 + k;
            As[k][i] = (gi < g.M && gk < kend) ? ld_as_f32<TA>(g.A, (int64_t)gi * g.sai + (int64_t)gk * g.sak) : 0.f;
            int j, kb;
            if (b_jfast) {
                kb = tid / 16;
                j = (tid % 16) * 4 + e;
            } else {
                j = tid / 4;
                kb = (tid % 4) * 4 + e;
            }
            const int gj = j0 + j, gkb = k0 + kb;
            Bs[kb][j] = (gj < g.N && gkb < kend) ? ld_as_f32<TB>(g.B, (int64_t)gkb * g.sbk + (int64_t)gj * g.sbj) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GBK; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = i0 + ty * 4 + p;
        if (i >= g.M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx * 4 + q;
            if (j >= g.N) continue;
            float v = acc[p][q];
            if (EPI == EPI_STORE) {
                g.C[(int64_t)blockIdx.z * g.split_stride + (int64_t)i * g.ldc + j] = v;
            } else if (EPI == EPI_BIAS_GELU) {
                v += g.bias[j];
                if (g.C) g.C[(int64_t)i * g.ldc + j] = v;
                const float a = gelu_f(v);
                if (g.c2_bf16)
                    reinterpret_cast<__nv_bfloat16 *>(g.C2)[(int64_t)i * g.ldc2 + j] = __float2bfloat16_rn(a);
                else
                    reinterpret_cast<float *>(g.C2)[(int64_t)i * g.ldc2 + j] = a;
            } else if (EPI == EPI_BIAS_SOFTPLUS) {
                v += g.bias[j];
                if (g.C2) reinterpret_cast<float *>(g.C2)[(int64_t)i * g.ldc2 + j] = v;
                g.C[(int64_t)i * g.ldc + j] = softplus_f(v);
            } else {   // EPI_GELU_BACK: dZ = (dA) * gelu'(Z)
                g.C[(int64_t)i * g.ldc + j] = v * gelu_d_f(g.Z[(int64_t)i * g.ldz + j]);
            }
        }
    }
}

// Layers 1 and 2 with bf16 inputs and bf16 weights on the tensor cores (warp
// MMA m16n8k16, FP32 accumulation): Act = GELU(A B^T + bias) in bf16 and,
// when Z is set, the FP32 pre-activation.  A [M][Kd] (row stride lda) and
// B [N][Kd] (row stride ldb) are both k-contiguous; 128 x 128 tiles, k-steps
// of 32 through a 4-stage cp.async ring (rows of 64 bytes, 16-byte chunks
// XOR-swizzled by row so that ldmatrix reads are free of bank conflicts);
// 8 warps as 2 x 4, a 64 x 32 tile each.  Columns past Kd read as zeros
// (cp.async zero-fills the part of a chunk beyond its source size).
constexpr int MBM = 128, MBN = 128, MBK = 32, MST = 4;
constexpr int kMmaStageBytes = (MBM + MBN) * MBK * 2;
constexpr int kMmaSmem = MST * kMmaStageBytes;

struct MmaGemmArgs {
    int M, N, Kd;
    const __nv_bfloat16 *A;
    int64_t lda;
    const __nv_bfloat16 *B;
    int64_t ldb;
    const float *bias;
    float *Z;                 // optional pre-activation [M][ldz]
    int64_t ldz;
    __nv_bfloat16 *Act;       // GELU(Z) [M][ldact]
    int64_t ldact;
};

__device__ __forceinline__ void mlp_cp16(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void mlp_ldsm4(uint32_t a, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void mlp_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                 "{%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// byte offset of 16-byte chunk c (0..3) of tile row r
__device__ __forceinline__ uint32_t mlp_swz(int r, int c) { return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4)); }

__global__ void __launch_bounds__(256, 2) mlp_gemm_mma(MmaGemmArgs g) {
    extern __shared__ __align__(128) unsigned char mlp_sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int64_t m0 = (int64_t)blockIdx.y * MBM;
    const int n0 = blockIdx.x * MBN;
    const int nk = (g.Kd + MBK - 1) / MBK;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(mlp_sm);

    auto load = [&](int kt, int st) {
        const uint32_t sa = sbase + st * kMmaStageBytes, sb = sa + MBM * MBK * 2;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int idx = tid + e * 256;
            const int r = idx >> 2, c = idx & 3;
            const int k = kt * MBK + c * 8;
            const int kb = min(16, max(0, (g.Kd - k) * 2));
            const int64_t ga = m0 + r;
            const bool ra = ga < g.M && kb > 0;
            mlp_cp16(sa + mlp_swz(r, c), g.A + (ra ? ga * g.lda + k : 0), ra ? kb : 0);
            const int gb = n0 + r;
            const bool rb = gb < g.N && kb > 0;
            mlp_cp16(sb + mlp_swz(r, c), g.B + (rb ? (int64_t)gb * g.ldb + k : 0), rb ? kb : 0);
        }
    };

    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

#pragma unroll
    for (int st = 0; st < MST - 1; ++st) {
        if (st < nk) load(st, st);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int kt = 0; kt < nk; ++kt) {
        asm volatile("cp.async.wait_group %0;" ::"n"(MST - 2) : "memory");
        __syncthreads();
        if (kt + MST - 1 < nk) load(kt + MST - 1, (kt + MST - 1) % MST);
        asm volatile("cp.async.commit_group;" ::: "memory");
        const uint32_t sa = sbase + (kt % MST) * kMmaStageBytes, sb = sa + MBM * MBK * 2;
#pragma unroll
        for (int kk = 0; kk < MBK / 16; ++kk) {
            uint32_t af[4][4], bq[2][4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
                mlp_ldsm4(sa + mlp_swz(wm * 64 + mi * 16 + (lane & 15), kk * 2 + (lane >> 4)), af[mi]);
#pragma unroll
            for (int nj = 0; nj < 2; ++nj)
                mlp_ldsm4(sb + mlp_swz(wn * 32 + nj * 16 + (lane & 7) + ((lane >> 4) << 3), kk * 2 + ((lane >> 3) & 1)),
                          bq[nj]);
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mlp_mma(acc[mi][ni], af[mi], bq[ni >> 1][(ni & 1) * 2], bq[ni >> 1][(ni & 1) * 2 + 1]);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");

    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
        const int col = n0 + wn * 32 + ni * 8 + 2 * tq;
        if (col >= g.N) continue;   // N is a multiple of 8: col + 1 < N as well
        const float b0 = g.bias[col], b1 = g.bias[col + 1];
#pragma unroll
        for (int mi = 0; mi < 4; ++mi)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t row = m0 + wm * 64 + mi * 16 + gq + 8 * h;
                if (row >= g.M) continue;
                const float z0 = acc[mi][ni][2 * h] + b0, z1 = acc[mi][ni][2 * h + 1] + b1;
                if (g.Z) *reinterpret_cast<float2 *>(g.Z + row * g.ldz + col) = make_float2(z0, z1);
                *reinterpret_cast<__nv_bfloat162 *>(g.Act + row * g.ldact + col) =
                    __floats2bfloat162_rn(gelu_f(z0), gelu_f(z1));
            }
    }
}

// bf16 copy of a [rows][cols] f32 weight block with rows padded to ld (zeros)
__global__ void pad_bf16_kernel(const float *w, int rows, int cols, int ld, __nv_bfloat16 *out) {
    const int64_t n = (int64_t)rows * ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / ld), c = (int)(i % ld);
        out[i] = __float2bfloat16_rn(c < cols ? w[(int64_t)r * cols + c] : 0.f);
    }
}

// loss partials and dZ3 = 2/(M K) (y - t) sigmoid(z3), one thread per output
__global__ void mlp_loss_kernel(const float *Y, const float *Z3, const float *T, int64_t n, float scale, float *dZ3,
                                double *part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = Y[i] - T[i];
        s += (double)e * (double)e;
        dZ3[i] = scale * e * sigmoid_f(Z3[i]);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void mlp_loss_final(const double *part, int nb, double inv_n, double *loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0;
        for (int b = 0; b < nb; ++b) a += part[b];
        *loss = a * inv_n;
    }
}

// grad[o + j] = sum over splits of partials (fixed order); bias grads = column sums of dZ
__global__ void mlp_reduce_splits(const float *part, int splits, int64_t n, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int s = 0; s < splits; ++s) a += part[(int64_t)s * n + i];
        out[i] = a;
    }
}

__global__ void mlp_colsum(const float *dZ, int64_t M, int N, float *out) {
    // one block per column chunk of 32, threads over rows; fixed-order tree
    __shared__ float sh[8][33];
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int r = threadIdx.x >> 5;
    float a = 0.f;
    if (j < N)
        for (int64_t m = r; m < M; m += 8) a += dZ[m * N + j];
    sh[r][threadIdx.x & 31] = a;
    __syncthreads();
    if (r == 0 && j < N) {
        float s = 0.f;
        for (int q = 0; q < 8; ++q) s += sh[q][threadIdx.x & 31];
        out[j] = s;
    }
}

__global__ void to_bf16_kernel(const float *x, int64_t n, __nv_bfloat16 *y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void adamw_kernel(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                             float eps, float wd, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i]);
    }
}

// ------------------------------------------------------------------ host side
struct MlpLayout {
    int64_t oW1, ob1, oW2, ob2, oW3, ob3, n;
};

static MlpLayout mlp_layout(const fhr_mlp_dims *d) {
    MlpLayout L;
    L.oW1 = 0;
    L.ob1 = L.oW1 + (int64_t)d->H1 * d->Nk;
    L.oW2 = L.ob1 + d->H1;
    L.ob2 = L.oW2 + (int64_t)d->H2 * d->H1;
    L.oW3 = L.ob2 + d->H2;
    L.ob3 = L.oW3 + (int64_t)d->K * d->H2;
    L.n = L.ob3 + d->K;
    return L;
}

constexpr int kMlpChunk = 32768;      // pixel rows per training (forward + backward) chunk
constexpr int kMlpFwdChunk = 524288;  // pixel rows per inference chunk (4096 row tiles: 27 per SM)
constexpr int kSplitRows = 2048;      // contraction rows per split of a weight gradient

struct MlpWs {
    int *status;
    __nv_bfloat16 *wb;      // bf16 weights (packed like the params) or null
    __nv_bfloat16 *wp1, *wp2;   // bf16 W1, W2 with rows padded to a multiple of 8 (tensor-core layers)
    float *Z1, *Z2, *Z3, *Y;
    void *A1, *A2;
    float *dZ3, *dZ2, *dZ1;
    float *part;            // split-K partials
    double *lpart;
    double *lacc;
};

static int64_t mlp_splits(int64_t M) { return cdiv(M, kSplitRows); }
static int pad8(int n) { return (n + 7) / 8 * 8; }

static size_t carve_mlp(void *base, const fhr_mlp_dims *d, int train, MlpWs *w) {
    const MlpLayout L = mlp_layout(d);
    const int64_t R = train ? kMlpChunk : kMlpFwdChunk;
    const int es = d->weights_bf16 ? 2 : 4;
    Carve c(base);
    MlpWs t{};
    t.status = c.take<int>(kStatusBytes / sizeof(int));
    t.wb = d->weights_bf16 ? c.take<__nv_bfloat16>((size_t)L.n) : nullptr;
    if (d->weights_bf16) {
        t.wp1 = c.take<__nv_bfloat16>((size_t)d->H1 * pad8(d->Nk));
        t.wp2 = c.take<__nv_bfloat16>((size_t)d->H2 * pad8(d->H1));
    }
    if (train) {   // pre-activations, kept for the backward pass
        t.Z1 = c.take<float>((size_t)R * d->H1);
        t.Z2 = c.take<float>((size_t)R * d->H2);
        t.Z3 = c.take<float>((size_t)R * d->K);
        t.Y = c.take<float>((size_t)R * d->K);
    }
    t.A1 = c.take<char>((size_t)R * d->H1 * es);
    t.A2 = c.take<char>((size_t)R * d->H2 * es);
    if (train) {
        t.dZ3 = c.take<float>((size_t)R * d->K);
        t.dZ2 = c.take<float>((size_t)R * d->H2);
        t.dZ1 = c.take<float>((size_t)R * d->H1);
        const int64_t big = std::max<int64_t>((int64_t)d->H1 * d->Nk, (int64_t)d->H2 * d->H1);
        t.part = c.take<float>((size_t)mlp_splits(R) * big);
        t.lpart = c.take<double>(1024);
        t.lacc = c.take<double>(1);
    }
    if (w) *w = t;
    return c.size();
}

static fhr_status check_dims(fhr_ctx *ctx, const fhr_mlp_dims *d) {
    FHR_ARG(d, "dims is null");
    FHR_ARG(d->Nk > 0 && d->H1 > 0 && d->H2 > 0 && d->K >= 1 && d->K <= 64, "bad MLP dimensions");
    FHR_ARG(d->ldx >= d->Nk, "ldx < Nk");
    FHR_ARG(d->x_dtype == FHR_F32 || d->x_dtype == FHR_BF16, "bad x_dtype");
    return FHR_OK;
}

template <typename TA, typename TB, int EPI>
static fhr_status gemm(fhr_ctx *ctx, const GemmArgs &g, int splits = 1) {
    dim3 grid((unsigned)cdiv(g.N, GBN), (unsigned)cdiv(g.M, GBM), (unsigned)splits);
    gemm_kernel<TA, TB, EPI><<<grid, 256, 0, ctx->stream>>>(g);
    FHR_LAUNCHED();
    return FHR_OK;
}

// weights as seen by the GEMMs: bf16 copies or the f32 master
template <typename TW>
static const void *wptr(const float *prm, const MlpWs &w, int64_t off) {
    if (sizeof(TW) == 2) return w.wb + off;
    return prm + off;
}

// the tensor-core layers take bf16 rows and weights with 16-byte aligned rows
static bool mma_layers(const fhr_mlp_dims *d, const void *X) {
    return d->x_dtype == FHR_BF16 && d->weights_bf16 && d->ldx % 8 == 0 && d->H1 % 8 == 0 && d->H2 % 8 == 0 &&
           ((uintptr_t)X & 15) == 0;
}

// layers 1 and 2: the tcgen05 kernel (mlp_tc.cu) when the shape allows it, else warp MMA
constexpr int kOutMax = 8;   // outputs of mlp_out_kernel

// Layer 3 of the tensor-core forward (K <= kOutMax outputs from H2 bf16 activations,
// H2 % 8 == 0): Y = softplus(A2 W3^T + b3), one pixel row per thread, W3 staged in
// shared memory as FP32 (every thread reads the same entry: a broadcast).  The
// 64 x 64 tiles of gemm_kernel would spend most of their work on the K <= 8 columns.
__global__ void __launch_bounds__(256) mlp_out_kernel(const __nv_bfloat16 *__restrict__ A,
                                                      const __nv_bfloat16 *__restrict__ W,
                                                      const float *__restrict__ bias, int H2, int K, int64_t M,
                                                      float *__restrict__ Y, float *__restrict__ Z3) {
    extern __shared__ float w3[];   // [K][H2]
    for (int i = threadIdx.x; i < K * H2; i += blockDim.x) w3[i] = __bfloat162float(W[i]);
    __syncthreads();
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < M; row += (int64_t)gridDim.x * blockDim.x) {
        float acc[kOutMax];
#pragma unroll
        for (int j = 0; j < kOutMax; ++j) acc[j] = 0.f;
        const uint4 *a = reinterpret_cast<const uint4 *>(A + row * H2);
        for (int k = 0; k < H2; k += 8) {
            const uint4 q = __ldcs(a + k / 8);
            const uint32_t qq[4] = {q.x, q.y, q.z, q.w};
            float x[8];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                x[2 * e] = __uint_as_float(qq[e] << 16);
                x[2 * e + 1] = __uint_as_float(qq[e] & 0xffff0000u);
            }
#pragma unroll
            for (int j = 0; j < kOutMax; ++j) {
                if (j < K) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[j] = fmaf(x[e], w3[j * H2 + k + e], acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kOutMax; ++j) {
            if (j < K) {
                const float v = acc[j] + bias[j];
                if (Z3) Z3[row * K + j] = v;
                Y[row * K + j] = softplus_f(v);
            }
        }
    }
}

static fhr_status mma_layer(fhr_ctx *ctx, const MmaGemmArgs &g, int *status) {
    TcGemmArgs t{g.M, g.N, g.Kd, g.A, g.lda, g.B, g.ldb, g.bias, g.Z, g.ldz, g.Act, g.ldact, status};
    if (mlp_tc_ok(t)) return mlp_tc_layer(ctx, t);
    FHR_CUDA(cudaFuncSetAttribute(mlp_gemm_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem));
    dim3 grid((unsigned)cdiv(g.N, MBN), (unsigned)cdiv(g.M, MBM));
    mlp_gemm_mma<<<grid, 256, kMmaSmem, ctx->stream>>>(g);
    FHR_LAUNCHED();
    return FHR_OK;
}

// forward of `rows` pixel rows starting at X (row stride ldx); fills A1, A2,
// Yout (and Z1, Z2, Z3out when the pre-activations are wanted for a backward pass)
template <typename TX, typename TW>
static fhr_status forward_chunk(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *prm, const MlpWs &w, int64_t rows,
                                const void *X, float *Yout, float *Z3out, bool need_z) {
    const MlpLayout L = mlp_layout(d);
    if (sizeof(TX) == 2 && sizeof(TW) == 2 && mma_layers(d, X)) {
        MmaGemmArgs m{};
        m.M = (int)rows; m.N = d->H1; m.Kd = d->Nk;
        m.A = (const __nv_bfloat16 *)X; m.lda = d->ldx;
        m.B = w.wp1; m.ldb = pad8(d->Nk);
        m.bias = prm + L.ob1;
        m.Z = need_z ? w.Z1 : nullptr; m.ldz = d->H1;
        m.Act = (__nv_bfloat16 *)w.A1; m.ldact = d->H1;
        FHR_TRY(mma_layer(ctx, m, w.status));
        m.N = d->H2; m.Kd = d->H1;
        m.A = (const __nv_bfloat16 *)w.A1; m.lda = d->H1;
        m.B = w.wp2; m.ldb = pad8(d->H1);
        m.bias = prm + L.ob2;
        m.Z = need_z ? w.Z2 : nullptr; m.ldz = d->H2;
        m.Act = (__nv_bfloat16 *)w.A2; m.ldact = d->H2;
        FHR_TRY(mma_layer(ctx, m, w.status));
        if (d->H2 % 8 == 0 && d->K <= kOutMax) {
            const int blocks = (int)std::min<int64_t>(cdiv(rows, 256), (int64_t)ctx->sm_count * 8);
            const size_t smem = (size_t)d->K * d->H2 * sizeof(float);
            mlp_out_kernel<<<blocks, 256, smem, ctx->stream>>>((const __nv_bfloat16 *)w.A2,
                                                              (const __nv_bfloat16 *)wptr<TW>(prm, w, L.oW3),
                                                              prm + L.ob3, d->H2, d->K, rows, Yout, Z3out);
            FHR_LAUNCHED();
            return FHR_OK;
        }
        GemmArgs g{};
        g.M = (int)rows; g.N = d->K; g.Kd = d->H2;
        g.A = w.A2; g.sai = d->H2; g.sak = 1;
        g.B = wptr<TW>(prm, w, L.oW3); g.sbk = 1; g.sbj = d->H2;
        g.C = Yout; g.ldc = d->K; g.C2 = Z3out; g.ldc2 = d->K;
        g.bias = prm + L.ob3; g.kchunk = g.Kd;
        return gemm<TW, TW, EPI_BIAS_SOFTPLUS>(ctx, g);
    }
    GemmArgs g{};
    // layer 1: Z1 = X W1^T + b1
    g.M = (int)rows; g.N = d->H1; g.Kd = d->Nk;
    g.A = X; g.sai = d->ldx; g.sak = 1;
    g.B = wptr<TW>(prm, w, L.oW1); g.sbk = 1; g.sbj = d->Nk;
    g.C = need_z ? w.Z1 : nullptr; g.ldc = d->H1;
    g.C2 = w.A1; g.c2_bf16 = sizeof(TW) == 2; g.ldc2 = d->H1;
    g.bias = prm + L.ob1; g.kchunk = g.Kd;
    FHR_TRY((gemm<TX, TW, EPI_BIAS_GELU>(ctx, g)));
    // layer 2
    g.N = d->H2; g.Kd = d->H1;
    g.A = w.A1; g.sai = d->H1;
    g.B = wptr<TW>(prm, w, L.oW2); g.sbj = d->H1;
    g.C = need_z ? w.Z2 : nullptr; g.ldc = d->H2; g.C2 = w.A2; g.ldc2 = d->H2;
    g.bias = prm + L.ob2; g.kchunk = g.Kd;
    FHR_TRY((gemm<TW, TW, EPI_BIAS_GELU>(ctx, g)));
    // layer 3: Y = softplus(A2 W3^T + b3)
    g.N = d->K; g.Kd = d->H2;
    g.A = w.A2; g.sai = d->H2;
    g.B = wptr<TW>(prm, w, L.oW3); g.sbj = d->H2;
    g.C = Yout; g.ldc = d->K; g.C2 = Z3out; g.ldc2 = d->K;
    g.bias = prm + L.ob3; g.kchunk = g.Kd;
    FHR_TRY((gemm<TW, TW, EPI_BIAS_SOFTPLUS>(ctx, g)));
    return FHR_OK;
}

// backward of a chunk: accumulates parameter gradients into grad (+=)
template <typename TX, typename TW>
static fhr_status backward_chunk(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *prm, const MlpWs &w, int64_t rows,
                                 const void *X, float *grad) {
    const MlpLayout L = mlp_layout(d);
    const int splits = (int)mlp_splits(rows);
    auto wgrad = [&](const float *dZ, int nout, const void *act, int nin, int act_bf16, int64_t off) -> fhr_status {
        // grad[off + o*nin + i] += sum_m dZ[m][o] act[m][i]
        GemmArgs g{};
        g.M = nout; g.N = nin; g.Kd = (int)rows;
        g.A = dZ; g.sai = 1; g.sak = nout;
        g.B = act; g.sbk = nin; g.sbj = 1;
        g.C = w.part; g.ldc = nin; g.split_stride = (int64_t)nout * nin; g.kchunk = kSplitRows;
        if (act_bf16) FHR_TRY((gemm<float, __nv_bfloat16, EPI_STORE>(ctx, g, splits)));
        else FHR_TRY((gemm<float, float, EPI_STORE>(ctx, g, splits)));
        const int64_t n = (int64_t)nout * nin;
        mlp_reduce_splits<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 4096), 256, 0, ctx->stream>>>(w.part, splits, n,
                                                                                                    grad + off);
        FHR_LAUNCHED();
        return FHR_OK;
    };
    auto bgrad = [&](const float *dZ, int n, float *out) -> fhr_status {
        mlp_colsum<<<(unsigned)cdiv(n, 32), 256, 0, ctx->stream>>>(dZ, rows, n, out);
        FHR_LAUNCHED();
        return FHR_OK;
    };
    const int wb = sizeof(TW) == 2;
    // layer 3
    FHR_TRY(wgrad(w.dZ3, d->K, w.A2, d->H2, wb, L.oW3));
    FHR_TRY(bgrad(w.dZ3, d->K, grad + L.ob3));
    // dZ2 = (dZ3 W3) * gelu'(Z2)
    {
        GemmArgs g{};
        g.M = (int)rows; g.N = d->H2; g.Kd = d->K;
        g.A = w.dZ3; g.sai = d->K; g.sak = 1;
        g.B = wptr<TW>(prm, w, L.oW3); g.sbk = d->H2; g.sbj = 1;
        g.C = w.dZ2; g.ldc = d->H2; g.Z = w.Z2; g.ldz = d->H2; g.kchunk = g.Kd;
        FHR_TRY((gemm<float, TW, EPI_GELU_BACK>(ctx, g)));
    }
    FHR_TRY(wgrad(w.dZ2, d->H2, w.A1, d->H1, wb, L.oW2));
    FHR_TRY(bgrad(w.dZ2, d->H2, grad + L.ob2));
    // dZ1 = (dZ2 W2) * gelu'(Z1)
    {
        GemmArgs g{};
        g.M = (int)rows; g.N = d->H1; g.Kd = d->H2;
        g.A = w.dZ2; g.sai = d->H2; g.sak = 1;
        g.B = wptr<TW>(prm, w, L.oW2); g.sbk = d->H1; g.sbj = 1;
        g.C = w.dZ1; g.ldc = d->H1; g.Z = w.Z1; g.ldz = d->H1; g.kchunk = g.Kd;
        FHR_TRY((gemm<float, TW, EPI_GELU_BACK>(ctx, g)));
    }
    // layer 1 weights against the input rows (row stride ldx)
    {
        GemmArgs g{};
        g.M = d->H1; g.N = d->Nk; g.Kd = (int)rows;
        g.A = w.dZ1; g.sai = 1; g.sak = d->H1;
        g.B = X; g.sbk = d->ldx; g.sbj = 1;
        g.C = w.part; g.ldc = d->Nk; g.split_stride = (int64_t)d->H1 * d->Nk; g.kchunk = kSplitRows;
        FHR_TRY((gemm<float, TX, EPI_STORE>(ctx, g, splits)));
        const int64_t n = (int64_t)d->H1 * d->Nk;
        mlp_reduce_splits<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 4096), 256, 0, ctx->stream>>>(
            w.part, splits, n, grad + L.oW1);
        FHR_LAUNCHED();
    }
    FHR_TRY(bgrad(w.dZ1, d->H1, grad + L.ob1));
    return FHR_OK;
}

static fhr_status prep_weights(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *prm, const MlpWs &w) {
    if (!d->weights_bf16) return FHR_OK;
    const MlpLayout L = mlp_layout(d);
    to_bf16_kernel<<<(unsigned)std::min<int64_t>(cdiv(L.n, 256), 4096), 256, 0, ctx->stream>>>(prm, L.n, w.wb);
    FHR_LAUNCHED();
    pad_bf16_kernel<<<(unsigned)std::min<int64_t>(cdiv((int64_t)d->H1 * pad8(d->Nk), 256), 4096), 256, 0,
                      ctx->stream>>>(prm + L.oW1, d->H1, d->Nk, pad8(d->Nk), w.wp1);
    FHR_LAUNCHED();
    pad_bf16_kernel<<<(unsigned)std::min<int64_t>(cdiv((int64_t)d->H2 * pad8(d->H1), 256), 4096), 256, 0,
                      ctx->stream>>>(prm + L.oW2, d->H2, d->H1, pad8(d->H1), w.wp2);
    FHR_LAUNCHED();
    return FHR_OK;
}

template <typename TX, typename TW>
static fhr_status forward_all(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *prm, const MlpWs &w, int64_t M,
                              const void *X, float *Y) {
    const int es = d->x_dtype == FHR_BF16 ? 2 : 4;
    for (int64_t r0 = 0; r0 < M; r0 += kMlpFwdChunk) {
        const int64_t rows = std::min<int64_t>(kMlpFwdChunk, M - r0);
        FHR_TRY((forward_chunk<TX, TW>(ctx, d, prm, w, rows, (const char *)X + r0 * d->ldx * es, Y + r0 * d->K,
                                       nullptr, false)));
    }
    return FHR_OK;
}

fhr_status mlp_forward_impl(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *prm, int64_t M, const void *X, float *Y,
                            void *ws, size_t ws_bytes) {
    FHR_TRY(check_dims(ctx, d));
    FHR_ARG(prm && X && Y && ws, "null pointer argument");
    FHR_ARG(M >= 0, "M < 0");
    MlpWs w;
    const size_t need = carve_mlp(ws, d, 0, &w);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    FHR_CUDA(cudaSetDevice(ctx->device));
    cudaEvent_t *ev = timer_begin(ctx, TM_MLP_FORWARD);   // the whole forward, when profiling
    fhr_status s = prep_weights(ctx, d, prm, w);
    if (s == FHR_OK) {
        if (d->x_dtype == FHR_BF16)
            s = d->weights_bf16 ? forward_all<__nv_bfloat16, __nv_bfloat16>(ctx, d, prm, w, M, X, Y)
                                : forward_all<__nv_bfloat16, float>(ctx, d, prm, w, M, X, Y);
        else
            s = d->weights_bf16 ? forward_all<float, __nv_bfloat16>(ctx, d, prm, w, M, X, Y)
                                : forward_all<float, float>(ctx, d, prm, w, M, X, Y);
    }
    if (ev) cudaEventRecord(ev[1], ctx->stream);
    return s;
}

size_t mlp_ws_bytes(const fhr_mlp_dims *d, int train) { return carve_mlp(nullptr, d, train, nullptr); }

template <typename TX, typename TW>
static fhr_status grad_impl(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *prm, const MlpWs &w, int64_t M,
                            const void *X, const float *T, float *grad, double *loss) {
    FHR_ARG(M > 0 && M <= kMlpChunk, "fhr_mlp_grad takes 1..%d rows per call", kMlpChunk);
    FHR_TRY((forward_chunk<TX, TW>(ctx, d, prm, w, M, X, w.Y, w.Z3, true)));
    const int64_t n = M * d->K;
    const int nb = (int)std::min<int64_t>(cdiv(n, 256), 1024);
    mlp_loss_kernel<<<nb, 256, 0, ctx->stream>>>(w.Y, w.Z3, T, n, 2.f / (float)n, w.dZ3, w.lpart);
    FHR_LAUNCHED();
    mlp_loss_final<<<1, 32, 0, ctx->stream>>>(w.lpart, nb, 1.0 / (double)n, loss ? loss : w.lacc);
    FHR_LAUNCHED();
    return backward_chunk<TX, TW>(ctx, d, prm, w, M, X, grad);
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_mlp_workspace_size(fhr_ctx *ctx, const fhr_mlp_dims *d, int train, size_t *bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_dims(ctx, d));
    FHR_ARG(bytes, "bytes is null");
    *bytes = carve_mlp(nullptr, d, train, nullptr);
    return FHR_OK;
}

extern "C" fhr_status fhr_mlp_forward(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *params, int64_t M,
                                      const void *X, float *Y, void *ws, size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    return mlp_forward_impl(ctx, d, params, M, X, Y, ws, ws_bytes);
}

extern "C" fhr_status fhr_mlp_grad(fhr_ctx *ctx, const fhr_mlp_dims *d, const float *params, int64_t M, const void *X,
                                   const float *T, float *grad, double *loss, void *ws, size_t ws_bytes) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_TRY(check_dims(ctx, d));
    FHR_ARG(params && X && T && grad && ws, "null pointer argument");
    MlpWs w;
    const size_t need = carve_mlp(ws, d, 1, &w);
    FHR_ARG(ws_bytes >= need, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    FHR_CUDA(cudaSetDevice(ctx->device));
    FHR_TRY(prep_weights(ctx, d, params, w));
    if (d->x_dtype == FHR_BF16) {
        if (d->weights_bf16) return grad_impl<__nv_bfloat16, __nv_bfloat16>(ctx, d, params, w, M, X, T, grad, loss);
        return grad_impl<__nv_bfloat16, float>(ctx, d, params, w, M, X, T, grad, loss);
    }
    if (d->weights_bf16) return grad_impl<float, __nv_bfloat16>(ctx, d, params, w, M, X, T, grad, loss);
    return grad_impl<float, float>(ctx, d, params, w, M, X, T, grad, loss);
}

extern "C" fhr_status fhr_mlp_adamw(fhr_ctx *ctx, int64_t n, float *params, const float *grad, float *m, float *v,
                                    int step, float lr, float beta1, float beta2, float eps, float weight_decay) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_ARG(params && grad && m && v && n > 0 && step >= 1, "bad AdamW arguments");
    FHR_CUDA(cudaSetDevice(ctx->device));
    const float c1 = (float)(1.0 - pow((double)beta1, step)), c2 = (float)(1.0 - pow((double)beta2, step));
    adamw_kernel<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 4096), 256, 0, ctx->stream>>>(
        n, params, grad, m, v, lr, beta1, beta2, eps, weight_decay, c1, c2);
    FHR_LAUNCHED();
    return FHR_OK;
}
