// Count normalisation: Eq. (neglogattenuation) with the offset correction of
// Appendix A (Eq. back_offset).  HBM-bound: 2 bytes of counts in, 4 (f32) or
// 2 (bf16) bytes of P out per element; the open beam is read once.
#include "common.cuh"

namespace fhr {

// -log(y / y0) = ln max(y0, 1) - ln max(y, 1).  Each logarithm is carried as
// an FP32 pair hi + lo (hi = ln n rounded to FP32, lo the FP32 rounding of the
// remainder), so p = (hi0 - hi) + (lo0 - lo) is within about one ulp of the
// exact value even when p is small (hi0 - hi is exact when the two are within a
// factor 2).  Counts below kLnTab read the pair from a per-block table in shared
// memory (filled once per block in FP64), so the common case costs two table
// reads and three additions; larger counts take an FP64 logarithm.
constexpr int kLnTab = 2048;

__device__ __noinline__ float2 ln_pair(double n) {
    const double d = log(n);
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}

__device__ __forceinline__ float2 ln_count(const float2 *tab, uint32_t n) {
    return n < (uint32_t)kLnTab ? tab[n] : ln_pair((double)n);
}

__device__ __forceinline__ float neglog(const float2 *tab, uint32_t y, uint32_t y0) {
    const float2 a = ln_count(tab, y0), b = ln_count(tab, y);
    return (a.x - b.x) + (a.y - b.y);
}

__device__ __forceinline__ void fill_ln_table(float2 *tab) {
    for (int i = threadIdx.x; i < kLnTab; i += blockDim.x) tab[i] = ln_pair((double)max(i, 1));
    __syncthreads();
}

// dead entry (detector pixel (r, c), bin k): [Nk] or [Nr][Nc][Nk] mask
__device__ __forceinline__ bool is_dead(const uint8_t *dead, int per_pixel, int r, int c, int Nc, int Nk, int k) {
    return dead && (per_pixel ? dead[((size_t)r * Nc + c) * Nk + k] : dead[k]);
}

// b[v][k] = mean over the live background entries (r, c) of -log(y/y0)
// (0 when there is none); compensated sum.
__global__ void offset_reduce_kernel(const uint16_t *y, const uint16_t *y0, const uint8_t *bg, const uint8_t *dead,
                                     int per_pixel, int Nv, int Nr, int Nc, int Nk, float *b) {
    __shared__ float2 tab[kLnTab];
    fill_ln_table(tab);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (k >= Nk) return;
    float s = 0.f, comp = 0.f;
    int nb = 0;
    for (int r = 0; r < Nr; ++r)
        for (int c = 0; c < Nc; ++c) {
            if (!bg[r * Nc + c] || is_dead(dead, per_pixel, r, c, Nc, Nk, k)) continue;
            ++nb;
            const uint32_t yy = y[(((size_t)v * Nr + r) * Nc + c) * Nk + k];
            const uint32_t yo = y0[((size_t)r * Nc + c) * Nk + k];
            const float x = neglog(tab, yy, yo) - comp;
            const float t = s + x;
            comp = (t - s) - x;
            s = t;
        }
    b[(size_t)v * Nk + k] = nb > 0 ? s / (float)nb : 0.f;
}

template <typename TO>
__device__ __forceinline__ void store8(TO *dst, const float *p);
template <>
__device__ __forceinline__ void store8<float>(float *dst, const float *p) {
    reinterpret_cast<float4 *>(dst)[0] = make_float4(p[0], p[1], p[2], p[3]);
    reinterpret_cast<float4 *>(dst)[1] = make_float4(p[4], p[5], p[6], p[7]);
}
template <>
__device__ __forceinline__ void store8<__nv_bfloat16>(__nv_bfloat16 *dst, const float *p) {
    uint32_t u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(p[2 * i], p[2 * i + 1]);
        u[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(u[0], u[1], u[2], u[3]);
}
template <typename TO>
__device__ __forceinline__ void store1(TO *dst, float p);
template <>
__device__ __forceinline__ void store1<float>(float *dst, float p) { *dst = p; }
template <>
__device__ __forceinline__ void store1<__nv_bfloat16>(__nv_bfloat16 *dst, float p) { *dst = __float2bfloat16_rn(p); }

// Work unit = (detector pixel (r, c), pass): a warp's lanes take bins
// [256 pass + 8 lane, +8) of that pixel in every view v.  The open-beam
// logarithms and the dead mask of those bins are formed once per unit and
// reused for all Nv views, so y0 is read once and each output element costs one
// table read.  Output row j = (v Nc + c) Nr + r.
// VEC: counts rows are 16-byte aligned (Nk % 8 == 0), 8 counts per 16-byte load.
constexpr int kNormViews = 4;   // views whose counts a lane loads before using them

// Open-beam logarithm of a dead or padding bin: p = -huge - ln y is then
// clamped to exactly 0 by the max(., 0) below, so the mask costs nothing per view.
constexpr float kDeadLog = 1e30f;

// 8 bins of one view: p = (ln y0 - ln y) - b, clamped at 0 (a = 8 packed counts).
template <typename TO>
__device__ __forceinline__ void normalise_chunk(const float2 *tab, const float2 *o, const uint32_t *a, const float *bv,
                                                int k0, int Nk, int ldP, TO *dst) {
    float p[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 h0 = ln_count(tab, a[i] & 0xffffu), h1 = ln_count(tab, a[i] >> 16);
        p[2 * i] = (o[2 * i].x - h0.x) + (o[2 * i].y - h0.y);
        p[2 * i + 1] = (o[2 * i + 1].x - h1.x) + (o[2 * i + 1].y - h1.y);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float q = p[i];
        if (bv && k0 + i < Nk) q -= bv[k0 + i];
        p[i] = fmaxf(q, 0.f);
    }
    if (k0 + 8 <= ldP) store8<TO>(dst, p);
    else
        for (int i = 0; i < 8 && k0 + i < ldP; ++i) store1<TO>(dst + i, p[i]);
}

template <typename TO>
__device__ __forceinline__ void normalise_view(const float2 *tab, const float2 *o, uint4 w, const float *bv, int k0,
                                               int Nk, int ldP, TO *dst) {
    const uint32_t aa[4] = {w.x, w.y, w.z, w.w};
    normalise_chunk<TO>(tab, o, aa, bv, k0, Nk, ldP, dst);
}

template <bool VEC, typename TO>
__global__ void __launch_bounds__(256) normalise_kernel(const uint16_t *__restrict__ y, const uint16_t *__restrict__ y0,
                                                        const uint8_t *__restrict__ dead, int per_pixel,
                                                        const float *__restrict__ b, int Nv, int Nr, int Nc, int Nk,
                                                        int ldP, TO *__restrict__ P) {
    __shared__ float2 tab[kLnTab];
    fill_ln_table(tab);
    const int nch = (ldP + 7) / 8;
    const int npass = (nch + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int64_t units = (int64_t)Nr * Nc * npass;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    const size_t vstride = (size_t)Nr * Nc * Nk;   // counts of one view
    const size_t pstride = (size_t)Nc * Nr * ldP;  // P rows of one view
    for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < units; u += wstride) {
        const int64_t pix = u / npass;
        const int ch = (int)(u - pix * npass) * 32 + lane;
        if (ch >= nch) continue;
        const int r = (int)(pix % Nr), c = (int)(pix / Nr);
        const int k0 = ch * 8;
        const size_t yoff = ((size_t)r * Nc + c) * Nk + k0;   // (r, c, k0) in y0 and in view 0 of y
        float2 o[8];
        const bool full = VEC && k0 + 8 <= Nk;
        if (full) {
            const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(y0 + yoff));
            const uint32_t qq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                o[2 * i] = ln_count(tab, qq[i] & 0xffffu);
                o[2 * i + 1] = ln_count(tab, qq[i] >> 16);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) o[i] = ln_count(tab, k0 + i < Nk ? y0[yoff + i] : 1u);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (k0 + i >= Nk || is_dead(dead, per_pixel, r, c, Nc, Nk, k0 + i)) o[i] = make_float2(-kDeadLog, 0.f);
        TO *prow = P + ((size_t)c * Nr + r) * ldP + k0;   // view 0's row
        int v = 0;
        if (full) {
            for (; v + kNormViews <= Nv; v += kNormViews) {
                uint4 a[kNormViews];
#pragma unroll
                for (int j = 0; j < kNormViews; ++j)
                    a[j] = __ldcs(reinterpret_cast<const uint4 *>(y + (size_t)(v + j) * vstride + yoff));
#pragma unroll
                for (int j = 0; j < kNormViews; ++j)
                    normalise_view<TO>(tab, o, a[j], b ? b + (size_t)(v + j) * Nk : nullptr, k0, Nk, ldP,
                                       prow + (size_t)(v + j) * pstride);
            }
            for (; v < Nv; ++v) {
                const uint4 a = __ldcs(reinterpret_cast<const uint4 *>(y + (size_t)v * vstride + yoff));
                normalise_view<TO>(tab, o, a, b ? b + (size_t)v * Nk : nullptr, k0, Nk, ldP, prow + (size_t)v * pstride);
            }
        } else {
            for (; v < Nv; ++v) {
                const uint16_t *yr = y + (size_t)v * vstride + yoff;
                uint32_t aa[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t lo = k0 + 2 * i < Nk ? yr[2 * i] : 1u;
                    const uint32_t hi = k0 + 2 * i + 1 < Nk ? yr[2 * i + 1] : 1u;
                    aa[i] = lo | (hi << 16);
                }
                normalise_chunk<TO>(tab, o, aa, b ? b + (size_t)v * Nk : nullptr, k0, Nk, ldP,
                                           prow + (size_t)v * pstride);
            }
        }
    }
}

}  // namespace fhr

using namespace fhr;

extern "C" fhr_status fhr_normalise(fhr_ctx *ctx, const fhr_norm_params *p, const uint16_t *y, const uint16_t *y0,
                                    const uint8_t *bg, const uint8_t *dead, float *b_out, void *P) {
    if (!ctx) return FHR_ERR_ARG;
    FHR_ARG(p, "params is null");
    FHR_ARG(p->Nv > 0 && p->Nr > 0 && p->Nc > 0 && p->Nk > 0, "sizes must be positive");
    FHR_ARG(p->ldP >= p->Nk, "ldP < Nk");
    FHR_ARG(p->p_dtype == FHR_F32 || p->p_dtype == FHR_BF16, "bad p_dtype");
    FHR_ARG(p->dead_per_pixel == 0 || p->dead_per_pixel == 1, "dead_per_pixel must be 0 or 1");
    FHR_ARG(p->ldP % (p->p_dtype == FHR_BF16 ? 8 : 4) == 0, "ldP must make rows 16-byte aligned");
    FHR_ARG(y && y0 && P, "null pointer argument");
    FHR_ARG(!bg || b_out, "b_out is required with a background mask");
    FHR_ARG(aligned(P, 16), "P must be 16-byte aligned");
    FHR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const float *b = nullptr;
    if (bg) {
        dim3 grid((unsigned)cdiv(p->Nk, 128), (unsigned)p->Nv);
        offset_reduce_kernel<<<grid, 128, 0, st>>>(y, y0, bg, dead, p->dead_per_pixel, p->Nv, p->Nr, p->Nc, p->Nk,
                                                   b_out);
        FHR_LAUNCHED();
        b = b_out;
    }
    // the 8-bin chunks of the f32 output need ldP % 8 == 0 for full 32-byte stores;
    // other ldP take the scalar store tail
    const bool vec = (p->Nk % 8 == 0) && aligned(y, 16) && aligned(y0, 16);
    const int64_t units = (int64_t)p->Nr * p->Nc * cdiv(cdiv(p->ldP, 8), 32);
    const int blocks = (int)std::min<int64_t>(cdiv(units, 8), (int64_t)ctx->sm_count * 8);
    const int ldp8 = p->ldP;
#define LAUNCH(V, T)                                                                                     \
    FHR_TIMED(TM_NORMALISE, (normalise_kernel<V, T><<<blocks, 256, 0, st>>>(y, y0, dead, p->dead_per_pixel, b, p->Nv, \
                                                                            p->Nr, p->Nc, p->Nk, ldp8,                \
                                                                            reinterpret_cast<T *>(P))))
    if (p->p_dtype == FHR_F32) {
        if (vec) LAUNCH(true, float);
        else LAUNCH(false, float);
    } else {
        if (vec) LAUNCH(true, __nv_bfloat16);
        else LAUNCH(false, __nv_bfloat16);
    }
#undef LAUNCH
    return FHR_OK;
}
