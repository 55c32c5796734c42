// Subspace expansion, Eq. (sub_expansion): x^h = x^s (D^s)^T.
// Output-write bound: each thread writes 4 consecutive bins of one voxel with
// streaming stores; the dictionary slab is staged in shared memory.
#include "common.cuh"

namespace fhr {

template <typename TO>
__device__ __forceinline__ void st4(TO *dst, float a, float b, float c, float d);
template <>
__device__ __forceinline__ void st4<float>(float *dst, float a, float b, float c, float d) {
    __stcs(reinterpret_cast<float4 *>(dst), make_float4(a, b, c, d));
}
template <>
__device__ __forceinline__ void st4<__nv_bfloat16>(__nv_bfloat16 *dst, float a, float b, float c, float d) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 u = make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
    __stcs(reinterpret_cast<uint2 *>(dst), u);
}
template <typename TO>
__device__ __forceinline__ void st1(TO *dst, float a);
template <>
__device__ __forceinline__ void st1<float>(float *dst, float a) { __stcs(dst, a); }
template <>
__device__ __forceinline__ void st1<__nv_bfloat16>(__nv_bfloat16 *dst, float a) { *dst = __float2bfloat16_rn(a); }

template <int K, typename TO, bool VEC>
__global__ void __launch_bounds__(256) expand_kernel(const float *__restrict__ xs, const float *__restrict__ D,
                                                     int N, int Nr, int Nk, int k0, int nk, TO *__restrict__ xh) {
    extern __shared__ float dsm[];   // [nk][K]
    for (int i = threadIdx.x; i < nk * K; i += blockDim.x) dsm[i] = D[(size_t)k0 * K + i];
    __syncthreads();
    const int nch = (nk + 3) / 4;
    const int64_t nvox = (int64_t)Nr * N * N;
    const int64_t total = nvox * nch;
    const int Wl = Nr * K;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vox = idx / nch;            // (r, iy, ix)
        const int ch = (int)(idx - vox * nch);
        const int64_t pix = vox % ((int64_t)N * N);
        const int r = (int)(vox / ((int64_t)N * N));
        const float *a = xs + pix * Wl + r * K;
        float x[K];
#pragma unroll
        for (int j = 0; j < K; ++j) x[j] = __ldg(a + j);
        const int kk = ch * 4;
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float s = 0.f;
            if (kk + e < nk) {
#pragma unroll
                for (int j = 0; j < K; ++j) s = fmaf(x[j], dsm[(kk + e) * K + j], s);
            }
            o[e] = s;
        }
        TO *dst = xh + vox * nk + kk;
        if (VEC) st4<TO>(dst, o[0], o[1], o[2], o[3]);
        else
            for (int e = 0; e < 4 && kk + e < nk; ++e) st1<TO>(dst + e, o[e]);
    }
}

template <int K>
static fhr_status launch_expand(fhr_ctx *ctx, const float *xs, const float *D, int N, int Nr, int Nk, int k0,
                                int nk, int dt, void *xh) {
    const bool vec = (nk % 4 == 0) && aligned(xh, 16);
    const size_t smem = sizeof(float) * (size_t)nk * K;
    const int64_t total = (int64_t)Nr * N * N * ((nk + 3) / 4);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), (int64_t)ctx->sm_count * 8));
#define GO(T, V)                                                                                           \
    do {                                                                                                   \
        auto fn = expand_kernel<K, T, V>;                                                                  \
        FHR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));       \
        FHR_TIMED(TM_EXPAND, (fn<<<blocks, 256, smem, ctx->stream>>>(xs, D, N, Nr, Nk, k0, nk,            \
                                                                     reinterpret_cast<T *>(xh))));          \
    } while (0)
    if (dt == FHR_F32) {
        if (vec) GO(float, true);
        else GO(float, false);
    } else {
        if (vec) GO(__nv_bfloat16, true);
        else GO(__nv_bfloat16, false);
    }
#undef GO
    return FHR_OK;
}

fhr_status expand_impl(fhr_ctx *ctx, int N, int Nr, int K, int Nk, int k0, int k1, const float *xs, const float *D,
                       int dt, void *xh) {
    FHR_ARG(N > 0 && Nr > 0 && Nk > 0, "sizes must be positive");
    FHR_ARG(K >= 1 && K <= 8, "K must be 1..8");
    FHR_ARG(xs && D && xh, "null pointer argument");
    FHR_ARG(dt == FHR_F32 || dt == FHR_BF16, "bad xh_dtype");
    if (k0 == 0 && k1 == 0) k1 = Nk;
    FHR_ARG(k0 >= 0 && k0 < k1 && k1 <= Nk, "bad bin slab [k0, k1)");
    FHR_ARG((size_t)(k1 - k0) * K * sizeof(float) <= (size_t)ctx->max_smem_optin, "bin slab too large");
    FHR_CUDA(cudaSetDevice(ctx->device));
    const int nk = k1 - k0;
    switch (K) {
        case 1: return launch_expand<1>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
        case 2: return launch_expand<2>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
        case 3: return launch_expand<3>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
        case 4: return launch_expand<4>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
        case 5: return launch_expand<5>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
        case 6: return launch_expand<6>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
        case 7: return launch_expand<7>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
        default: return launch_expand<8>(ctx, xs, D, N, Nr, Nk, k0, nk, dt, xh);
    }
}

}  // namespace fhr

extern "C" fhr_status fhr_expand(fhr_ctx *ctx, int N, int Nr, int K, int Nk, int k0, int k1, const float *xs,
                                 const float *D, int xh_dtype, void *xh) {
    if (!ctx) return FHR_ERR_ARG;
    return fhr::expand_impl(ctx, N, Nr, K, Nk, k0, k1, xs, D, xh_dtype, xh);
}
