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

// One voxel per block row (threadIdx.y), its bins strided over threadIdx.x in
// chunks of 4: the voxel's K coefficients are read once, the dictionary slab sits
// transposed in shared memory ([K][nk rounded up to 4], float4 reads free of bank
// conflicts), and each chunk is one 16-byte (f32) or 8-byte (bf16) streaming store.
template <int K, typename TO, bool VEC>
__global__ void __launch_bounds__(256) expand_kernel(const float *__restrict__ xs, const float *__restrict__ D,
                                                     int N, int Nr, int Nk, int k0, int nk, TO *__restrict__ xh) {
    extern __shared__ __align__(16) float dsm[];   // [K][nk4]
    const int nch = (nk + 3) / 4, nk4 = nch * 4;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int i = tid; i < K * nk4; i += nt) {
        const int j = i / nk4, k = i - j * nk4;
        dsm[i] = k < nk ? D[(size_t)(k0 + k) * K + j] : 0.f;
    }
    __syncthreads();
    const int64_t NN = (int64_t)N * N, nvox = (int64_t)Nr * NN;
    const int Wl = Nr * K;
    for (int64_t vox = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; vox < nvox;
         vox += (int64_t)gridDim.x * blockDim.y) {   // voxel (r, iy, ix)
        const int r = (int)(vox / NN);
        const int64_t pix = vox - r * NN;
        const float *a = xs + pix * Wl + r * K;
        float x[K];
#pragma unroll
        for (int j = 0; j < K; ++j) x[j] = __ldg(a + j);
        TO *row = xh + vox * nk;
        for (int ch = threadIdx.x; ch < nch; ch += blockDim.x) {
            const int kk = ch * 4;
            float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float4 d = *reinterpret_cast<const float4 *>(dsm + j * nk4 + kk);
                o[0] = fmaf(x[j], d.x, o[0]);
                o[1] = fmaf(x[j], d.y, o[1]);
                o[2] = fmaf(x[j], d.z, o[2]);
                o[3] = fmaf(x[j], d.w, o[3]);
            }
            if (VEC) st4<TO>(row + kk, o[0], o[1], o[2], o[3]);
            else
                for (int e = 0; e < 4 && kk + e < nk; ++e) st1<TO>(row + kk + e, o[e]);
        }
    }
}

// voxels per batch of the register-dictionary kernel (their coefficients staged together)
constexpr int kExpandBatch = 64;

// The same with the dictionary in registers: a thread keeps the columns of its (at
// most R) chunks for every voxel it visits, so the inner loop reads no shared memory
// (with the slab in shared memory, the K x 4 floats read per 4-bin chunk outweighed
// the chunk's own output write).  Slabs of up to R x 256 chunks (1024 R bins).

template <int K, typename TO, bool VEC, int R>
__global__ void __launch_bounds__(512) expand_reg_kernel(const float *__restrict__ xs, const float *__restrict__ D,
                                                         int N, int Nr, int Nk, int k0, int nk,
                                                         TO *__restrict__ xh) {
    __shared__ float cs[2][kExpandBatch * K];
    const int nch = (nk + 3) / 4;
    float d[R][K][4];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int kk = (threadIdx.x + r * blockDim.x) * 4;
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[r][j][e] = kk + e < nk ? __ldg(D + (size_t)(k0 + kk + e) * K + j) : 0.f;
    }
    const int64_t NN = (int64_t)N * N, nvox = (int64_t)Nr * NN;
    const int Wl = Nr * K;
    // batches of V consecutive voxels (r, iy, ix) (a multiple of the block's rows): a
    // batch's V x K coefficients are loaded one per thread a whole batch ahead and
    // staged in shared memory, so no row write waits on a coefficient load
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const int V = min(kExpandBatch, (nt / K) / (int)blockDim.y * (int)blockDim.y);
    const int64_t nbatch = (nvox + V - 1) / V;
    auto load = [&](int64_t b) -> float {
        if (tid >= V * K) return 0.f;
        const int64_t vox = b * V + tid / K;
        if (vox >= nvox) return 0.f;
        const int rs = (int)(vox / NN);
        return __ldg(xs + (vox - rs * NN) * Wl + rs * K + tid % K);
    };
    int64_t b = blockIdx.x;
    float cn = b < nbatch ? load(b) : 0.f;
    int buf = 0;
    for (; b < nbatch; b += gridDim.x, buf ^= 1) {
        if (tid < V * K) cs[buf][tid] = cn;
        __syncthreads();   // (also orders the previous batch's reads of cs[buf ^ 1] before its refill)
        if (b + gridDim.x < nbatch) cn = load(b + gridDim.x);
        for (int vi = threadIdx.y; vi < V; vi += blockDim.y) {
            const int64_t vox = b * V + vi;
            if (vox >= nvox) break;
            float x[K];
#pragma unroll
            for (int j = 0; j < K; ++j) x[j] = cs[buf][vi * K + j];
            TO *row = xh + vox * nk;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ch = threadIdx.x + r * blockDim.x;
                if (ch >= nch) break;
                const int kk = ch * 4;
                float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < K; ++j) {   // packed FP32 FMAs, two bins each
                    const float2 xx = make_float2(x[j], x[j]);
                    const float2 lo = __ffma2_rn(xx, make_float2(d[r][j][0], d[r][j][1]), make_float2(o[0], o[1]));
                    const float2 hi = __ffma2_rn(xx, make_float2(d[r][j][2], d[r][j][3]), make_float2(o[2], o[3]));
                    o[0] = lo.x; o[1] = lo.y; o[2] = hi.x; o[3] = hi.y;
                }
                if (VEC) st4<TO>(row + kk, o[0], o[1], o[2], o[3]);
                else
                    for (int e = 0; e < 4 && kk + e < nk; ++e) st1<TO>(row + kk + e, o[e]);
            }
        }
    }
}

// most warps per voxel row (a block of 32 kExpandWarps threads at most)
constexpr int kExpandWarps = 8;

template <int K>
static fhr_status launch_expand(fhr_ctx *ctx, const float *xs, const float *D, int N, int Nr, int Nk, int k0,
                                int nk, int dt, void *xh) {
    const bool vec = (nk % 4 == 0) && aligned(xh, 16);
    const int nch = (nk + 3) / 4;
    const size_t smem = sizeof(float) * (size_t)nch * 4 * K;
    // threads per voxel: whole warps, at most kExpandWarps, covering the chunks in as few
    // rounds as possible
    const int warps = (nch + 31) / 32, rounds = (warps + kExpandWarps - 1) / kExpandWarps;
    const int bx = 32 * ((warps + rounds - 1) / rounds);
    const int by = std::max(1, 256 / bx);
    const int64_t nvox = (int64_t)Nr * N * N;
    const dim3 block(bx, by);
    // one resident wave of blocks (grid-stride over voxels): as many as fit on the SMs
    auto grid = [&](const void *fn, size_t sm) -> int {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bx * by, sm) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(nvox, by), (int64_t)ctx->sm_count * per_sm));   // (an upper bound on the batches too)
    };
    if (rounds <= 2) {   // the dictionary columns fit in registers
#define GOR(T, V, R)                                                                                       \
    FHR_TIMED(TM_EXPAND, (expand_reg_kernel<K, T, V, R><<<grid((const void *)expand_reg_kernel<K, T, V, R>, 0), \
                                                          block, 0, ctx->stream>>>(xs, D, N, Nr, Nk, k0, nk,    \
                                                                                   reinterpret_cast<T *>(xh))))
#define GOR2(T, V)           \
    if (rounds == 1)         \
        GOR(T, V, 1);        \
    else                     \
        GOR(T, V, 2)
        if (dt == FHR_F32) {
            if (vec) GOR2(float, true);
            else GOR2(float, false);
        } else {
            if (vec) GOR2(__nv_bfloat16, true);
            else GOR2(__nv_bfloat16, false);
        }
#undef GOR2
#undef GOR
        return FHR_OK;
    }
#define GO(T, V)                                                                                           \
    do {                                                                                                   \
        auto fn = expand_kernel<K, T, V>;                                                                  \
        FHR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));       \
        FHR_TIMED(TM_EXPAND, (fn<<<grid((const void *)fn, smem), block, smem, ctx->stream>>>(             \
                                 xs, D, N, Nr, Nk, k0, nk, reinterpret_cast<T *>(xh))));                  \
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
    FHR_ARG((size_t)((k1 - k0 + 3) / 4 * 4) * K * sizeof(float) <= (size_t)ctx->max_smem_optin, "bin slab too large");
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
