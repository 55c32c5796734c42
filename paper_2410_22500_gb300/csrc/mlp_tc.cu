// The network's wide layers on the fifth-generation tensor cores (tcgen05):
// one CTA per 128 rows of A, the whole of N (<= 256) as one tile.
//
//   warp 0   lane 0 copies, per k-step of 64 bins, the A tile [128][64] and
//            the B tile [N][64] (bf16, 128-byte rows, 128-byte swizzle) into a
//            4-stage ring with tensor-map copies (full / empty mbarriers);
//   warp 1   owns the tensor-memory accumulator (N fp32 columns x 128 lanes);
//            lane 0 issues four tcgen05.mma (M 128, N, K 16) per k-step and
//            commits each stage back to the producer when its MMAs have read it;
//   warps 2-5  read the accumulator (warp w reads lanes 32 (w % 4) ..), add the
//            bias, apply GELU and store bf16 activations (and FP32 Z).
// Every wait is bounded; on a timeout the CTA still frees its tensor memory.
#include "mlp_tc.h"
#include "tma.cuh"

namespace fhr {

constexpr int kTcBM = 128, kTcBK = 64, kTcStages = 4, kTcThreads = 320;   // 2 + 8 warps

// shared-memory descriptor of a K-major operand tile in the 128-byte swizzle:
// 8-row x 128-byte atoms, 1024 bytes apart (stride byte offset); the leading
// byte offset is not used for this layout; descriptor version 1 (bit 46)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N, M
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// arrives once on the mbarrier when every tcgen05 operation this thread issued has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// lane i of the warp receives columns [col, col + 16) of tensor-memory lane (lane base + i)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tc_gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

// Persistent: a CTA takes the 128-row tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// with two accumulators in tensor memory (columns [0, ncols) and [ncols, 2 ncols)),
// so the epilogue of one tile runs while the MMAs of the next fill the other.
// ncols: columns per accumulator (a power of two >= max(32, N), 2 ncols <= 512).
__global__ void __launch_bounds__(kTcThreads, 1) mlp_gemm_tc(const __grid_constant__ CUtensorMap ma,
                                                             const __grid_constant__ CUtensorMap mb, TcGemmArgs g,
                                                             uint32_t ncols) {
    extern __shared__ __align__(128) unsigned char tc_sm[];
    constexpr int S = kTcStages;
    constexpr int NE = kTcThreads / 32 - 2;   // epilogue warps
    const int N = g.N;
    const uint32_t A_BYTES = kTcBM * kTcBK * 2, B_BYTES = (uint32_t)N * kTcBK * 2;
    const uint32_t STAGE = A_BYTES + B_BYTES;   // a multiple of 2 KB (N % 16 == 0)
    // the 128-byte swizzle wants 1024-byte aligned tiles
    unsigned char *base = tc_sm + ((1024u - (smem_u32(tc_sm) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + (size_t)S * STAGE);
    uint64_t *empty = full + S;
    uint64_t *accf = empty + S;   // accumulator a complete (MMA -> epilogue)
    uint64_t *acce = accf + 2;    // accumulator a drained (epilogue -> MMA)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (g.Kd + kTcBK - 1) / kTcBK;
    const int64_t ntiles = (g.M + kTcBM - 1) / kTcBM;
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], NE);
        }
        fence_mbar_init();
    }
    if (warp == 1) {
        tc_alloc(smem_u32(tslot), 2 * ncols);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---- producer: the (tile, k-step) sequence through one ring
        int st = 0;
        uint32_t par = 0;
        int64_t n = 0;   // stages filled
        bool ok = true;
        for (int64_t j = 0; j < my_tiles && ok; ++j) {
            const int m0 = (int)((blockIdx.x + j * gridDim.x) * kTcBM);
            for (int k = 0; k < nk; ++k, ++n) {
                if (n >= S && !mbar_wait_bounded(&empty[st], par ^ 1u)) {
                    report(g.status, FHR_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                unsigned char *sa = base + (size_t)st * STAGE;
                mbar_arrive_expect_tx(&full[st], STAGE);
                tma_load_2d(sa, &ma, k * kTcBK, m0, &full[st]);
                tma_load_2d(sa + A_BYTES, &mb, k * kTcBK, 0, &full[st]);
                if (++st == S) {
                    st = 0;
                    par ^= 1u;
                }
            }
        }
        // no copy may land after the CTA exits
        for (int64_t q = n > S ? n - S : 0; q < n; ++q) mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1));
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issue: four K = 16 steps per stage, the descriptors advanced 32 bytes each
        const uint32_t idesc = tc_idesc(kTcBM, N);
        int st = 0;
        uint32_t par = 0;
        bool ok = true;
        for (int64_t j = 0; j < my_tiles && ok; ++j) {
            const int a = (int)(j & 1);
            // the epilogue of tile j - 2 has drained accumulator a
            if (j >= 2 && !mbar_wait_bounded(&acce[a], (uint32_t)(((j >> 1) - 1) & 1))) {
                report(g.status, FHR_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)a * ncols;
            for (int k = 0; k < nk; ++k) {
                if (!mbar_wait_bounded(&full[st], par)) {
                    report(g.status, FHR_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(base + (size_t)st * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
                for (int kk = 0; kk < kTcBK / 16; ++kk)
                    tc_mma(d, tc_desc(a0 + 32u * kk), tc_desc(b0 + 32u * kk), idesc, (k | kk) != 0 ? 1u : 0u);
                tc_commit(&empty[st]);
                if (++st == S) {
                    st = 0;
                    par ^= 1u;
                }
            }
            if (ok) tc_commit(&accf[a]);
        }
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows) and the
        // 16-column groups h, h + 2, ... (h = the warp's half), then releases the accumulator
        const int q = warp & 3, h = (warp - 2) / 4;
        for (int64_t j = 0; j < my_tiles; ++j) {
            const int a = (int)(j & 1);
            const bool ok = mbar_wait_bounded(&accf[a], (uint32_t)((j >> 1) & 1));
            tc_fence_after();
            if (!ok) {
                if (lane == 0) report(g.status, FHR_ERR_TIMEOUT);
                break;
            }
            const int64_t row = (blockIdx.x + j * gridDim.x) * kTcBM + 32 * q + lane;
            const bool live = row < g.M;
            for (int c0 = 16 * h; c0 < N; c0 += 32) {
                uint32_t r[16];
                tc_ld16(tmem + (uint32_t)a * ncols + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, r);
                tc_wait_ld();
                if (!live) continue;
                float z[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) z[i] = __uint_as_float(r[i]) + __ldg(g.bias + c0 + i);
                if (g.Z) {
                    float4 *zp = reinterpret_cast<float4 *>(g.Z + row * g.ldz + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) zp[i] = make_float4(z[4 * i], z[4 * i + 1], z[4 * i + 2], z[4 * i + 3]);
                }
                uint32_t hb[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    __nv_bfloat162 v = __floats2bfloat162_rn(tc_gelu(z[2 * i]), tc_gelu(z[2 * i + 1]));
                    hb[i] = *reinterpret_cast<uint32_t *>(&v);
                }
                uint4 *ap = reinterpret_cast<uint4 *>(g.Act + row * g.ldact + c0);
                ap[0] = make_uint4(hb[0], hb[1], hb[2], hb[3]);
                ap[1] = make_uint4(hb[4], hb[5], hb[6], hb[7]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[a]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tc_dealloc(tmem, 2 * ncols);
    }
}

bool mlp_tc_ok(const TcGemmArgs &g) {
    return g.N >= 16 && g.N <= 256 && g.N % 16 == 0 && g.Kd >= 1 && g.lda % 8 == 0 && g.ldb % 8 == 0 &&
           g.ldact % 8 == 0 && (!g.Z || g.ldz % 4 == 0) && ((uintptr_t)g.A & 15) == 0 && ((uintptr_t)g.B & 15) == 0 &&
           ((uintptr_t)g.Act & 15) == 0 && (!g.Z || ((uintptr_t)g.Z & 15) == 0) && tma_available();
}

size_t mlp_tc_smem(int N) {
    return (size_t)kTcStages * ((size_t)kTcBM * kTcBK * 2 + (size_t)N * kTcBK * 2) + 1024 + (2 * kTcStages + 4) * 8 + 16;
}

fhr_status mlp_tc_layer(fhr_ctx *ctx, const TcGemmArgs &g) {
    CUtensorMap ma, mb;
    {
        const uint64_t da[2] = {(uint64_t)g.Kd, (uint64_t)g.M}, sa[1] = {(uint64_t)g.lda * 2};
        const uint32_t ba[2] = {kTcBK, kTcBM};
        const uint64_t db[2] = {(uint64_t)g.Kd, (uint64_t)g.N}, sb[1] = {(uint64_t)g.ldb * 2};
        const uint32_t bb[2] = {kTcBK, (uint32_t)g.N};
        FHR_ARG(tma_make_map(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.A, da, sa, ba, CU_TENSOR_MAP_SWIZZLE_128B) &&
                    tma_make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.B, db, sb, bb, CU_TENSOR_MAP_SWIZZLE_128B),
                "tensor maps of the layer's operands could not be encoded");
    }
    uint32_t ncols = 32;
    while ((int)ncols < g.N) ncols <<= 1;   // two accumulators: 2 ncols <= 512 columns
    const size_t smem = mlp_tc_smem(g.N);
    FHR_CUDA(cudaFuncSetAttribute(mlp_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t tiles = cdiv(g.M, kTcBM);
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)ctx->sm_count);
    mlp_gemm_tc<<<grid, kTcThreads, smem, ctx->stream>>>(ma, mb, g, ncols);
    FHR_LAUNCHED();
    return FHR_OK;
}

}  // namespace fhr
