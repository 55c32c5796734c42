// Fused one-pass NMF kernel on the tensor cores (fast HALS, Sec. III /
// Eq. sub_extract_solve).  Same contract as the CUDA-core pass in
// nmf_pass.cuh (PassArgs, per-CTA partials), different work split:
//
//   producer warp   one 1-D bulk copy per pixel row into a padded shared
//                   row (stride = 16 mod 128 bytes, so every fragment load
//                   below is free of bank conflicts); tiles of 8 rows;
//   CW consumer     each owns a fixed range of NKW bins (a multiple of 16):
//   warps (13 f32,  phase 1 (tile t): partial r = D^T p for the 8 rows over
//   12 bf16)        its bins with warp MMAs (D^T as the 16 x k operand: rows
//                   0..7 its high, rows 8..15 its low part; P^T as the k x 8
//                   operand), written to shared memory; phase 3 (tile
//                   t - LAG): Q += P^T w over its bins (P^T as the 16 x k
//                   operand, w as the k x 8 operand), Q in MMA accumulators
//                   for the whole launch;
//   15 - CW update  (tiles in turn) sum the CW partials of r, run the HALS
//   warps           V half-step of the 8 pixels and write W; they stage w
//                   for phase 3 and add w^T w to G_W from the staged
//                   fragments with two MMAs (so the consumers' work is even).
// The update warps and the producer sit on one SM sub-partition (warps w and
// w + 4k share one), with a single consumer warp when there are two update
// warps and none when there are three, since the update is latency-bound;
// phase 3 runs LAG tiles behind phase 1 (1 for f32 rows, 3 for bf16) so that
// latency is off the per-tile critical path.  The pass is bound by the tiles in
// flight: a stage is free for the next copy only after phase 3 of its tile.
//
// Precision.  f32 P: TF32 products with the three-term split x = big + small
// (big = x rounded or truncated to TF32, small = x - big) for P, D and w,
// dropping only small*small (D's small part is kept to bf16, 2^-20 of D), so
// products carry ~20 bits; bf16 P: P is exact in bf16, D and w are split into
// bf16 hi + lo (~16 bits).  Accumulation is FP32 in both.
#pragma once

#include "nmf_pass.cuh"

namespace fhr {

constexpr int kMmaRows = 8;            // pixel rows per tile

// the producer issues a tile's bulk copies from one lane per row (true) or all from lane 0
template <typename TP>
struct MmaProducerLanes {
    static constexpr bool V = sizeof(TP) == 2;
};
// 16 warps in all (128 registers per thread): CW consumer warps, 15 - CW update
// warps and the producer.  13 + 2 for f32 rows, 12 + 3 for bf16 (whose shorter
// rows make the per-tile HALS update weigh more, and whose 1504-bin rows split
// into 12 x 128 bins with less padding than 13 x 128)
constexpr int kMmaWarps = 16;
constexpr int kMmaThreads = kMmaWarps * 32;
template <typename TP>
struct MmaCW {
    static constexpr int V = sizeof(TP) == 4 ? 13 : 12;
};
constexpr int kMmaWbStride = 48;       // bytes per s-row of the staged w (conflict-free ldmatrix)

// bins per consumer warp (a multiple of 16) for rows of Nk live bins
__host__ __device__ inline int mma_nkw(int Nk, int cw) {
    const int per = (Nk + cw - 1) / cw;
    return (per + 15) / 16 * 16;
}

struct MmaSmem {
    size_t tiles, wst, wb, red, gsm, invd, wsc, ssq, gwx, bars, total;
    uint32_t rs;   // bytes per staged pixel row
};

// nb: hand-off buffers between phase 1 and phase 3 (pipeline lag + 1)
__host__ __device__ inline MmaSmem mma_smem_layout(int Nk, int esize, int stages, int nb, int cw) {
    MmaSmem L;
    size_t o = 0;
    auto take = [&](size_t bytes, size_t align) {
        o = (o + align - 1) / align * align;
        size_t r = o;
        o += bytes;
        return r;
    };
    const size_t cols = (size_t)cw * mma_nkw(Nk, cw);
    L.rs = (uint32_t)((cols * esize + 127) / 128 * 128 + 16);
    L.tiles = take((size_t)stages * kMmaRows * L.rs, 128);
    L.wst = take((size_t)stages * kMmaRows * kMaxK * sizeof(float), 128);   // W rows of each staged tile
    L.wb = take((size_t)nb * 2 * 8 * kMmaWbStride, 128);     // [buffer][big|small or hi|lo][s][48 B]
    L.red = take((size_t)nb * 16 * 64 * sizeof(float), 16);   // [buffer][warp, padded to 16][row][s]
    L.gsm = take((size_t)kMaxK * kMaxK * sizeof(float), 16);
    L.invd = take((size_t)kMaxK * sizeof(float), 16);
    L.wsc = take((size_t)kMaxK * sizeof(float), 16);
    L.ssq = take((size_t)cw * sizeof(float), 16);
    L.gwx = take((size_t)(kMmaWarps - 1 - cw) * 32 * 4 * sizeof(float), 16);   // G_W fragments of the update warps
    L.bars = take((size_t)(2 * stages + 2 * nb) * sizeof(uint64_t), 8);
    L.total = (o + 127) / 128 * 128;
    return L;
}

// ---- warp-level tensor-core primitives (PTX)
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t a, uint32_t &r0, uint32_t &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t a, uint32_t &r0, uint32_t &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void lds_u2(uint32_t a, uint32_t &x, uint32_t &y) {
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "r"(a));
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) { asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v)); }
__device__ __forceinline__ void sts_u16(uint32_t a, uint16_t v) { asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(v)); }
__device__ __forceinline__ void sts_v2f(uint32_t a, float x, float y) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y));
}
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

// D += A B, m16n8k8, TF32 inputs (32-bit containers), FP32 accumulate
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// D += A B, m16n8k16, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t tf32_big(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// x = big + small exactly: big keeps the 10 explicit mantissa bits of a TF32
// (read exactly by the tensor core), small = x - big is a plain FP32 pattern
// whose own TF32 reading is within 2^-21 |x|
__device__ __forceinline__ void tf32_split(uint32_t xb, uint32_t &big, uint32_t &small) {
    big = xb & 0xffffe000u;
    small = __float_as_uint(__uint_as_float(xb) - __uint_as_float(big));
}
__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}
__device__ __forceinline__ float bf16_lo_f(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// ssq += squares of the one (f32) or two (bf16) values in a 32-bit word
template <bool F32>
__device__ __forceinline__ float sq_acc(uint32_t v, float ssq) {
    if (F32) {
        const float x = __uint_as_float(v);
        return fmaf(x, x, ssq);
    }
    const float lo = bf16_lo_f(v), hi = bf16_hi_f(v);
    return fmaf(lo, lo, fmaf(hi, hi, ssq));
}

// GEMM1 k-steps: 8 bins (TF32) or 16 bins (BF16) per MMA
template <typename TP>
struct MmaK {
    static constexpr int STEP = sizeof(TP) == 4 ? 8 : 16;
};

// index of G[s][t] in the row-major upper triangle of an 8 x 8 symmetric matrix
__host__ __device__ constexpr int mma_tri(int s, int t) {
    return s <= t ? s * kMaxK - s * (s - 1) / 2 + (t - s) : t * kMaxK - t * (t - 1) / 2 + (s - t);
}

// f32 staging order of a tile's 8 rows in the TF32 k dimension of phase 3:
// k index j <-> row mma_perm(j) makes the four rows read by one load instruction
// fall 8 banks apart.
__device__ __forceinline__ int mma_perm(int j) { return j < 4 ? 2 * j : 2 * (j - 4) + 1; }
__device__ __forceinline__ int mma_perm_inv(int r) { return (r & 1) ? 4 + (r >> 1) : (r >> 1); }

// LAG: phase 3 of tile i - LAG follows phase 1 of tile i, so the update of a
// tile has LAG tile periods to complete
template <typename TP, int NKW, int LAG>
__global__ void __launch_bounds__(kMmaThreads, 1) nmf_mma_kernel(PassArgs a) {
    constexpr int NB = LAG + 1;
    constexpr bool F32 = sizeof(TP) == 4;
    constexpr int ES = (int)sizeof(TP);
    constexpr int KS = NKW / MmaK<TP>::STEP;    // GEMM1 k-steps per warp
    constexpr int MB = NKW / 16;                // GEMM2 m-blocks per warp
    constexpr int CW = MmaCW<TP>::V;            // consumer warps
    constexpr int NU = kMmaWarps - 1 - CW;      // update warps
    constexpr int NT = CW * 32;                 // consumer threads

    const int tid = threadIdx.x;
    const int hw = tid >> 5, lane = tid & 31;   // hardware warp index
    const int g = lane >> 2, tig = lane & 3;
    const int K = a.K;
    // roles: warps 1 and 5 update, warp 9 produces (warps w and w + 4k share an SM
    // sub-partition, so the latency-bound update warps share theirs with one
    // consumer and the mostly idle producer); the other 13 warps are consumers 0..12
    // (with three update warps, warp 13 is the third: sub-partition 1 then holds no consumer)
    const bool upd3 = NU == 3 && hw == 13;
    const int role = (hw == 1 || hw == 5 || upd3) ? 1 : (hw == 9 ? 2 : 0);
    const int warp = role == 0 ? hw - (hw > 1) - (hw > 5) - (hw > 9) - (NU == 3 && hw > 13)
                               : (role == 1 ? (hw == 1 ? 0 : (hw == 5 ? 1 : 2)) : 0);
    const int S = a.stages;
    const int64_t ntiles = (a.Np + kMmaRows - 1) / kMmaRows;
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    extern __shared__ __align__(128) unsigned char smem[];
    const MmaSmem Lyt = mma_smem_layout(a.Nk, ES, S, NB, CW);
    const uint32_t sb = smem_u32(smem);
    const uint32_t tiles_a = sb + (uint32_t)Lyt.tiles;
    const uint32_t wb_a = sb + (uint32_t)Lyt.wb;
    const uint32_t red_a = sb + (uint32_t)Lyt.red;
    const float *wst = reinterpret_cast<const float *>(smem + Lyt.wst);
    const bool reads_w = a.mode == PASS_HALS || a.mode == PASS_GIVEN_W;
    float *gsm = reinterpret_cast<float *>(smem + Lyt.gsm);
    float *invd = reinterpret_cast<float *>(smem + Lyt.invd);
    float *wsc = reinterpret_cast<float *>(smem + Lyt.wsc);
    float *ssqs = reinterpret_cast<float *>(smem + Lyt.ssq);
    float *gwx = reinterpret_cast<float *>(smem + Lyt.gwx);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + Lyt.bars);
    uint64_t *empty = full + S;
    uint64_t *redfull = empty + S;
    uint64_t *wready = redfull + NB;
    const uint32_t RS = Lyt.rs;
    const uint32_t stage_bytes = kMmaRows * RS;

    // zero the ring (row padding must read as finite zeros), the staged w and the partials
    {
        uint4 *z = reinterpret_cast<uint4 *>(smem + Lyt.tiles);
        const size_t n = (Lyt.red + (size_t)NB * 64 * 16 * sizeof(float) - Lyt.tiles) / 16;
        for (size_t i = tid; i < n; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NT);
        }
        for (int i = 0; i < NB; ++i) {
            mbar_init(&redfull[i], NT);
            mbar_init(&wready[i], 1);
        }
        fence_mbar_init();
    }
    for (int i = tid; i < kMaxK * kMaxK; i += blockDim.x) gsm[i] = a.st->G[i];
    if (tid < kMaxK) {
        invd[tid] = a.st->invdiag[tid];
        wsc[tid] = a.st->wscale[tid];
    }
    __syncthreads();

    if (role == 2) {
        // ---------------- producer warp: one bulk copy per pixel row.  With LANES, lane r
        // issues row r (lane 8 the tile's W rows), so a tile's
        // copies leave in one warp instruction (the gain for the shorter bf16 rows);
        // otherwise lane 0 alone runs the ring and issues them in turn.
        constexpr bool LANES = MmaProducerLanes<TP>::V;
        if (!LANES && lane != 0) return;
        int s = 0;
        uint32_t par = 0;
        int64_t i = 0;
        int64_t r0 = (int64_t)blockIdx.x * kMmaRows;
        const int64_t rstep = (int64_t)gridDim.x * kMmaRows;
        // a staged row holds the bins the consumers read (RS bytes, the first Nk live);
        // when P's rows are exactly RS bytes apart a full tile is one contiguous copy
        const uint32_t row_bytes = (uint32_t)min((size_t)a.ldP * ES, (size_t)RS);
        const bool one_copy = (size_t)a.ldP * ES == (size_t)RS;
        for (; i < my_tiles; ++i, r0 += rstep) {
            bool ok = true;
            if (lane == 0 && i >= S) ok = mbar_wait_bounded(&empty[s], par ^ 1u);
            if constexpr (LANES) ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) report(a.status, FHR_ERR_TIMEOUT);
                break;
            }
            const int rows = (int)((a.Np - r0) < kMmaRows ? (a.Np - r0) : kMmaRows);
            // the W rows of a full tile travel with it (8 K floats: a multiple of 16 bytes)
            const uint32_t wbytes = (reads_w && rows == kMmaRows) ? (uint32_t)(kMmaRows * K * sizeof(float)) : 0u;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)rows * row_bytes + wbytes);
            unsigned char *dst = smem + Lyt.tiles + (size_t)s * stage_bytes;
            const TP *src = reinterpret_cast<const TP *>(a.P) + r0 * a.ldP;
            // (no L2 prefetch of later tiles: measured 4.82 -> 4.45 ms per pass without it on
            // 7.86M x 1504 bf16 rows; prefetching two or three rings ahead was slower still)
            if constexpr (LANES) {
                __syncwarp();
                if (one_copy && rows == kMmaRows) {
                    if (lane == 0) bulk_g2s(dst, src, kMmaRows * RS, &full[s]);
                } else if (lane < rows) {
                    bulk_g2s(dst + (size_t)lane * RS, src + (size_t)lane * a.ldP, row_bytes, &full[s]);
                }
                if (lane == kMmaRows) {
                    if (wbytes)
                        bulk_g2s(smem + Lyt.wst + (size_t)s * kMmaRows * kMaxK * sizeof(float), a.W + r0 * K, wbytes,
                                 &full[s]);
                }
            } else {
                if (one_copy && rows == kMmaRows)
                    bulk_g2s(dst, src, kMmaRows * RS, &full[s]);
                else
                    for (int r = 0; r < rows; ++r)
                        bulk_g2s(dst + (size_t)r * RS, src + (size_t)r * a.ldP, row_bytes, &full[s]);
                if (wbytes)
                    bulk_g2s(smem + Lyt.wst + (size_t)s * kMmaRows * kMaxK * sizeof(float), a.W + r0 * K, wbytes,
                             &full[s]);
            }
            if (++s == S) {
                s = 0;
                par ^= 1u;
            }
        }
        if (lane == 0)
            for (int64_t j = (i > S ? i - S : 0); j < i; ++j)
                if (!mbar_wait_bounded(&full[(int)(j % S)], (uint32_t)((j / S) & 1))) report(a.status, FHR_ERR_TIMEOUT);
        return;
    }

    if (role == 1) {
        // ---------------- update warps: warp u takes the tiles i with i % 2 == u;
        // lane = (row, group of 4 partial sums)
        const int uw = warp;   // 0 .. NU - 1
        const int row = lane >> 2, grp = lane & 3;
        const int lmat = lane >> 3;
        float gw[4] = {0.f, 0.f, 0.f, 0.f};   // G_W of this warp's tiles (rows s and s + 8 of the accumulator)
        // G (constant for the launch): upper triangle in registers
        float gu[kMaxK * (kMaxK + 1) / 2];
        {
            int p = 0;
#pragma unroll
            for (int s = 0; s < kMaxK; ++s)
#pragma unroll
                for (int t = s; t < kMaxK; ++t, ++p) gu[p] = gsm[s * kMaxK + t];
        }
        float iv[kMaxK], sc[kMaxK];
#pragma unroll
        for (int s = 0; s < kMaxK; ++s) {
            iv[s] = invd[s];
            sc[s] = wsc[s];
        }
        int su = uw % S;   // NU < S: the ring holds at least LAG + 2 stages
        uint32_t paru = 0;
        for (int64_t i = uw; i < my_tiles; i += NU) {
            const int b = (int)(i % NB);
            const uint32_t hpar = (uint32_t)((i / NB) & 1);
            const int64_t r0 = (blockIdx.x + i * gridDim.x) * kMmaRows;
            const int rows = (int)((a.Np - r0) < kMmaRows ? (a.Np - r0) : kMmaRows);
            // the tile's W rows arrive with its data: read them before waiting for phase 1
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[su], paru))) {   // warp-uniform exit
                report(a.status, FHR_ERR_TIMEOUT);
                break;
            }
            const bool live = row < rows;
            float w[kMaxK];
#pragma unroll
            for (int s = 0; s < kMaxK; ++s) w[s] = 0.f;
            if (reads_w && live) {
                if (rows == kMmaRows) {
#pragma unroll
                    for (int s = 0; s < kMaxK; ++s)
                        if (s < K) w[s] = wst[su * kMmaRows * kMaxK + row * K + s] * sc[s];
                } else {
#pragma unroll
                    for (int s = 0; s < kMaxK; ++s)
                        if (s < K) w[s] = a.W[(r0 + row) * K + s] * sc[s];
                }
            }
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&redfull[b], hpar))) {
                report(a.status, FHR_ERR_TIMEOUT);
                break;
            }
            su += NU;
            if (su >= S) {
                su -= S;
                paru ^= 1u;
            }
            // r[s] for this lane's row: the partials of warps 4 grp .. 4 grp + 3 (two
            // 16-byte loads each: s 0..3, 4..7), then the four groups combined by two exchanges
            float r[kMaxK];
#pragma unroll
            for (int s = 0; s < kMaxK; ++s) r[s] = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t ra = red_a + (uint32_t)(((b * 16 + 4 * grp + j) * 64 + row * 8) * 4);
                const float4 v0 = lds_f4(ra), v1 = lds_f4(ra + 16);
                r[0] += v0.x; r[1] += v0.y; r[2] += v0.z; r[3] += v0.w;
                r[4] += v1.x; r[5] += v1.y; r[6] += v1.z; r[7] += v1.w;
            }
#pragma unroll
            for (int s = 0; s < kMaxK; ++s) {
                if (s < K) {
                    r[s] += __shfl_xor_sync(0xffffffffu, r[s], 1);
                    r[s] += __shfl_xor_sync(0xffffffffu, r[s], 2);
                }
            }
            if (a.mode == PASS_HALS) {
                // Gauss-Seidel over s with u = G w kept current:
                // w_s <- max(0, w_s + (r_s - u_s) / G_ss), then u += G[:, s] (w_s' - w_s)
                float u[kMaxK];
#pragma unroll
                for (int s = 0; s < kMaxK; ++s) {
                    float acc = 0.f;
#pragma unroll
                    for (int t = 0; t < kMaxK; ++t) acc = fmaf(gu[mma_tri(s, t)], w[t], acc);
                    u[s] = acc;
                }
#pragma unroll
                for (int s = 0; s < kMaxK; ++s) {
                    if (s < K && iv[s] != 0.f) {
                        const float nw = fmaxf(0.f, fmaf(r[s] - u[s], iv[s], w[s]));
                        const float d = nw - w[s];
                        w[s] = nw;
#pragma unroll
                        for (int t = 0; t < kMaxK; ++t) u[t] = fmaf(gu[mma_tri(t, s)], d, u[t]);
                    }
                }
                if (live && grp == 0) {
#pragma unroll
                    for (int s = 0; s < kMaxK; ++s)
                        if (s < K) a.W[(r0 + row) * K + s] = w[s];
                }
            } else if (a.mode != PASS_GIVEN_W) {
#pragma unroll
                for (int s = 0; s < kMaxK; ++s) w[s] = r[s];
                if (a.mode == PASS_PROJECT_STORE && live && grp == 0) {
#pragma unroll
                    for (int s = 0; s < kMaxK; ++s)
                        if (s < K) a.W[(r0 + row) * K + s] = w[s] * sc[s];
                }
            }
#pragma unroll
            for (int s = 0; s < kMaxK; ++s)
                if (!live || s >= K) w[s] = 0.f;
            // stage w for phase 3 (this lane writes s = grp and s = grp + 4)
            const uint32_t wbb = wb_a + (uint32_t)(b * 2 * 8 * kMmaWbStride);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int s = grp + 4 * h;
                // w[s] by a static select: indexing w with the lane-dependent s would
                // place the whole array in local memory for the HALS loop above
                float v = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (grp == q) v = w[q + 4 * h];
                if (F32) {
                    const uint32_t big = tf32_big(v);
                    const uint32_t small = __float_as_uint(v - __uint_as_float(big));
                    const uint32_t off = (uint32_t)(s * kMmaWbStride + mma_perm_inv(row) * 4);
                    sts_u32(wbb + off, big);
                    sts_u32(wbb + 8 * kMmaWbStride + off, small);
                } else {
                    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
                    const uint32_t off = (uint32_t)(s * kMmaWbStride + row * 2);
                    sts_u16(wbb + off, __bfloat16_as_ushort(hi));
                    sts_u16(wbb + 8 * kMmaWbStride + off, __bfloat16_as_ushort(lo));
                }
            }
            __syncwarp();
            // G_W += w^T w on the tensor cores, from the staged fragments (read before the
            // hand-off releases the buffer):
            // f32  A = [w_big^T; w_small^T] (rows 0..7; 8..15), B = w_big, then A = w_big^T, B = w_small;
            // bf16 A = [w_hi^T | w_lo^T] along k, B = [w_hi; w_hi], then A = w_hi^T, B = w_lo
            uint32_t wB0, wB1, wS0, wS1;
            if (F32) {
                ldsm_x4(wbb + (uint32_t)((lmat >> 1) * 8 * kMmaWbStride + (lane & 7) * kMmaWbStride + (lmat & 1) * 16),
                        wB0, wB1, wS0, wS1);
            } else {
                ldsm_x2(wbb + (uint32_t)((lmat & 1) * 8 * kMmaWbStride + (lane & 7) * kMmaWbStride), wB0, wS0);
                wB1 = wS1 = 0u;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&wready[b]);
            if (F32) {
                mma_tf32(gw, wB0, wS0, wB1, wS1, wB0, wB1);
                mma_tf32(gw, wB0, 0u, wB1, 0u, wS0, wS1);
            } else {
                mma_bf16(gw, wB0, 0u, wS0, 0u, wB0, wB0);
                mma_bf16(gw, wB0, 0u, 0u, 0u, wS0, 0u);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) gwx[(uw * 32 + lane) * 4 + e] = gw[e];
        bar_sync(1, NT + NU * 32);
        if (uw == 0) {
            // G_W[s][t]: accumulator rows s (high part) and s + 8 (low part), column t
            const int g = lane >> 2, tig = lane & 3;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int t = 2 * tig + e;
                float v = 0.f;
#pragma unroll
                for (int u = 0; u < NU; ++u) v += gwx[(u * 32 + lane) * 4 + e] + gwx[(u * 32 + lane) * 4 + 2 + e];
                if (g < K && t < K) a.Gpart[(size_t)blockIdx.x * K * K + g * K + t] = v;
            }
        }
        if (uw == 0 && lane == 0 && a.want_ssq) {
            float acc = 0.f;
            for (int wp = 0; wp < CW; ++wp) acc += ssqs[wp];
            a.ssqpart[blockIdx.x] = acc;
        }
        return;
    }

    // ---------------- consumer warps
    const int c0 = warp * NKW;   // first bin of this warp
    // D^T fragments, the 16 x k operand of phase 1: rows 0..7 the high parts,
    // rows 8..15 the low parts, both in registers, [k-step][a0/a1, a2/a3]
    uint32_t da[KS][2];   // f32: big; bf16: hi
    // low parts in registers: bf16 as they are; f32 (TF32 remainders, below 2^-11 of
    // the value) rounded to bf16 and packed two to a register
    uint32_t dlr[KS][F32 ? 1 : 2];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (F32) {
                const int k = c0 + ks * 8 + tig + 4 * h;
                const float v = (g < K && k < a.Nk) ? (float)(a.D64[(size_t)k * K + g] * a.st->invn[g]) : 0.f;
                const uint32_t big = tf32_big(v);
                da[ks][h] = big;
                const uint32_t sb16 = (uint32_t)bf16_bits(v - __uint_as_float(big));
                dlr[ks][0] = h ? (dlr[ks][0] | (sb16 << 16)) : sb16;
            } else {
                const int k = c0 + ks * 16 + 2 * tig + 8 * h;
                float v0 = 0.f, v1 = 0.f;
                if (g < K && k < a.Nk) v0 = (float)(a.D64[(size_t)k * K + g] * a.st->invn[g]);
                if (g < K && k + 1 < a.Nk) v1 = (float)(a.D64[(size_t)(k + 1) * K + g] * a.st->invn[g]);
                const float h0 = __bfloat162float(__float2bfloat16_rn(v0));
                const float h1 = __bfloat162float(__float2bfloat16_rn(v1));
                da[ks][h] = pack_bf16(v0, v1);
                dlr[ks][h] = pack_bf16(v0 - h0, v1 - h1);
            }
        }
    }
    float Q[MB][4];
#pragma unroll
    for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int e = 0; e < 4; ++e) Q[m][e] = 0.f;
    float ssq = 0.f;
    bool ok = true;
    int s_cur = 0, s3 = 0;            // stages of the tiles in phase 1 and in phase 3
    uint32_t par_cur = 0;
    int b1 = 0, b3 = 0;               // hand-off buffers of the tiles in phase 1 and in phase 3
    uint32_t h1 = 0, h3 = 0;          // and their parities
    int64_t r0_cur = (int64_t)blockIdx.x * kMmaRows;
    const int64_t rstep = (int64_t)gridDim.x * kMmaRows;
    // ldmatrix row addresses: lane supplies row (lane & 7) of matrix (lane >> 3)
    const uint32_t lrow = (uint32_t)(lane & 7) * RS;
    const int lmat = lane >> 3;
    for (int64_t i = 0; i < my_tiles + LAG && ok; ++i) {
        if (i < my_tiles) {
            const int b = b1;
            if (!mbar_wait_bounded(&full[s_cur], par_cur)) {
                ok = false;
                break;
            }
            const int rows = (int)((a.Np - r0_cur) < kMmaRows ? (a.Np - r0_cur) : kMmaRows);
            const uint32_t tl = tiles_a + (uint32_t)s_cur * stage_bytes;
            // ---- phase 1: r^T (s x rows) += D^T (s x k) P^T (k x rows), two accumulators
            float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < KS; ks += 2) {
                // matrices: (k-step ks: b0, b1), (k-step ks+1: b0, b1)
                uint32_t p0, p1, p2, p3;
                ldsm_x4(tl + lrow + (uint32_t)((c0 + ks * MmaK<TP>::STEP) * ES + lmat * 16), p0, p1, p2, p3);
                if (a.want_ssq && g < rows) {
                    ssq = sq_acc<F32>(p0, sq_acc<F32>(p1, ssq));
                    if (ks + 1 < KS) ssq = sq_acc<F32>(p2, sq_acc<F32>(p3, ssq));
                }
                {   // k-step ks into accumulator 0
                    uint32_t dl0, dl1;
                    if constexpr (F32) {   // TF32 patterns of the bf16-rounded remainders
                        dl0 = dlr[ks][0] << 16;
                        dl1 = dlr[ks][0] & 0xffff0000u;
                    } else {
                        dl0 = dlr[ks][0];
                        dl1 = dlr[ks][F32 ? 0 : 1];
                    }
                    if (F32) {
                        uint32_t b0b, b0s, b1b, b1s;
                        tf32_split(p0, b0b, b0s);
                        tf32_split(p1, b1b, b1s);
                        // rows 0..7: D_big P_big; rows 8..15: D_small P_big; then rows 0..7 += D_big P_small
                        mma_tf32(acc0, da[ks][0], dl0, da[ks][1], dl1, b0b, b1b);
                        mma_tf32(acc0, da[ks][0], 0u, da[ks][1], 0u, b0s, b1s);
                    } else {
                        // rows 0..7: D_hi P; rows 8..15: D_lo P
                        mma_bf16(acc0, da[ks][0], dl0, da[ks][1], dl1, p0, p1);
                    }
                }
                if (ks + 1 < KS) {   // k-step ks + 1 into accumulator 1
                    const int k1 = ks + 1 < KS ? ks + 1 : 0;   // in range for the unrolled copy
                    uint32_t dl0, dl1;
                    if constexpr (F32) {
                        dl0 = dlr[k1][0] << 16;
                        dl1 = dlr[k1][0] & 0xffff0000u;
                    } else {
                        dl0 = dlr[k1][0];
                        dl1 = dlr[k1][F32 ? 0 : 1];
                    }
                    if (F32) {
                        uint32_t b0b, b0s, b1b, b1s;
                        tf32_split(p2, b0b, b0s);
                        tf32_split(p3, b1b, b1s);
                        mma_tf32(acc1, da[k1][0], dl0, da[k1][1], dl1, b0b, b1b);
                        mma_tf32(acc1, da[k1][0], 0u, da[k1][1], 0u, b0s, b1s);
                    } else {
                        mma_bf16(acc1, da[k1][0], dl0, da[k1][1], dl1, p2, p3);
                    }
                }
            }
            // partial r: rows s = g (high part) and g + 8 (low part) of the
            // accumulators, columns 2 tig and 2 tig + 1 (pixel rows) -> red[b][warp][row][s]
            {
                const uint32_t ra = red_a + (uint32_t)(((b * 16 + warp) * 64 + 2 * tig * 8 + g) * 4);
                sts_f32(ra, (acc0[0] + acc0[2]) + (acc1[0] + acc1[2]));
                sts_f32(ra + 8 * 4, (acc0[1] + acc0[3]) + (acc1[1] + acc1[3]));
            }
            mbar_arrive(&redfull[b]);
            if (++b1 == NB) {
                b1 = 0;
                h1 ^= 1u;
            }
            r0_cur += rstep;
            if (++s_cur == S) {
                s_cur = 0;
                par_cur ^= 1u;
            }
        }
        // ---- phase 3 of tile i - LAG: Q (k x s) += P^T (k x rows) w (rows x s)
        if (i >= LAG) {
            const int b = b3;
            if (!mbar_wait_bounded(&wready[b], h3)) {
                ok = false;
                break;
            }
            const uint32_t tl = tiles_a + (uint32_t)s3 * stage_bytes;
            const uint32_t wbb = wb_a + (uint32_t)(b * 2 * 8 * kMmaWbStride);
            // w as the k x 8 operand: f32 b0 = w[perm(tig)][g], b1 = w[perm(tig + 4)][g];
            // bf16 b0 = {w[2 tig][g], w[2 tig + 1][g]}, b1 = 0 (rows 8..15)
            uint32_t wB0, wB1, wS0, wS1;   // f32: big b0, big b1, small b0, small b1; bf16: hi b0, -, lo b0, -
            if (F32) {
                // matrices: big words 0-3, big words 4-7, small words 0-3, small words 4-7
                const uint32_t addr = wbb + (uint32_t)((lmat >> 1) * 8 * kMmaWbStride + (lane & 7) * kMmaWbStride +
                                                       (lmat & 1) * 16);
                ldsm_x4(addr, wB0, wB1, wS0, wS1);
            } else {
                const uint32_t addr = wbb + (uint32_t)((lmat & 1) * 8 * kMmaWbStride + (lane & 7) * kMmaWbStride);
                ldsm_x2(addr, wB0, wS0);
                wB1 = 0u;
                wS1 = 0u;
            }
#pragma unroll
            for (int m = 0; m < MB; ++m) {
                const int m0 = c0 + m * 16;
                if (F32) {
                    // A = P^T (16 bins x 8 k) with MMA row m <-> bin m0 + 2 (m % 8) + m / 8, so that
                    // a0, a1 (rows g, g + 8) are the adjacent bins m0 + 2g, m0 + 2g + 1 of pixel row
                    // perm(tig) (one 8-byte load) and a2, a3 the same bins of row perm(tig + 4)
                    uint32_t x0, x1, x2, x3;
                    lds_u2(tl + (uint32_t)mma_perm(tig) * RS + (uint32_t)((m0 + 2 * g) * 4), x0, x1);
                    lds_u2(tl + (uint32_t)mma_perm(tig + 4) * RS + (uint32_t)((m0 + 2 * g) * 4), x2, x3);
                    uint32_t b0_, s0_, b1_, s1_, b2_, s2_, b3_, s3_;
                    tf32_split(x0, b0_, s0_);
                    tf32_split(x1, b1_, s1_);
                    tf32_split(x2, b2_, s2_);
                    tf32_split(x3, b3_, s3_);
                    mma_tf32(Q[m], b0_, b1_, b2_, b3_, wB0, wB1);
                    mma_tf32(Q[m], b0_, b1_, b2_, b3_, wS0, wS1);
                    mma_tf32(Q[m], s0_, s1_, s2_, s3_, wB0, wB1);
                } else {
                    // A = P^T (16 bins x 16 k, k >= 8 zero): .trans of the 8 x 8 blocks
                    // (rows 0..7, bins m0..m0+7) and (rows 0..7, bins m0+8..m0+15)
                    uint32_t a0, a1;   // lanes 16..31 repeat the addresses of lanes 0..15
                    ldsm_x2_t(tl + lrow + (uint32_t)((m0 + (lmat & 1) * 8) * 2), a0, a1);
                    // k 0..7: the 8 rows against w_hi; k 8..15: the same rows against w_lo
                    mma_bf16(Q[m], a0, a1, a0, a1, wB0, wS0);
                }
            }
            mbar_arrive(&empty[s3]);
            if (++s3 == S) s3 = 0;
            if (++b3 == NB) {
                b3 = 0;
                h3 ^= 1u;
            }
        }
    }
    if (!ok) report(a.status, FHR_ERR_TIMEOUT);

    // per-CTA partials of Q: c0 = (MMA row g, s 2 tig), c1 = (.., 2 tig + 1), c2, c3 = row g + 8;
    // MMA row g is bin m0 + g (bf16) or m0 + 2g (f32), row g + 8 bin m0 + g + 8 or m0 + 2g + 1
#pragma unroll
    for (int m = 0; m < MB; ++m) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = c0 + m * 16 + (F32 ? 2 * g + (e >> 1) : g + (e >> 1) * 8);
            const int s = 2 * tig + (e & 1);
            if (k < a.Nk && s < K) a.Qpart[((size_t)blockIdx.x * a.Nk + k) * K + s] = Q[m][e];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
    if (lane == 0) ssqs[warp] = ssq;
    bar_sync(1, NT + NU * 32);
}

}  // namespace fhr
