// Shared-memory staged gathers of the projector pair (A and A^T of Eq. recon),
// fed by tensor-map bulk copies (cp.async.bulk.tensor).
//
// The table-driven gathers of proj.cuh read every candidate value from L1/L2,
// one dependent load per weight.  These kernels stage what a block needs next
// in shared memory instead, several lines or views ahead, through a ring of
// mbarrier-tracked tensor copies issued by a producer warp:
//   forward   block = (view v, 32 consecutive rays, 64 channels).  Per image
//             line l (the axis most parallel to the rays) the rays' candidate
//             pixels lie in one run of at most 49 pixels (about 30 on
//             average); the run (boxes of {64 channels, 8 pixels} of the image,
//             as many as it needs) and the rays' table entries (weights, first
//             candidate) are copied in; each thread sums its ray's 2-4
//             candidates for its channels from shared memory;
//   backward  block = (8 x 8 pixel tile, 64 channels).  Per view v the tile's
//             footprint is at most 14 consecutive bins; that slab of the
//             sinogram (box {64 channels, 16 bins, 1}) and the tile's table
//             entries are copied in; each thread sums its pixel's 3 candidate
//             bins.  The MBIR form then applies the SQS update (mbir.cuh).
// Each output is summed over the same weights in the same order as the
// table-driven kernels (lines then candidates; views then candidates), so the
// two give the same bits.  Used when Wl and Nc are multiples of 4 (16-byte
// tensor strides); other shapes keep the table-driven kernels.
#pragma once

#include <cuda.h>   // CUtensorMap and its enums (types only; the encoder comes from the driver at run time)

#include "mbir.cuh"

namespace fhr {

constexpr int kTmaRays = 32;        // rays per forward block
constexpr int kTmaSpan = 56;        // pixels per staged line: >= ceil(31 sqrt 2) + 1 + 4
constexpr int kTmaRunBox = 8;       // pixels per tensor copy of a run (a run takes ceil(len / 8) copies)
constexpr int kTmaCw = 64;          // channels per block
constexpr int kTmaFwdStages = 6;
constexpr int kTmaTile = 8;         // backward tile side
constexpr int kTmaBins = 16;        // bins per staged view: >= ceil(7 sqrt 2) + 1 + 3
constexpr int kTmaBwdStages = 12;
// channel groups of 4 per thread: forward, plain backward, backward + SQS update
constexpr int kTmaFwdG = 1, kTmaBwdG = 2, kTmaUpdG = 2;
// largest image side and view count of the staged path (their run starts are kept in
// shared memory)
constexpr int kTmaMaxN = 4096, kTmaMaxNv = 8192;

// shared-memory bytes of one forward stage: image run, ray weights, first candidates
constexpr uint32_t kTmaFwdX = kTmaSpan * kTmaCw * 4;
constexpr uint32_t kTmaFwdStage = kTmaFwdX + kTmaRays * 16 + kTmaRays * 4;
// one backward stage: sinogram slab, tile table
constexpr uint32_t kTmaBwdS = kTmaBins * kTmaCw * 4;
constexpr uint32_t kTmaBwdStage = kTmaBwdS + kTmaTile * kTmaTile * 16;

static_assert(kTmaFwdX % 128 == 0 && kTmaFwdStage % 128 == 0 && kTmaBwdS % 128 == 0 && kTmaBwdStage % 128 == 0,
              "stages keep 128-byte alignment");

// stages, run starts, then the full and empty mbarriers
__host__ __device__ inline size_t tma_fwd_smem(int N) {
    return (size_t)kTmaFwdStages * kTmaFwdStage + (size_t)N * 4 + kTmaFwdStages * 16 + 16;
}
__host__ __device__ inline size_t tma_bwd_smem(int Nv) {
    return (size_t)kTmaBwdStages * kTmaBwdStage + (size_t)Nv * 4 + kTmaBwdStages * 16 + 16;
}

// ---- tensor copies (PTX): global -> this CTA's shared memory, completion on an mbarrier
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// After a timeout the block stops; before it exits, thread 0 waits (bounded) for
// the copies it issued into stages [from, to) so that none lands after exit.
__device__ __forceinline__ void tma_drain(uint64_t *bars, int S, int from, int to) {
    for (int l = from; l < to; ++l) mbar_wait_bounded(&bars[l % S], (uint32_t)((l / S) & 1));
}

// y[v][c][w] = sum over lines and candidates of A x (V non-null: y = V - A x).
// Block = (channel chunk, view, ray block), chunk-major.  Threads: 32 rays x
// TR consumers, TR = 64 / (4 G) (thread (r, t) holds channels w0 + 4 t + 4 TR g,
// g < G), then one producer warp whose lane 0 refills each stage as soon as
// every consumer warp has released it (full / empty mbarriers, no block-wide
// barrier inside the sweep).
template <int G>
__global__ void __launch_bounds__(kTmaRays * kTmaCw / (4 * G) + 32) proj_fwd_tma(
    const __grid_constant__ CUtensorMap mx_row, const __grid_constant__ CUtensorMap mx_col,
    const __grid_constant__ CUtensorMap mfw, const __grid_constant__ CUtensorMap mfws, const int *__restrict__ fspan,
    const uint8_t *__restrict__ rowmaj, float *__restrict__ y, const float *__restrict__ V, int N, int Nc, int Nv,
    int Wl, int *status) {
    constexpr int TR = kTmaCw / (4 * G);
    constexpr int NT = kTmaRays * TR;   // consumer threads
    constexpr int S = kTmaFwdStages;
    extern __shared__ __align__(128) unsigned char smem[];
    int *sstart = reinterpret_cast<int *>(smem + (size_t)S * kTmaFwdStage);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * kTmaFwdStage + (((size_t)N * 4 + 7) & ~(size_t)7));
    uint64_t *empty = full + S;

    const int NB = (Nc + kTmaRays - 1) / kTmaRays;
    int bid = blockIdx.x;
    const int chunk = bid / (Nv * NB);
    bid -= chunk * Nv * NB;
    const int v = bid / NB, b = bid - v * NB;
    const int w0 = chunk * kTmaCw;
    const int tid = threadIdx.x;

    for (int l = tid; l < N; l += NT + 32) sstart[l] = fspan[((size_t)v * NB + b) * N + l];
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= NT) {
        // ---- producer: lane 0 of the last warp
        if (tid != NT) return;
        const bool rows = rowmaj[v] != 0;
        int l = 0;
        for (; l < N; ++l) {
            const int st = l % S;
            if (l >= S && !mbar_wait_bounded(&empty[st], (uint32_t)((l / S - 1) & 1))) {
                report(status, FHR_ERR_TIMEOUT);
                break;
            }
            unsigned char *base = smem + (size_t)st * kTmaFwdStage;
            const int s0 = sstart[l] & 0xffff;
            const int nbox = min((sstart[l] >> 16) + kTmaRunBox - 1, kTmaSpan) / kTmaRunBox;
            mbar_arrive_expect_tx(&full[st], (uint32_t)(nbox * kTmaRunBox * kTmaCw * 4 + kTmaRays * 20));
            for (int q = 0; q < nbox; ++q) {
                unsigned char *dst = base + (size_t)q * kTmaRunBox * kTmaCw * 4;
                if (rows) tma_load_3d(dst, &mx_row, w0, s0 + q * kTmaRunBox, l, &full[st]);
                else tma_load_3d(dst, &mx_col, w0, l, s0 + q * kTmaRunBox, &full[st]);
            }
            tma_load_2d(base + kTmaFwdX, &mfw, b * kTmaRays * 4, v * N + l, &full[st]);
            tma_load_2d(base + kTmaFwdX + kTmaRays * 16, &mfws, b * kTmaRays, v * N + l, &full[st]);
        }
        tma_drain(full, S, l > S ? l - S : 0, l);   // no copy lands after this thread exits
        return;
    }

    // ---- consumers
    const int lane = tid & 31;
    const int r = tid / TR, t = tid - r * TR;
    const int c = b * kTmaRays + r;
    const bool live = c < Nc;
    float4 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int l = 0; l < N; ++l) {
        const int st = l % S;
        const unsigned char *base = smem + (size_t)st * kTmaFwdStage;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[st], (uint32_t)((l / S) & 1)))) {
            if (lane == 0) report(status, FHR_ERR_TIMEOUT);
            return;   // the producer drains what it issued
        }
        if (live) {
            const float4 w = reinterpret_cast<const float4 *>(base + kTmaFwdX)[r];
            const int run = sstart[l];
            const int s = reinterpret_cast<const int *>(base + kTmaFwdX + kTmaRays * 16)[r] - (run & 0xffff);
            if (s >= 0 && s + 4 <= min(run >> 16, kTmaSpan)) {
                const float *xs = reinterpret_cast<const float *>(base) + (size_t)s * kTmaCw + 4 * t;
                if (w.x != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g) VecF<4>::fma(acc[g], w.x, *reinterpret_cast<const float4 *>(xs + 4 * TR * g));
                }
                if (w.y != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.y, *reinterpret_cast<const float4 *>(xs + kTmaCw + 4 * TR * g));
                }
                if (w.z != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.z, *reinterpret_cast<const float4 *>(xs + 2 * kTmaCw + 4 * TR * g));
                }
                if (w.w != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.w, *reinterpret_cast<const float4 *>(xs + 3 * kTmaCw + 4 * TR * g));
                }
            } else {
                report(status, FHR_ERR_UNSUPPORTED);   // a run wider than the staged box
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
    if (!live) return;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int w = w0 + 4 * t + 4 * TR * g;
        if (w >= Wl) continue;
        const size_t o = ((size_t)v * Nc + c) * Wl + w;
        float4 a = acc[g];
        if (V) {
            const float4 vv = *reinterpret_cast<const float4 *>(V + o);
            a = make_float4(vv.x - a.x, vv.y - a.y, vv.z - a.z, vv.w - a.w);
        }
        *reinterpret_cast<float4 *>(y + o) = a;
    }
}

// Arguments of the fused SQS update (the MBIR form of the backward gather).
struct TmaUpdate {
    const float *z, *xprev;
    float *znext;
    const float *dA;
    const MbirChan *chp;
    MbirPrior pr;
    float mom_a;
    int Nr, K;
};

// Backward gather over 8 x 8 pixel tiles: x[pix][w] = sum over views and
// candidate bins of A y (UPDATE: the SQS step from z, written to xout, with
// the momentum point when u.znext is set).  Block = (channel chunk, tile),
// chunk-major.  Threads: 64 pixels x TP consumers, TP = 64 / (4 G), then one
// producer warp (full / empty mbarriers as in the forward gather).
template <int G, bool UPDATE>
__global__ void __launch_bounds__(kTmaTile * kTmaTile * kTmaCw / (4 * G) + 32, UPDATE ? 2 : 1) proj_bwd_tma(
    const __grid_constant__ CUtensorMap msino, const __grid_constant__ CUtensorMap mbk, const int *__restrict__ bspan,
    float *__restrict__ xout, TmaUpdate u, int N, int Nc, int Nv, int Wl, int bins_box, int *status) {
    constexpr int TP = kTmaCw / (4 * G);
    constexpr int NT = kTmaTile * kTmaTile * TP;   // consumer threads
    constexpr int S = kTmaBwdStages;
    extern __shared__ __align__(128) unsigned char smem[];
    int *bstart = reinterpret_cast<int *>(smem + (size_t)S * kTmaBwdStage);
    uint64_t *full =
        reinterpret_cast<uint64_t *>(smem + (size_t)S * kTmaBwdStage + (((size_t)Nv * 4 + 7) & ~(size_t)7));
    uint64_t *empty = full + S;

    const int NTX = (N + kTmaTile - 1) / kTmaTile;
    const int ntiles = NTX * NTX;
    const int chunk = blockIdx.x / ntiles;
    const int tile = blockIdx.x - chunk * ntiles;
    const int ty = tile / NTX, tx0 = tile - ty * NTX;
    const int w0 = chunk * kTmaCw;
    const int tid = threadIdx.x;

    for (int vv = tid; vv < Nv; vv += NT + 32) bstart[vv] = bspan[(size_t)vv * ntiles + tile];
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= NT) {
        // ---- producer: lane 0 of the last warp
        if (tid != NT) return;
        const uint32_t txb = (uint32_t)kTmaCw * bins_box * 4 + kTmaTile * kTmaTile * 16;
        int vv = 0;
        for (; vv < Nv; ++vv) {
            const int st = vv % S;
            if (vv >= S && !mbar_wait_bounded(&empty[st], (uint32_t)((vv / S - 1) & 1))) {
                report(status, FHR_ERR_TIMEOUT);
                break;
            }
            unsigned char *base = smem + (size_t)st * kTmaBwdStage;
            mbar_arrive_expect_tx(&full[st], txb);
            tma_load_3d(base, &msino, w0, bstart[vv], vv, &full[st]);
            tma_load_3d(base + kTmaBwdS, &mbk, tx0 * kTmaTile * 4, ty * kTmaTile, vv, &full[st]);
        }
        tma_drain(full, S, vv > S ? vv - S : 0, vv);   // no copy lands after this thread exits
        return;
    }

    // ---- consumers
    const int lane = tid & 31;
    const int p = tid / TP, t = tid - p * TP;
    const int py = p / kTmaTile, px = p - py * kTmaTile;
    const int iy = ty * kTmaTile + py, ix = tx0 * kTmaTile + px;
    const bool live = iy < N && ix < N;
    float4 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int vv = 0; vv < Nv; ++vv) {
        const int st = vv % S;
        const unsigned char *base = smem + (size_t)st * kTmaBwdStage;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[st], (uint32_t)((vv / S) & 1)))) {
            if (lane == 0) report(status, FHR_ERR_TIMEOUT);
            return;   // the producer drains what it issued
        }
        if (live) {
            const float4 w = reinterpret_cast<const float4 *>(base + kTmaBwdS)[p];
            const int s = (int)w.w - bstart[vv];
            if (s >= 0 && s <= bins_box - 3) {
                const float *ys = reinterpret_cast<const float *>(base) + (size_t)s * kTmaCw + 4 * t;
                if (w.x != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g) VecF<4>::fma(acc[g], w.x, *reinterpret_cast<const float4 *>(ys + 4 * TP * g));
                }
                if (w.y != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.y, *reinterpret_cast<const float4 *>(ys + kTmaCw + 4 * TP * g));
                }
                if (w.z != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.z, *reinterpret_cast<const float4 *>(ys + 2 * kTmaCw + 4 * TP * g));
                }
            } else {
                report(status, FHR_ERR_UNSUPPORTED);   // a footprint wider than the staged slab
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }
    if (!live) return;
    const int pix = iy * N + ix;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int w = w0 + 4 * t + 4 * TP * g;
        if (w >= Wl) continue;
        if constexpr (UPDATE) {
            mbir_update_group<4, false>(acc[g], u.z, u.xprev, xout, u.znext, u.dA, u.chp, u.pr, u.mom_a, N, Nc, Nv,
                                        u.Nr, u.K, Wl, pix, w);
        } else {
            *reinterpret_cast<float4 *>(xout + (size_t)pix * Wl + w) = acc[g];
        }
    }
}

// run starts of the staged gathers: fspan[v][ray block][line] = the first candidate of
// the block's first ray that the block reads in that line (the smallest over its rays);
// bspan[v][tile] = the smallest first candidate bin over the tile's pixels
__global__ void proj_span_fw(const ProjTables t, int N, int Nc, int Nv, int *fspan);
__global__ void proj_span_bk(const ProjTables t, int N, int Nc, int Nv, int *bspan);

// Tensor-map path available for this shape (16-byte strides) and driver?
bool tma_gathers_ok(const fhr_geom *g, int Wl);
fhr_status tma_forward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *x, float *y,
                       const float *V, int *status);
fhr_status tma_backward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *y, float *x,
                        const TmaUpdate *upd, int *status);

}  // namespace fhr
