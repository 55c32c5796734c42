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
//             average); the run (one box {64 channels, 24..56 pixels} of the
//             image, the smallest that holds it) and the rays' table entries
//             (weights, first candidate) are copied in; each thread sums its ray's 2-4
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

#include "mbir.cuh"
#include "tma.cuh"

namespace fhr {

constexpr int kTmaRays = 32;        // rays per forward block of one view (16 in blocks of 4 views)
constexpr int kTmaSpan = 56;        // pixels per staged line: >= ceil(31 sqrt 2) + 1 + 4
// a run of len pixels is copied as one box of the smallest height kTmaRunH[h] >= len
constexpr int kTmaRunMaps = 5;
__host__ __device__ constexpr int tma_run_height(int h) { return 24 + 8 * h; }   // 24, 32, 40, 48, 56
__host__ __device__ inline int tma_run_map(int len) { return len <= 24 ? 0 : min((len - 17) / 8, kTmaRunMaps - 1); }

// The image maps of the forward gather: box {64 channels, height, 1} over rows
// (row lines) and {64 channels, 1, height} (column lines), per run height.
struct TmaRunMaps {
    CUtensorMap row[kTmaRunMaps], col[kTmaRunMaps];
};
constexpr int kTmaCw = 64;          // channels per block
constexpr int kTmaFwdStages = 4;
constexpr int kTmaTile = 8;         // backward tile side
constexpr int kTmaBins = 16;        // bins per staged view: >= ceil(7 sqrt 2) + 1 + 3
constexpr int kTmaBwdStages = 12;
// zero-weight candidates skipped (a branch each) or summed (0 * x); the backward
// gather sums its first two candidates unconditionally
constexpr bool kTmaSkipZero = true;
// channel groups of 4 per thread: forward (one view per block, four views per
// block), plain backward, backward + SQS update
constexpr int kTmaFwdG = 1, kTmaFwdG4 = 4, kTmaBwdG = 2, kTmaUpdG = 4;
// largest image side and view count of the staged path (their run starts are kept in
// shared memory)
constexpr int kTmaMaxN = 4096, kTmaMaxNv = 8192;

// one backward stage: sinogram slab, tile table
constexpr uint32_t kTmaBwdS = kTmaBins * kTmaCw * 4;
constexpr uint32_t kTmaBwdStage = kTmaBwdS + kTmaTile * kTmaTile * 16;

static_assert(kTmaBwdS % 128 == 0 && kTmaBwdStage % 128 == 0, "stages keep 128-byte alignment");

// stages, run starts, then the full and empty mbarriers
__host__ __device__ inline size_t tma_bwd_smem(int Nv) {
    return (size_t)kTmaBwdStages * kTmaBwdStage + (size_t)Nv * 4 + kTmaBwdStages * 16 + 16;
}

// After a timeout the block stops; before it exits, thread 0 waits (bounded) for
// the copies it issued into stages [from, to) so that none lands after exit.
__device__ __forceinline__ void tma_drain(uint64_t *bars, int S, int from, int to) {
    for (int l = from; l < to; ++l) mbar_wait_bounded(&bars[l % S], (uint32_t)((l / S) & 1));
}

// Position in a ring of S stages, advanced one step at a time (no division in
// the loops): stage index and the parity of its current use.
struct Ring {
    int st = 0;
    uint32_t par = 0;
    __device__ __forceinline__ void next(int S) {
        if (++st == S) {
            st = 0;
            par ^= 1u;
        }
    }
};

// Forward block shapes: VG consecutive views x R rays.  Adjacent views see
// nearly the same pixels in a line (their runs differ by about (N/2) dtheta
// sqrt 2 pixels), so one staged run serves VG views' rays.
template <int VG, int R>
struct FwdShape {
    static constexpr int VR = VG * R;   // (view, ray) pairs per block
    static constexpr uint32_t X = kTmaSpan * kTmaCw * 4;
    static constexpr uint32_t STAGE = (X + VR * 20 + 127) / 128 * 128;
};

__host__ __device__ inline size_t tma_fwd_smem_vg(int vr, int N) {
    const size_t stage = ((size_t)kTmaSpan * kTmaCw * 4 + (size_t)vr * 20 + 127) / 128 * 128;
    return (size_t)kTmaFwdStages * stage + (size_t)2 * N * 4 + kTmaFwdStages * 16 + 16;
}

// y[v][c][w] = sum over lines and candidates of A x (V non-null: y = V - A x).
// Block = (channel chunk, group of VG views, block of R rays), chunk-major.
// Consumers: VG x R x TR threads, TR = 64 / (4 G) (thread (view, ray, t) holds
// G float4 groups of channels: w0 + 4 t + 4 TR g, g < G, the groups' order
// XOR-permuted between the rays of a quarter-warp), then one producer warp whose lane 0
// refills each stage once every consumer warp has released it (full / empty
// mbarriers, no block-wide barrier inside the sweep).  A group whose views do
// not share the line axis (it straddles 45 or 135 degrees) sweeps the lines
// twice, once per axis, each view's threads taking part in their axis's sweep.
// Each ray's sum runs over the lines in order, as in the table-driven gather.
template <int VG, int R, int G>
__global__ void __launch_bounds__(VG * R * kTmaCw / (4 * G) + 32) proj_fwd_tma(
    const __grid_constant__ TmaRunMaps mx, const __grid_constant__ CUtensorMap mfw,
    const __grid_constant__ CUtensorMap mfws, const int *__restrict__ fspan,
    const uint8_t *__restrict__ rowmaj, float *__restrict__ y, const float *__restrict__ V, int N, int Nc, int Nv,
    int Wl, int *status) {
    using SH = FwdShape<VG, R>;
    constexpr int TR = kTmaCw / (4 * G);
    constexpr int NT = VG * R * TR;   // consumer threads
    constexpr int S = kTmaFwdStages;
    extern __shared__ __align__(128) unsigned char smem[];
    int *sstart = reinterpret_cast<int *>(smem + (size_t)S * SH::STAGE);   // [pass][line]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * SH::STAGE + (size_t)2 * N * 4);
    uint64_t *empty = full + S;

    const int NB = (Nc + R - 1) / R;
    const int NG = (Nv + VG - 1) / VG;
    int bid = blockIdx.x;
    const int chunk = bid / (NG * NB);
    bid -= chunk * NG * NB;
    const int gi = bid / NB, b = bid - gi * NB;
    const int v0 = gi * VG;
    const int w0 = chunk * kTmaCw;
    const int tid = threadIdx.x;
    // sweeps: the axis of view v0, then (when some view of the group differs) the other
    const bool ax0 = rowmaj[v0] != 0;
    bool mixed = false;
#pragma unroll
    for (int q = 1; q < VG; ++q)
        if (v0 + q < Nv && (rowmaj[v0 + q] != 0) != ax0) mixed = true;
    const int npass = mixed ? 2 : 1;

    for (int i = tid; i < npass * N; i += NT + 32) {
        const int p = i / N, l = i - p * N;
        sstart[i] = fspan[(((size_t)gi * 2 + p) * NB + b) * N + l];
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int steps = npass * N;

    if (tid >= NT) {
        // ---- producer: lane 0 of the last warp
        if (tid != NT) return;
        int i = 0;
        Ring rg;
        for (; i < steps; ++i, rg.next(S)) {
            if (i >= S && !mbar_wait_bounded(&empty[rg.st], rg.par ^ 1u)) {
                report(status, FHR_ERR_TIMEOUT);
                break;
            }
            const int p = i >= N, l = i - p * N;
            const bool rows = p ? !ax0 : ax0;
            unsigned char *base = smem + (size_t)rg.st * SH::STAGE;
            const int s0 = sstart[i] & 0xffff;
            const int h = tma_run_map(sstart[i] >> 16);
            mbar_arrive_expect_tx(&full[rg.st], (uint32_t)(tma_run_height(h) * kTmaCw * 4 + SH::VR * 20));
            if (rows) tma_load_3d(base, &mx.row[h], w0, s0, l, &full[rg.st]);
            else tma_load_3d(base, &mx.col[h], w0, l, s0, &full[rg.st]);
            tma_load_3d(base + SH::X, &mfw, b * R * 4, l, v0, &full[rg.st]);
            tma_load_3d(base + SH::X + SH::VR * 16, &mfws, b * R, l, v0, &full[rg.st]);
        }
        tma_drain(full, S, i > S ? i - S : 0, i);   // no copy lands after this thread exits
        return;
    }
    // ---- consumers: thread (view q, ray r, channel group t)
    const int lane = tid & 31;
    const int q = tid / (R * TR);
    const int rr = tid - q * R * TR;
    const int r = rr / TR, t = rr - r * TR;
    const int v = v0 + q, c = b * R + r;
    const bool live = v < Nv && c < Nc;
    const bool my_axis = live && (rowmaj[v] != 0);   // true: row lines
    // channel offsets: the Q rays of a quarter-warp take their channel groups in
    // XOR-permuted order, so their float4 reads of different staged pixels fall in
    // disjoint banks
    constexpr int Q = TR >= 8 ? 1 : 8 / TR;
    int off[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) off[j] = 4 * t + 4 * TR * (j ^ (r & (Q - 1)));
    auto chan = [&](int g) { return off[g & (Q - 1)] + 4 * TR * (g & ~(Q - 1)); };
    float4 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    Ring rg;
    for (int i = 0; i < steps; ++i, rg.next(S)) {
        const int st = rg.st;
        const unsigned char *base = smem + (size_t)st * SH::STAGE;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[st], rg.par))) {
            if (lane == 0) report(status, FHR_ERR_TIMEOUT);
            return;   // the producer drains what it issued
        }
        const int p = i >= N;
        const bool active = live && (my_axis == (p ? !ax0 : ax0));
        if (active) {
            const float4 w = reinterpret_cast<const float4 *>(base + SH::X)[q * R + r];
            const int run = sstart[i];
            const int s = reinterpret_cast<const int *>(base + SH::X + SH::VR * 16)[q * R + r] - (run & 0xffff);
            if (s >= 0 && s + 4 <= min(run >> 16, kTmaSpan)) {
                const float *xs = reinterpret_cast<const float *>(base) + (size_t)s * kTmaCw;
                // (here every candidate keeps its zero-weight branch: summing the first two
                // unconditionally measured 3.69 -> 3.80 ms on the 256^3 shapes)
                if (!kTmaSkipZero || w.x != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g) VecF<4>::fma(acc[g], w.x, *reinterpret_cast<const float4 *>(xs + chan(g)));
                }
                if (!kTmaSkipZero || w.y != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.y, *reinterpret_cast<const float4 *>(xs + kTmaCw + chan(g)));
                }
                if (!kTmaSkipZero || w.z != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.z, *reinterpret_cast<const float4 *>(xs + 2 * kTmaCw + chan(g)));
                }
                if (!kTmaSkipZero || w.w != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.w, *reinterpret_cast<const float4 *>(xs + 3 * kTmaCw + chan(g)));
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
        const int w = w0 + chan(g);
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
// (the update form with 16 channels per thread, capped at 72 registers for 3 CTAs per SM:
// 4.86 -> 4.48 ms per iteration on the 256^3 shapes; 8 channels, 2 CTAs of 544 threads
// before; uncapped, 16 channels fit only 2 CTAs and took 5.0 ms)
__global__ void __launch_bounds__(kTmaTile * kTmaTile * kTmaCw / (4 * G) + 32, UPDATE ? 3 : 1) proj_bwd_tma(
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
        Ring rg;
        for (; vv < Nv; ++vv, rg.next(S)) {
            const int st = rg.st;
            if (vv >= S && !mbar_wait_bounded(&empty[st], rg.par ^ 1u)) {
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
    // channel offsets XOR-permuted over the Q pixels of a quarter-warp (as in the forward gather)
    constexpr int Q = TP >= 8 ? 1 : 8 / TP;
    int off[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) off[j] = 4 * t + 4 * TP * (j ^ (p & (Q - 1)));
    auto chan = [&](int g) { return off[g & (Q - 1)] + 4 * TP * (g & ~(Q - 1)); };
    float4 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    Ring rg;
    for (int vv = 0; vv < Nv; ++vv, rg.next(S)) {
        const int st = rg.st;
        const unsigned char *base = smem + (size_t)st * kTmaBwdStage;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[st], rg.par))) {
            if (lane == 0) report(status, FHR_ERR_TIMEOUT);
            return;   // the producer drains what it issued
        }
        if (live) {
            const float4 w = reinterpret_cast<const float4 *>(base + kTmaBwdS)[p];
            const int s = (int)w.w - bstart[vv];
            if (s >= 0 && s <= bins_box - 3) {
                const float *ys = reinterpret_cast<const float *>(base) + (size_t)s * kTmaCw;
                // the first two candidates are summed unconditionally (a zero weight adds
                // exact zeros, so the bits match the table-driven gather's skip): 4.84 ->
                // 4.73 ms per update on the 256^3 shapes
#pragma unroll
                for (int g = 0; g < G; ++g) VecF<4>::fma(acc[g], w.x, *reinterpret_cast<const float4 *>(ys + chan(g)));
#pragma unroll
                for (int g = 0; g < G; ++g)
                    VecF<4>::fma(acc[g], w.y, *reinterpret_cast<const float4 *>(ys + kTmaCw + chan(g)));
                if (!kTmaSkipZero || w.z != 0.f) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        VecF<4>::fma(acc[g], w.z, *reinterpret_cast<const float4 *>(ys + 2 * kTmaCw + chan(g)));
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
        const int w = w0 + chan(g);
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
__global__ void proj_span_fw(const ProjTables t, int N, int Nc, int Nv, int VG, int R, int *fspan);
__global__ void proj_span_bk(const ProjTables t, int N, int Nc, int Nv, int *bspan);

// Tensor-map path available for this shape (16-byte strides) and driver?
bool tma_gathers_ok(const fhr_geom *g, int Wl);
// Views per forward block: 4 (with 16 rays) when adjacent views' runs are known to
// overlap enough (default angles and N pi / Nv <= 8.95: the union run of 4 views x
// 16 rays stays within 50 pixels), else 1 (with 32 rays).
int tma_fwd_vg(const fhr_geom *g);
fhr_status tma_forward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *x, float *y,
                       const float *V, int *status);
fhr_status tma_backward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *y, float *x,
                        const TmaUpdate *upd, int *status);

}  // namespace fhr
