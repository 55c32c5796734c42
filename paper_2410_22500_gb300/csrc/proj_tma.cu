// Host side of the staged gathers (proj_tma.cuh): run-start tables, tensor
// maps and launches.
#include <mutex>

#include "proj_tma.cuh"

namespace fhr {

// packed run of block (group gi, sweep p, ray block b) in line l: first pixel |
// length << 16, over the group's views on sweep p's line axis and the block's rays
__global__ void proj_span_fw(const ProjTables t, int N, int Nc, int Nv, int VG, int R, int *fspan) {
    const int NB = (Nc + R - 1) / R, NG = (Nv + VG - 1) / VG;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)NG * 2 * NB * N) return;
    const int l = (int)(idx % N);
    const int b = (int)((idx / N) % NB);
    const int p = (int)((idx / ((int64_t)N * NB)) % 2);
    const int gi = (int)(idx / ((int64_t)N * NB * 2));
    const int v0 = gi * VG;
    const bool axis = p ? t.rowmaj[v0] == 0 : t.rowmaj[v0] != 0;
    int lo = 1 << 30, hi = -1;
    for (int v = v0; v < min(Nv, v0 + VG); ++v) {
        if ((t.rowmaj[v] != 0) != axis) continue;
        const int *s0 = t.fws + ((size_t)v * N + l) * Nc;
        for (int c = b * R; c < min(Nc, (b + 1) * R); ++c) {
            lo = min(lo, s0[c]);
            hi = max(hi, s0[c]);
        }
    }
    fspan[idx] = hi < 0 ? 0 : (lo | ((hi + 4 - lo) << 16));
}

__global__ void proj_span_bk(const ProjTables t, int N, int Nc, int Nv, int *bspan) {
    const int NTX = (N + kTmaTile - 1) / kTmaTile;
    const int ntiles = NTX * NTX;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Nv * ntiles) return;
    const int tile = (int)(idx % ntiles);
    const int v = (int)(idx / ntiles);
    const int ty = tile / NTX, tx = tile % NTX;
    int lo = Nc;
    for (int a = 0; a < kTmaTile; ++a)
        for (int q = 0; q < kTmaTile; ++q) {
            const int iy = ty * kTmaTile + a, ix = tx * kTmaTile + q;
            if (iy < N && ix < N) lo = min(lo, (int)t.bk[(size_t)v * N * N + (size_t)iy * N + ix].w);
        }
    bspan[idx] = lo;
}

// ---- tensor maps: cuTensorMapEncodeTiled is a driver entry point, fetched once
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

bool tma_available() { return encoder() != nullptr; }

bool tma_make_map(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const uint64_t *dims,
                  const uint64_t *strides, const uint32_t *box, CUtensorMapSwizzle swizzle) {
    EncodeTiledFn enc = encoder();
    if (!enc) return false;
    cuuint64_t d[5], s[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
    }
    for (int i = 0; i + 1 < rank; ++i) s[i] = strides[i];
    return enc(m, dt, (cuuint32_t)rank, const_cast<void *>(base), d, s, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool make_map(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const uint64_t *dims,
                     const uint64_t *strides, const uint32_t *box) {
    return tma_make_map(m, dt, rank, base, dims, strides, box);
}

int tma_fwd_vg(const fhr_geom *g) {
    return (g->angles == nullptr && (double)g->N * 3.141592653589793 / (double)g->Nv <= 8.95) ? 4 : 1;
}

bool tma_gathers_ok(const fhr_geom *g, int Wl) {
    return Wl % 4 == 0 && g->Nc % 4 == 0 && g->N <= kTmaMaxN && g->Nv <= kTmaMaxNv && tma_available();
}

fhr_status tma_forward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *x, float *y,
                       const float *V, int *status) {
    const int N = g->N, Nc = g->Nc, Nv = g->Nv;
    TmaRunMaps mx;
    CUtensorMap mfw, mfws;
    {
        const uint64_t dims[3] = {(uint64_t)Wl, (uint64_t)N, (uint64_t)N};
        const uint64_t st[2] = {(uint64_t)Wl * 4, (uint64_t)N * Wl * 4};
        for (int h = 0; h < kTmaRunMaps; ++h) {
            const uint32_t ht = (uint32_t)tma_run_height(h);
            const uint32_t brow[3] = {kTmaCw, ht, 1}, bcol[3] = {kTmaCw, 1, ht};
            FHR_ARG(make_map(&mx.row[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, x, dims, st, brow) &&
                        make_map(&mx.col[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, x, dims, st, bcol),
                    "tensor map of the image could not be encoded");
        }
        const int vg = tma_fwd_vg(g), rb = vg == 4 ? 16 : kTmaRays;
        const uint64_t dw[3] = {(uint64_t)Nc * 4, (uint64_t)N, (uint64_t)Nv};
        const uint64_t sw[2] = {(uint64_t)Nc * 16, (uint64_t)N * Nc * 16};
        const uint32_t bw[3] = {(uint32_t)rb * 4, 1, (uint32_t)vg};
        const uint64_t ds[3] = {(uint64_t)Nc, (uint64_t)N, (uint64_t)Nv};
        const uint64_t ss[2] = {(uint64_t)Nc * 4, (uint64_t)N * Nc * 4};
        const uint32_t bs[3] = {(uint32_t)rb, 1, (uint32_t)vg};
        FHR_ARG(make_map(&mfw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, t.fw, dw, sw, bw) &&
                    make_map(&mfws, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, t.fws, ds, ss, bs),
                "tensor map of the forward table could not be encoded");
    }
    const int64_t chunks = cdiv(Wl, kTmaCw);
    if (tma_fwd_vg(g) == 4) {
        constexpr int VG = 4, R = 16, G = kTmaFwdG4;
        const size_t smem = tma_fwd_smem_vg(VG * R, N);
        FHR_CUDA(cudaFuncSetAttribute(proj_fwd_tma<VG, R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const unsigned blocks = (unsigned)(chunks * cdiv(Nv, VG) * cdiv(Nc, R));
        FHR_TIMED(TM_PROJ_FWD, (proj_fwd_tma<VG, R, G><<<blocks, VG * R * kTmaCw / (4 * G) + 32, smem, ctx->stream>>>(
                                   mx, mfw, mfws, t.fspan, t.rowmaj, y, V, N, Nc, Nv, Wl, status)));
    } else {
        constexpr int VG = 1, R = kTmaRays, G = kTmaFwdG;
        const size_t smem = tma_fwd_smem_vg(VG * R, N);
        FHR_CUDA(cudaFuncSetAttribute(proj_fwd_tma<VG, R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const unsigned blocks = (unsigned)(chunks * Nv * cdiv(Nc, R));
        FHR_TIMED(TM_PROJ_FWD, (proj_fwd_tma<VG, R, G><<<blocks, VG * R * kTmaCw / (4 * G) + 32, smem, ctx->stream>>>(
                                   mx, mfw, mfws, t.fspan, t.rowmaj, y, V, N, Nc, Nv, Wl, status)));
    }
    return FHR_OK;
}

fhr_status tma_backward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *y, float *x,
                        const TmaUpdate *upd, int *status) {
    const int N = g->N, Nc = g->Nc, Nv = g->Nv;
    const int bins = std::min(kTmaBins, Nc);
    CUtensorMap ms, mb;
    {
        const uint64_t dims[3] = {(uint64_t)Wl, (uint64_t)Nc, (uint64_t)Nv};
        const uint64_t st[2] = {(uint64_t)Wl * 4, (uint64_t)Nc * Wl * 4};
        const uint32_t box[3] = {kTmaCw, (uint32_t)bins, 1};
        FHR_ARG(make_map(&ms, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, y, dims, st, box),
                "tensor map of the sinogram could not be encoded");
        const uint64_t db[3] = {(uint64_t)N * 4, (uint64_t)N, (uint64_t)Nv};
        const uint64_t sb[2] = {(uint64_t)N * 16, (uint64_t)N * N * 16};
        const uint32_t bb[3] = {kTmaTile * 4, kTmaTile, 1};
        FHR_ARG(make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, t.bk, db, sb, bb),
                "tensor map of the backward table could not be encoded");
    }
    const size_t smem = tma_bwd_smem(Nv);
    const int NTX = (int)cdiv(N, kTmaTile);
    const unsigned blocks = (unsigned)((int64_t)cdiv(Wl, kTmaCw) * NTX * NTX);
    if (upd) {
        FHR_CUDA(cudaFuncSetAttribute(proj_bwd_tma<kTmaUpdG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        FHR_TIMED(TM_MBIR_UPDATE,
                  (proj_bwd_tma<kTmaUpdG, true><<<blocks, kTmaTile * kTmaTile * kTmaCw / (4 * kTmaUpdG) + 32, smem,
                                                  ctx->stream>>>(ms, mb, t.bspan, x, *upd, N, Nc, Nv, Wl, bins,
                                                                 status)));
    } else {
        FHR_CUDA(cudaFuncSetAttribute(proj_bwd_tma<kTmaBwdG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        TmaUpdate none{};
        FHR_TIMED(TM_PROJ_BWD,
                  (proj_bwd_tma<kTmaBwdG, false><<<blocks, kTmaTile * kTmaTile * kTmaCw / (4 * kTmaBwdG) + 32, smem,
                                                   ctx->stream>>>(ms, mb, t.bspan, x, none, N, Nc, Nv, Wl, bins,
                                                                  status)));
    }
    return FHR_OK;
}

}  // namespace fhr
