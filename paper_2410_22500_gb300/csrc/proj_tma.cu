// Host side of the staged gathers (proj_tma.cuh): run-start tables, tensor
// maps and launches.
#include <mutex>

#include "proj_tma.cuh"

namespace fhr {

__global__ void proj_span_fw(const ProjTables t, int N, int Nc, int Nv, int *fspan) {
    const int NB = (Nc + kTmaRays - 1) / kTmaRays;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Nv * NB * N) return;
    const int l = (int)(idx % N);
    const int b = (int)((idx / N) % NB);
    const int v = (int)(idx / ((int64_t)N * NB));
    const int *s0 = t.fws + ((size_t)v * N + l) * Nc;
    int lo = s0[b * kTmaRays], hi = lo;
    for (int c = b * kTmaRays + 1; c < min(Nc, (b + 1) * kTmaRays); ++c) {
        lo = min(lo, s0[c]);
        hi = max(hi, s0[c]);
    }
    fspan[idx] = lo | ((hi + 4 - lo) << 16);   // first pixel of the run, run length
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

// A tiled map over a row-major array: dims[0] innermost, strides in bytes of
// dims 1..rank-1, zero fill outside the array.
static bool make_map(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const uint64_t *dims,
                     const uint64_t *strides, const uint32_t *box) {
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
    return enc(m, dt, (cuuint32_t)rank, const_cast<void *>(base), d, s, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_gathers_ok(const fhr_geom *g, int Wl) {
    return Wl % 4 == 0 && g->Nc % 4 == 0 && g->N <= kTmaMaxN && g->Nv <= kTmaMaxNv && encoder() != nullptr;
}

fhr_status tma_forward(fhr_ctx *ctx, const fhr_geom *g, const ProjTables &t, int Wl, const float *x, float *y,
                       const float *V, int *status) {
    const int N = g->N, Nc = g->Nc, Nv = g->Nv;
    CUtensorMap mrow, mcol, mfw, mfws;
    {
        const uint64_t dims[3] = {(uint64_t)Wl, (uint64_t)N, (uint64_t)N};
        const uint64_t st[2] = {(uint64_t)Wl * 4, (uint64_t)N * Wl * 4};
        const uint32_t brow[3] = {kTmaCw, kTmaRunBox, 1}, bcol[3] = {kTmaCw, 1, kTmaRunBox};
        FHR_ARG(make_map(&mrow, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, x, dims, st, brow) &&
                    make_map(&mcol, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, x, dims, st, bcol),
                "tensor map of the image could not be encoded");
        const uint64_t dw[2] = {(uint64_t)Nc * 4, (uint64_t)Nv * N}, sw[1] = {(uint64_t)Nc * 16};
        const uint32_t bw[2] = {kTmaRays * 4, 1};
        const uint64_t ds[2] = {(uint64_t)Nc, (uint64_t)Nv * N}, ss[1] = {(uint64_t)Nc * 4};
        const uint32_t bs[2] = {kTmaRays, 1};
        FHR_ARG(make_map(&mfw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, t.fw, dw, sw, bw) &&
                    make_map(&mfws, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, t.fws, ds, ss, bs),
                "tensor map of the forward table could not be encoded");
    }
    const size_t smem = tma_fwd_smem(N);
    FHR_CUDA(cudaFuncSetAttribute(proj_fwd_tma<kTmaFwdG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int NB = (int)cdiv(Nc, kTmaRays);
    const unsigned blocks = (unsigned)((int64_t)cdiv(Wl, kTmaCw) * Nv * NB);
    FHR_TIMED(TM_PROJ_FWD, (proj_fwd_tma<kTmaFwdG><<<blocks, kTmaRays * kTmaCw / (4 * kTmaFwdG) + 32, smem, ctx->stream>>>(
                               mrow, mcol, mfw, mfws, t.fspan, t.rowmaj, y, V, N, Nc, Nv, Wl, status)));
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
