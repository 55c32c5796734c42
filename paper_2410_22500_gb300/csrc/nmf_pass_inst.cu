// Instantiations and launch configuration of the fused NMF pass: the
// tensor-core kernel (nmf_mma.cuh) up to 1664 (f32) / 2112 (bf16) bins per
// row (13 consumer warps x 128 / 12 x 176 bins), the CUDA-core kernel
// (nmf_pass.cuh) beyond.
#include "nmf_internal.h"
#include "nmf_mma.cuh"
#include "nmf_pass.cuh"

namespace fhr {

template <typename TP>
using PassFn = void (*)(PassArgs);

template <typename TP>
static PassFn<TP> pick(int K, int cpt);

#define CASE(K_, C_) \
    if (K == K_ && cpt == C_) return nmf_pass_kernel<K_, C_, TP>;

template <>
PassFn<float> pick<float>(int K, int cpt) {
    using TP = float;
    CASE(1, 1) CASE(1, 2) CASE(1, 3) CASE(1, 4) CASE(2, 1) CASE(2, 2) CASE(2, 3) CASE(2, 4)
    CASE(3, 1) CASE(3, 2) CASE(3, 3) CASE(3, 4) CASE(4, 1) CASE(4, 2) CASE(4, 3) CASE(4, 4)
    CASE(5, 1) CASE(5, 2) CASE(5, 3) CASE(6, 1) CASE(6, 2) CASE(6, 3) CASE(7, 1) CASE(7, 2) CASE(7, 3)
    CASE(8, 1) CASE(8, 2) CASE(8, 3)
    return nullptr;
}

template <>
PassFn<__nv_bfloat16> pick<__nv_bfloat16>(int K, int cpt) {
    using TP = __nv_bfloat16;
    CASE(1, 1) CASE(1, 2) CASE(2, 1) CASE(2, 2) CASE(3, 1) CASE(3, 2) CASE(4, 1) CASE(4, 2) CASE(5, 1) CASE(5, 2)
    CASE(6, 1) CASE(7, 1) CASE(8, 1)
    return nullptr;
}
#undef CASE

// pipeline lag of the tensor-core pass: phase 3 one tile behind phase 1 for f32
// rows (their ring holds only five 39 KB stages, so every stage not held for phase 3
// is one more tile in flight: 0.705 -> 0.693 ms on 737,280 x 1200 rows), three for
// bf16 rows, whose three update warps then each have three tile periods for their
// HALS step (a lag of two measured the same; one exceeds the update's latency)
template <typename TP>
struct MmaLag {
    static constexpr int V = sizeof(TP) == 2 ? 3 : 1;
};

template <typename TP>
static const void *pick_mma(int nkw) {
    constexpr int L = MmaLag<TP>::V;
    switch (nkw) {
        case 16: return (const void *)nmf_mma_kernel<TP, 16, L>;
        case 32: return (const void *)nmf_mma_kernel<TP, 32, L>;
        case 48: return (const void *)nmf_mma_kernel<TP, 48, L>;
        case 64: return (const void *)nmf_mma_kernel<TP, 64, L>;
        case 80: return (const void *)nmf_mma_kernel<TP, 80, L>;
        case 96: return (const void *)nmf_mma_kernel<TP, 96, L>;
        case 112: return (const void *)nmf_mma_kernel<TP, 112, L>;
        case 128: return (const void *)nmf_mma_kernel<TP, 128, L>;
        default: break;
    }
    if constexpr (sizeof(TP) == 2) {   // BF16 keeps fewer registers per bin
        switch (nkw) {
            case 144: return (const void *)nmf_mma_kernel<TP, 144, L>;
            case 160: return (const void *)nmf_mma_kernel<TP, 160, L>;
            case 176: return (const void *)nmf_mma_kernel<TP, 176, L>;
            default: break;
        }
    }
    return nullptr;
}

static fhr_status mma_config(fhr_ctx *ctx, int K, int Nk, int p_dtype, PassConfig *cfg) {
    const int esize = p_dtype == FHR_BF16 ? 2 : 4;
    const int cw = p_dtype == FHR_BF16 ? MmaCW<__nv_bfloat16>::V : MmaCW<float>::V;
    const void *fn = p_dtype == FHR_BF16 ? pick_mma<__nv_bfloat16>(mma_nkw(Nk, cw)) : pick_mma<float>(mma_nkw(Nk, cw));
    if (!fn) return FHR_ERR_UNSUPPORTED;
    const int nb = (p_dtype == FHR_BF16 ? MmaLag<__nv_bfloat16>::V : MmaLag<float>::V) + 1;
    int stages = 8;
    while (stages > nb + 1 && mma_smem_layout(Nk, esize, stages, nb, cw).total > (size_t)ctx->max_smem_optin)
        --stages;
    const size_t smem = mma_smem_layout(Nk, esize, stages, nb, cw).total;
    if (smem > (size_t)ctx->max_smem_optin) return FHR_ERR_UNSUPPORTED;
    FHR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FHR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMmaThreads, smem));
    if (per_sm < 1) return FHR_ERR_UNSUPPORTED;
    cfg->cpt = 0;
    cfg->nt = kMmaThreads - 64;
    cfg->stages = stages;
    cfg->smem = smem;
    cfg->grid = ctx->sm_count * per_sm;
    cfg->fn = fn;
    cfg->K = K;
    return FHR_OK;
}

// Columns per thread: Q for the owned columns stays in registers for the whole
// launch (cpt * vec * K floats); D is read from shared memory.
static int max_cpt(int K, int vec) {
    if (vec == 8) return K <= 5 ? 2 : 1;
    return K <= 4 ? 4 : 3;
}

static size_t pass_smem(int K, int NT, int ldP, int esize, int stages) {
    return pass_smem_layout(K, NT / 32, ldP, esize, stages).total;
}

fhr_status pass_config(fhr_ctx *ctx, int K, int Nk, int ldP, int p_dtype, PassConfig *cfg) {
    cfg->K = K;
    {
        const fhr_status st = mma_config(ctx, K, Nk, p_dtype, cfg);
        if (st == FHR_OK) return FHR_OK;
        if (st != FHR_ERR_UNSUPPORTED) return st;
    }
    const int vec = p_dtype == FHR_BF16 ? 8 : 4;
    const int esize = p_dtype == FHR_BF16 ? 2 : 4;
    const int ncol = ldP / vec;
    // columns per thread: the largest count whose column balance is within 2% of the best
    int nts[5] = {0, 0, 0, 0, 0};
    double effs[5] = {-1, -1, -1, -1, -1}, best = -1;
    for (int cpt = 1; cpt <= max_cpt(K, vec); ++cpt) {
        int nt = (int)((cdiv(ncol, cpt) + 31) / 32 * 32);
        if (nt + 64 > 256) continue;
        nts[cpt] = nt;
        effs[cpt] = (double)ncol / ((double)nt * cpt);
        if (effs[cpt] > best) best = effs[cpt];
    }
    int best_cpt = 0, best_nt = 0;
    for (int cpt = 1; cpt <= 4; ++cpt)
        if (nts[cpt] && effs[cpt] >= best - 0.02) {
            best_cpt = cpt;
            best_nt = nts[cpt];
        }
    if (best_nt == 0) return set_error(ctx, FHR_ERR_UNSUPPORTED, "Nk too large for the fused pass");
    cfg->cpt = best_cpt;
    cfg->nt = best_nt;
    const size_t stage = (size_t)kPassRows * ldP * esize;
    // two CTAs per SM when the ring fits half of the SM's shared memory
    // (each SM has ~228 KB; a CTA may use up to max_smem_optin)
    const size_t half = (size_t)ctx->max_smem_optin / 2 - 1024;
    int stages = 6;
    while (stages > 3 && pass_smem(K, best_nt, ldP, esize, stages) > half) --stages;
    if (pass_smem(K, best_nt, ldP, esize, stages) > half) {
        stages = 6;
        while (stages > 2 && pass_smem(K, best_nt, ldP, esize, stages) > (size_t)ctx->max_smem_optin) --stages;
    }
    if (pass_smem(K, best_nt, ldP, esize, stages) > (size_t)ctx->max_smem_optin)
        return set_error(ctx, FHR_ERR_UNSUPPORTED, "Nk too large: a %zu-byte tile does not fit shared memory", stage);
    cfg->stages = stages;
    cfg->smem = pass_smem(K, best_nt, ldP, esize, stages);
    const void *fn = p_dtype == FHR_BF16 ? (const void *)pick<__nv_bfloat16>(K, best_cpt)
                                         : (const void *)pick<float>(K, best_cpt);
    if (!fn) return set_error(ctx, FHR_ERR_UNSUPPORTED, "no pass kernel for K=%d", K);
    FHR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg->smem));
    int per_sm = 0;
    FHR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, best_nt + 64, cfg->smem));
    if (per_sm < 1) return set_error(ctx, FHR_ERR_UNSUPPORTED, "fused pass does not fit on an SM");
    cfg->grid = ctx->sm_count * per_sm;
    cfg->fn = fn;
    return FHR_OK;
}

fhr_status launch_pass(fhr_ctx *ctx, const PassConfig &cfg, const PassArgs &a) {
    PassArgs b = a;
    b.stages = cfg.stages;
    b.K = cfg.K;
    void *args[] = {&b};
    FHR_TIMED(a.mode == PASS_HALS ? TM_NMF_PASS : TM_NNDSVD_PASS,
              cudaLaunchKernel(cfg.fn, dim3(cfg.grid), dim3(cfg.nt + 64), args, cfg.smem, ctx->stream));
    return FHR_OK;
}

}  // namespace fhr

extern "C" fhr_status fhr_nmf_row_stride(int Nk, int p_dtype, int *ldP) {
    using namespace fhr;
    if (Nk < 1 || !ldP || (p_dtype != FHR_F32 && p_dtype != FHR_BF16)) return FHR_ERR_ARG;
    const bool bf = p_dtype == FHR_BF16;
    const int mult = bf ? 8 : 4, es = bf ? 2 : 4;
    const int plain = (Nk + mult - 1) / mult * mult;
    const int cw = bf ? MmaCW<__nv_bfloat16>::V : MmaCW<float>::V;
    const int nkw = mma_nkw(Nk, cw);
    const bool mma = bf ? pick_mma<__nv_bfloat16>(nkw) != nullptr : pick_mma<float>(nkw) != nullptr;
    int best = plain;
    if (mma) {
        const int rs = (int)mma_smem_layout(Nk, es, 2, 2, cw).rs;   // bytes of a staged row
        const int tile = rs / es;
        if (rs % es == 0 && tile % mult == 0 && (int64_t)(tile - Nk) * 20 <= Nk) best = tile;
    }
    *ldP = best;
    return FHR_OK;
}

