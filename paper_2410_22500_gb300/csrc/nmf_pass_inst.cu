// Instantiations and launch dispatch of the fused NMF pass.
#include "nmf_pass.cuh"
#include "nmf_internal.h"

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
    CASE(1, 1) CASE(1, 2) CASE(1, 3) CASE(2, 1) CASE(2, 2) CASE(2, 3) CASE(3, 1) CASE(3, 2) CASE(3, 3)
    CASE(4, 1) CASE(4, 2) CASE(4, 3) CASE(5, 1) CASE(5, 2) CASE(5, 3) CASE(6, 1) CASE(6, 2) CASE(7, 1)
    CASE(7, 2) CASE(8, 1) CASE(8, 2)
    return nullptr;
}

template <>
PassFn<__nv_bfloat16> pick<__nv_bfloat16>(int K, int cpt) {
    using TP = __nv_bfloat16;
    CASE(1, 1) CASE(2, 1) CASE(3, 1) CASE(4, 1) CASE(5, 1) CASE(6, 1) CASE(7, 1) CASE(8, 1)
    return nullptr;
}
#undef CASE

static int max_cpt(int K, int vec) {
    // D and Q for the owned columns stay in registers: 2 * cpt * vec * K <= 128
    int c = 128 / (2 * vec * K);
    if (vec == 8) c = 1;
    return c < 1 ? 1 : (c > 3 ? 3 : c);
}

static size_t pass_smem(int K, int NT, int ldP, int esize, int stages) {
    const int ROWS = kPassRows, NW = NT / 32;
    size_t b = (size_t)stages * ROWS * ldP * esize;
    b += sizeof(float) * ((size_t)NW * ROWS * K + ROWS * K + K * K + 2 * K + ROWS * K * K);
    b = (b + 7) / 8 * 8 + 2 * stages * sizeof(uint64_t);
    return b;
}

fhr_status pass_config(fhr_ctx *ctx, int K, int Nk, int ldP, int p_dtype, PassConfig *cfg) {
    const int vec = p_dtype == FHR_BF16 ? 8 : 4;
    const int esize = p_dtype == FHR_BF16 ? 2 : 4;
    const int ncol = ldP / vec;
    // columns per thread: the largest count whose column balance is within 2% of the best
    int nts[4] = {0, 0, 0, 0};
    double effs[4] = {-1, -1, -1, -1}, best = -1;
    for (int cpt = 1; cpt <= max_cpt(K, vec); ++cpt) {
        int nt = (int)((cdiv(ncol, cpt) + 31) / 32 * 32);
        if (nt + 32 > 256) continue;
        nts[cpt] = nt;
        effs[cpt] = (double)ncol / ((double)nt * cpt);
        if (effs[cpt] > best) best = effs[cpt];
    }
    int best_cpt = 0, best_nt = 0;
    for (int cpt = 1; cpt <= 3; ++cpt)
        if (nts[cpt] && effs[cpt] >= best - 0.02) {
            best_cpt = cpt;
            best_nt = nts[cpt];
        }
    if (best_nt == 0) return set_error(ctx, FHR_ERR_UNSUPPORTED, "Nk too large for the fused pass");
    cfg->cpt = best_cpt;
    cfg->nt = best_nt;
    const size_t stage = (size_t)kPassRows * ldP * esize;
    const size_t budget = (size_t)ctx->max_smem_optin;
    int stages = 4;
    while (stages > 2 && pass_smem(K, best_nt, ldP, esize, stages) > budget) --stages;
    if (pass_smem(K, best_nt, ldP, esize, stages) > budget)
        return set_error(ctx, FHR_ERR_UNSUPPORTED, "Nk too large: a %zu-byte tile does not fit shared memory", stage);
    // prefer more resident CTAs over deeper rings when tiles are small
    cfg->stages = stages;
    cfg->smem = pass_smem(K, best_nt, ldP, esize, stages);
    const void *fn = p_dtype == FHR_BF16 ? (const void *)pick<__nv_bfloat16>(K, best_cpt)
                                         : (const void *)pick<float>(K, best_cpt);
    if (!fn) return set_error(ctx, FHR_ERR_UNSUPPORTED, "no pass kernel for K=%d", K);
    FHR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg->smem));
    int per_sm = 0;
    FHR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, best_nt + 32, cfg->smem));
    if (per_sm < 1) return set_error(ctx, FHR_ERR_UNSUPPORTED, "fused pass does not fit on an SM");
    cfg->grid = ctx->sm_count * per_sm;
    cfg->fn = fn;
    return FHR_OK;
}

fhr_status launch_pass(fhr_ctx *ctx, const PassConfig &cfg, const PassArgs &a) {
    PassArgs b = a;
    b.stages = cfg.stages;
    void *args[] = {&b};
    FHR_TIMED(TM_NMF_PASS, cudaLaunchKernel(cfg.fn, dim3(cfg.grid), dim3(cfg.nt + 32), args, cfg.smem, ctx->stream));
    return FHR_OK;
}

}  // namespace fhr
