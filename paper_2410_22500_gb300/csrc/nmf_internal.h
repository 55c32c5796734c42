// Internal interfaces between the NMF translation units.
#pragma once
#include "common.cuh"
#include "nmf_pass.cuh"

namespace fhr {

struct PassConfig {
    int cpt = 0, nt = 0, stages = 0, grid = 0, K = 0;
    size_t smem = 0;
    const void *fn = nullptr;
};

fhr_status pass_config(fhr_ctx *ctx, int K, int Nk, int ldP, int p_dtype, PassConfig *cfg);
fhr_status launch_pass(fhr_ctx *ctx, const PassConfig &cfg, const PassArgs &a);

}  // namespace fhr
