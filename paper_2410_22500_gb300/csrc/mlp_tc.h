// Tensor-core (tcgen05) dense layer of the learned warm start's network:
// Act = GELU(A B^T + bias) in bf16 (and the FP32 pre-activation Z when set),
// A [M][Kd] bf16 rows (stride lda), B [N][Kd] bf16 weights (stride ldb), FP32
// accumulation in tensor memory.  Internal to libfhr.
#pragma once

#include "common.cuh"

namespace fhr {

struct TcGemmArgs {
    int M, N, Kd;
    const __nv_bfloat16 *A;
    int64_t lda;
    const __nv_bfloat16 *B;
    int64_t ldb;
    const float *bias;
    float *Z;   // optional [M][ldz]
    int64_t ldz;
    __nv_bfloat16 *Act;   // [M][ldact]
    int64_t ldact;
    int *status;          // device status word for expired waits (may be null)
};

// shapes the tcgen05 layer takes: 16 <= N <= 256, N % 16 == 0, 16-byte row strides
bool mlp_tc_ok(const TcGemmArgs &g);
fhr_status mlp_tc_layer(fhr_ctx *ctx, const TcGemmArgs &g);

}  // namespace fhr
