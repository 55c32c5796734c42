// Tensor-map bulk copies (TMA): the device-side copy instructions and the host
// encoder of tiled tensor maps, shared by the staged projector gathers and the
// tensor-core MLP layers.
#pragma once

#include <cuda.h>   // CUtensorMap and its enums (types only; the encoder comes from the driver at run time)

#include "common.cuh"

namespace fhr {

// global -> this CTA's shared memory, completion on an mbarrier
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

// A tiled map over a row-major array: dims[0] innermost, strides in bytes of
// dims 1..rank-1, zero fill outside the array.  False when the driver has no
// encoder or rejects the map.
bool tma_make_map(CUtensorMap *m, CUtensorMapDataType dt, int rank, const void *base, const uint64_t *dims,
                  const uint64_t *strides, const uint32_t *box, CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE);
bool tma_available();

}  // namespace fhr
