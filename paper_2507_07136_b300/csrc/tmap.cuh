// tmap.cuh -- host-side encoding of tiled TMA tensor maps (CUtensorMap) for the
// cp.async.bulk.tensor loads and stores of the tensor-core kernels.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace lsv2 {

// A 3-D row-major tensor of BF16 or FP32 elements with extents {d0 (innermost), d1, d2} and
// packed strides (d0 and d0 * d1 elements), moved in boxes of {b0, b1, 1} elements with the
// 128-byte swizzle (b0 * element size must be <= 128 and a multiple of 16).  Loads of
// coordinates outside the tensor read zeros; stores there write nothing.  `promote_l2`
// widens L2 fills of loads to 256 bytes.  Returns false if the driver rejects the map (base
// not 16-byte aligned, a stride not a multiple of 16 bytes, extents out of range) or the
// encoder entry point is not available.
bool encode_tmap_3d(CUtensorMap* map, const void* base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2,
                    uint32_t b0, uint32_t b1, bool promote_l2);

// The same for a 4-D tensor {d0, d1, d2, d3} in boxes of {b0, b1, 1, 1}.
bool encode_tmap_4d(CUtensorMap* map, const void* base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3,
                    uint32_t b0, uint32_t b1, bool promote_l2);

}  // namespace lsv2
