// gram.cuh -- the squared feature norm of the relevancy epilogues (Sec. 3.2 through Eq. 7).
//
// |F|^2 = W^T (S S^T) W.  Once per call S S^T is factored as C C^T (C lower triangular:
// query_factor_kernel), the tensor-core product writes the 64 columns Y = W C beside the text
// columns, and |F|^2 = |Y|^2: a sum of squares of TMEM values, with no second read of W.
#pragma once

#include "device.cuh"

namespace lsv2 {

// Sum of the squares of 32 TMEM columns (FP32 bit patterns) in one fixed order: eight chains of
// four, added pairwise.  Every relevancy kernel forms |F|^2 as sumsq32(columns 0..31) +
// sumsq32(columns 32..63), so all of them (and both halves of a split epilogue) agree bit for bit.
__device__ __forceinline__ float sumsq32(const uint32_t (&y)[32])
{
    float acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float v = __uint_as_float(y[i]);
        acc[i] = v * v;
    }
#pragma unroll
    for (int j = 8; j < 32; ++j) {
        const float v = __uint_as_float(y[j]);
        acc[j & 7] = fmaf(v, v, acc[j & 7]);
    }
    return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

__device__ __forceinline__ float chol_norm2(const uint32_t (&y0)[32], const uint32_t (&y1)[32])
{
    return sumsq32(y0) + sumsq32(y1);
}

}  // namespace lsv2
