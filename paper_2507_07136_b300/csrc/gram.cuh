// gram.cuh -- the squared feature norm of the relevancy epilogues (Sec. 3.2 through Eq. 7):
// |F|^2 = W^T (S S^T) W from the Gram columns an MMA left in TMEM and the pixel's BF16 W row.
#pragma once

#include <cuda_bf16.h>

#include "device.cuh"

namespace lsv2 {

// |F|^2 = sum_j W_j Y_j over the 64 Gram columns Y = (W S S^T): W from this pixel's row of the
// swizzled BF16 tile, Y from TMEM (y0: columns 0..31, y1: 32..63).  Eight partial sums (eight
// independent FMA chains) are added pairwise.
__device__ __forceinline__ float gram_norm2(const uint8_t* sA, int row, const uint32_t (&y0)[32],
                                            const uint32_t (&y1)[32])
{
    float acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
        const uint4 wq = *reinterpret_cast<const uint4*>(sA + row * 128 + ((kc ^ (row & 7)) << 4));
        const uint32_t wv[4] = {wq.x, wq.y, wq.z, wq.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = kc * 8 + 2 * h;
            const __nv_bfloat162 w2 = *reinterpret_cast<const __nv_bfloat162*>(&wv[h]);
            const float ya = __uint_as_float(j < 32 ? y0[j & 31] : y1[j & 31]);
            const float yb = __uint_as_float(j + 1 < 32 ? y0[(j + 1) & 31] : y1[(j + 1) & 31]);
            acc[2 * h] = fmaf(__low2float(w2), ya, acc[2 * h]);
            acc[2 * h + 1] = fmaf(__high2float(w2), yb, acc[2 * h + 1]);
        }
    }
    return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

}  // namespace lsv2
