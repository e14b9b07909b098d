// decode.cuh -- launch interface of the Eq. 7 decode kernels.
#pragma once

#include "device.cuh"

namespace lsv2 {

cudaError_t launch_decode_f32(int levels, int64_t P, int D, const float* W, const float* S, float* F,
                              cudaStream_t stream);

}  // namespace lsv2
