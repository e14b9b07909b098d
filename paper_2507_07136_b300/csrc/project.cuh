// project.cuh -- launch interface of the EWA projection kernel.
#pragma once

#include "device.cuh"

namespace lsv2 {

cudaError_t launch_project(const lsv2_camera& cam, int64_t n, const float* means, const float* scales,
                           const float* quats, const float* opacity, const lsv2_proj& out, int32_t* status,
                           cudaStream_t stream);

}  // namespace lsv2
