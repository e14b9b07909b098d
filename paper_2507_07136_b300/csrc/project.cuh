// project.cuh -- launch interface of the EWA projection kernel.
#pragma once

#include "device.cuh"

namespace lsv2 {

constexpr int kMaxProjectViews = 64;

// Projects n Gaussians for V cameras; outputs of view v are at [v * n, (v + 1) * n).
cudaError_t launch_project(const lsv2_camera* cams, int V, int64_t n, const float* means, const float* scales,
                           const float* quats, const float* opacity, const lsv2_proj& out, int32_t* status,
                           cudaStream_t stream);

}  // namespace lsv2
