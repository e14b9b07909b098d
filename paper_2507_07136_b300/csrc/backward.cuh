// backward.cuh -- launch interface of the gradient kernels.
#pragma once

#include "device.cuh"

namespace lsv2 {

struct SplatBwdArgs {
    lsv2_camera cam;
    const uint32_t* tile_ranges;
    const uint32_t* gauss_ids;
    const float* xy;
    const float* axes;
    const float* conic_o;
    const float* extent;
    const float* final_T;
    const uint32_t* n_last;
    const float* dcoeff;
    void* workspace;
    float* recs;      // set by the launcher (inside workspace)
    float* grad2d;    // set by the launcher (inside workspace): [n][8] du dv da db dc
    uint32_t* queue;  // set by the launcher (inside workspace): work items taken (persistent kernel)
    float* dw;
    float* dopacity;
    int num_sms;      // SMs of the device (grid of the persistent kernel)
};

struct ProjBwdArgs {
    lsv2_camera cam;
    int64_t n;
    const float* means;
    const float* scales;
    const float* quats;
    const uint8_t* flags;
    const float* grad2d;
    float* dmeans;
    float* dscales;
    float* dquats;
};

size_t splat_backward_workspace_bytes(int64_t n, int levels, int K);
bool splat_backward_supported(int levels, int K);
// The decode adjoint of the L1 loss on the tensor cores (backward_tc.cu): D a multiple of 128, at
// most 512.
bool l1_decode_backward_tc_supported(int D);
cudaError_t launch_l1_decode_backward_tc(int levels, int64_t P, int D, const float* W, const float* S,
                                         const float* target, float* loss, float* dW, float* dS, int num_sms,
                                         int32_t* status, cudaStream_t stream);
cudaError_t launch_splat_backward(int levels, int K, const SplatBwdArgs& args, const ProjBwdArgs& pargs,
                                  const uint8_t* idx, const float* w, cudaStream_t stream);

}  // namespace lsv2
