// query.cuh -- launch interface of the relevancy kernels.
#pragma once

#include "device.cuh"

namespace lsv2 {

size_t query_workspace_bytes(int levels, int nt);
const float* query_ws_bt(const void* ws);
const float* query_ws_tnorm(const void* ws, int levels, int nt);
cudaError_t launch_query_prepare(int levels, int D, int nt, const float* S, const float* text, void* ws,
                                 cudaStream_t stream);
// In place on a prepared workspace: the Gram rows of B^T become the rows of C^T, S S^T = C C^T
// (the form the tensor-core relevancy kernels read).
cudaError_t launch_query_factor(int levels, int nt, void* ws, cudaStream_t stream);
cudaError_t launch_query_f32(int levels, int64_t P, int Q, int n_neg, float tau, const float* W, const void* ws,
                             float* rel, cudaStream_t stream);

}  // namespace lsv2
