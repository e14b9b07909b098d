// query_tc.cuh -- launch interface of the tensor-core (tcgen05) relevancy kernel.
#pragma once

#include "device.cuh"

namespace lsv2 {

bool query_tc_supported(int nt);
cudaError_t launch_query_tc(int levels, int64_t P, int Q, int n_neg, float tau, const float* W, const float* Bt,
                            const float* tnorm, void* rel, bool rel_bf16, int num_sms, int32_t* status,
                            cudaStream_t stream);

}  // namespace lsv2
