// decode_tc.cuh -- launch interface of the tensor-core (tcgen05) decode.
#pragma once

#include "device.cuh"

namespace lsv2 {

bool decode_tc_supported(int D);
cudaError_t launch_decode_tc(int levels, int64_t P, int D, const void* W, bool w_bf16, const void* S, bool s_bf16,
                             void* F, bool out_bf16, int num_sms, int32_t* status, cudaStream_t stream);

}  // namespace lsv2
