// query_tc.cuh -- launch interface of the tensor-core (tcgen05) relevancy kernel.
#pragma once

#include "device.cuh"

namespace lsv2 {

constexpr int kMaxQueryViews = 64;

struct QuerySeg {
    int64_t P;          // pixels of this view
    int64_t tile_base;  // first 128-pixel tile of this view (per level)
    size_t w_off;       // floats: this view's coefficient map
    size_t rel_off;     // elements: this view's relevancy block [Q][levels][P_v]
};

// Q queries of 1 + n_neg texts each: 64 + (1 + n_neg) * ceil(Q / 8) * 8 <= 512 and shared memory.
bool query_tc_supported(int Q, int n_neg);
// W: [levels][P][64] coefficient maps, BF16 when w_bf16 else FP32 (the views concatenated).
cudaError_t launch_query_tc_views(int levels, int V, const int64_t* P, int Q, int n_neg, float tau, const void* W,
                                  bool w_bf16, const float* Bt, const float* tnorm, void* rel, bool rel_bf16,
                                  int num_sms, int32_t* status, cudaStream_t stream);
cudaError_t launch_query_tc(int levels, int64_t P, int Q, int n_neg, float tau, const void* W, bool w_bf16,
                            const float* Bt, const float* tnorm, void* rel, bool rel_bf16, int num_sms,
                            int32_t* status, cudaStream_t stream);

}  // namespace lsv2
