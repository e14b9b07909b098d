// mlp_fused.cuh -- launch interface of the fused tensor-core MLP decoder (mlp_fused.cu).
#pragma once

#include "device.cuh"

namespace lsv2 {

constexpr int kMlpMaxSub = 16;   // layers after the last one is cut into parts of <= 256 outputs

// One product of the chain as the kernel runs it: a hidden layer, or a part of the last layer.
struct MlpSub {
    int K;        // input width (activation columns read)
    int Kp;       // K rounded up to 16 (the MMA's K step)
    int N;        // outputs of this part, a multiple of 16 in [16, 256]
    int nkb;      // 64-column K blocks (weight chunks) = ceil(Kp / 64)
    int w_off;    // byte offset of its first chunk in the packed weight image
    int b_off;    // element offset of its first bias
    int out_col;  // first output column it produces (parts of the last layer), else 0
    int relu;     // 1: hidden (ReLU, result kept on chip), 0: the last layer (written out)
    int n_full;   // output width of the caller's layer it belongs to
    int64_t w_src;   // element offset of that layer's matrix in the caller's weights
};

struct MlpPlan {
    int nsub, in_w, in_kp, out_w;
    int n_bias;   // biases of all layers (a multiple of 8)
    MlpSub L[kMlpMaxSub];
};

// The plan of the fused kernel for these widths (w_0 .. w_n), or false when it does not apply:
// w_0 a multiple of 8 up to 32, hidden widths multiples of 16 in [16, 256], the output width a
// multiple of 16, at most kMlpMaxSub parts, at most 4,800 biases in all (they are held in
// shared memory).  *image_bytes: the packed weights' size.
bool mlp_fused_plan(int n_layers, const int32_t* widths, MlpPlan* plan, size_t* image_bytes);

// Packs the weights into `image` (device, 16-byte aligned, image_bytes) and runs the fused
// kernel over all rows.  A device wait that runs out records LSV2_ERR_TIMEOUT in *status.
cudaError_t launch_mlp_fused(const MlpPlan& plan, int64_t rows, const void* x, bool x_f32, const void* weights,
                             const void* biases, void* y, void* image, int32_t* status, cudaStream_t stream);

}  // namespace lsv2
