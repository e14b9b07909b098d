// decode.cu -- Eq. 7 decode F_lev = W_lev S_lev on CUDA cores in FP32.
//
// (P x 64) . (64 x D) per level.  A CTA computes a 128-pixel x 128-feature tile with the
// whole K = 64 reduction resident in shared memory (W tile stored transposed so a thread's
// 8 pixels are one 32-byte read); each thread accumulates an 8 x 8 block with FP32 FMA.
// Arithmetic intensity is 64 FMA per 4-byte output, so this form is bound by the FP32 pipe,
// not by HBM; the tensor-core form lives in decode_tc.cu.
#include "device.cuh"
#include "decode.cuh"

namespace lsv2 {
namespace {

constexpr int kTP = 128, kTD = 128, kL = 64;

__global__ void __launch_bounds__(256) decode_f32_kernel(int64_t P, int D, const float* __restrict__ W,
                                                         const float* __restrict__ S, float* __restrict__ F)
{
    __shared__ __align__(16) float As[kL][kTP + 4];
    __shared__ __align__(16) float Bs[kL][kTD];
    const int lev = blockIdx.z;
    const int64_t p0 = (int64_t)blockIdx.y * kTP;
    const int d0 = blockIdx.x * kTD;
    const int tid = threadIdx.x;
    const float* Wl = W + (size_t)lev * P * kL;
    const float* Sl = S + (size_t)lev * kL * D;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = tid + 256 * i;
        const int p = idx >> 4, c4 = (idx & 15) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p0 + p < P) v = __ldcs(reinterpret_cast<const float4*>(Wl + (p0 + p) * kL + c4));
        As[c4 + 0][p] = v.x;
        As[c4 + 1][p] = v.y;
        As[c4 + 2][p] = v.z;
        As[c4 + 3][p] = v.w;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = tid + 256 * i;
        const int l = idx >> 5, c4 = (idx & 31) * 4;
        *reinterpret_cast<float4*>(&Bs[l][c4]) = __ldg(reinterpret_cast<const float4*>(Sl + (size_t)l * D + d0 + c4));
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
    for (int l = 0; l < kL; ++l) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[l][ty * 8]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[l][ty * 8 + 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[l][tx * 8]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[l][tx * 8 + 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    float* Fl = F + (size_t)lev * P * D;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t p = p0 + ty * 8 + i;
        if (p < P) {
            float4* dst = reinterpret_cast<float4*>(Fl + p * D + d0 + tx * 8);
            __stcs(dst, make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]));
            __stcs(dst + 1, make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]));
        }
    }
}

}  // namespace

cudaError_t launch_decode_f32(int levels, int64_t P, int D, const float* W, const float* S, float* F,
                              cudaStream_t stream)
{
    if (P == 0 || levels == 0) return cudaSuccess;
    dim3 grid((unsigned)(D / kTD), (unsigned)((P + kTP - 1) / kTP), (unsigned)levels);
    decode_f32_kernel<<<grid, 256, 0, stream>>>(P, D, W, S, F);
    return cudaGetLastError();
}

}  // namespace lsv2
