// query.cu -- relevancy scores (Sec. 3.2) through the linearity of Eq. 7.
//
// The rendered feature is F = W S, so for a text embedding t
//     <F, t> = W . (S t),     |F|^2 = W^T (S S^T) W,
// and the relevancy never needs the D-dim feature map.  Per level a small prepare kernel
// forms, accumulated in twice-FP32 precision and rounded to float, the columns of
//     B = [ S S^T | S t_0 | S t_1 | ... ]            (64 x (64 + #texts))
// and the text norms (for the tensor-core relevancy, query_factor_kernel then replaces the Gram
// rows by the rows of C^T, S S^T = C C^T); the FP32 kernel gives every (pixel, level) one thread that holds W in
// registers, forms y = W^T B column by column (B^T in shared memory, read as warp-wide
// broadcasts), |F|^2 = sum_j W_j y_j, and writes
//     rel = min_i softmax(tau [cos_pos, cos_neg_i])_0 = sigmoid(tau (cos_pos - max_i cos_neg_i)).
#include "device.cuh"
#include "query.cuh"

namespace lsv2 {
namespace {

constexpr int kL = 64;

// grid (64 + nt, levels), 256 threads: B^T[lev][j][k] = <x_j, S_k> with x_j = S_j (j < 64, Gram
// rows) or the text vector j - 64.  Thread (k = t % 64, part = t / 64) accumulates the terms
// d = 4 part + 16 i (+ 0..3) in Dot2 form; the four parts are added in FP64 and rounded to float.
// Also the text norms (level 0 only), the same way.
__global__ void __launch_bounds__(256) query_prepare_kernel(int D, int nt, const float* __restrict__ S,
                                                            const float* __restrict__ text,
                                                            float* __restrict__ Bt, float* __restrict__ tnorm)
{
    extern __shared__ float xs[];
    __shared__ double part_sum[4][kL];
    __shared__ double red[8];
    const int j = blockIdx.x, lev = blockIdx.y, t = threadIdx.x, k = t & 63, part = t >> 6;
    const int ncol = kL + nt;
    const float* Sl = S + (size_t)lev * kL * D;
    const float* x = j < kL ? Sl + (size_t)j * D : text + (size_t)(j - kL) * D;
    for (int d = t; d < D; d += 256) xs[d] = x[d];
    __syncthreads();
    const float* sk = Sl + (size_t)k * D;
    float hi = 0.0f, lo = 0.0f;
    for (int d = part * 4; d < D; d += 16) {
        const float4 s4 = __ldg(reinterpret_cast<const float4*>(sk + d));
        dot2_step(xs[d], s4.x, hi, lo);
        dot2_step(xs[d + 1], s4.y, hi, lo);
        dot2_step(xs[d + 2], s4.z, hi, lo);
        dot2_step(xs[d + 3], s4.w, hi, lo);
    }
    part_sum[part][k] = (double)hi + (double)lo;
    __syncthreads();
    if (part == 0)
        Bt[((size_t)lev * ncol + j) * kL + k] = (float)((part_sum[0][k] + part_sum[1][k]) + (part_sum[2][k] + part_sum[3][k]));
    if (lev == 0 && j >= kL) {
        float qh = 0.0f, ql = 0.0f;
        for (int d = t; d < D; d += 256) dot2_step(xs[d], xs[d], qh, ql);
        double q = (double)qh + (double)ql;
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if ((t & 31) == 0) red[t >> 5] = q;
        __syncthreads();
        if (t == 0) {
            double sum = 0.0;
            for (int w = 0; w < 8; ++w) sum += red[w];
            tnorm[j - kL] = (float)sqrt(sum);
        }
    }
}

// S S^T = C C^T with C lower triangular (Cholesky in FP32), one CTA of 256 threads per level.  In
// place: the 64 Gram rows of B^T (row j = G[j][0..63]) become the rows of C^T (row j holds C[k][j]
// at k, zero for k < j), the first 64 columns of B for the tensor-core relevancy, which then forms
// |F|^2 = W^T G W as |W C|^2, a sum of squares of its MMA's output.  Only the backward error
// matters for that quadratic form, and FP32 Cholesky's is far below the BF16 rounding of the
// operands.  A pivot at or below kPivotFloor times its diagonal entry of G (codebook row j within
// about 3e-3 of its length of the span of the rows before it, as for a repeated or zero row) gives
// a zero column; the factor then reproduces G to within about 3e-3 of sqrt(G_ii G_jj).
// Blocked by 8 columns, right-looking, in shared memory: per block one thread factors the 8 x 8
// diagonal block in registers, one thread per row below solves that row's 8 entries (forward
// substitution), and all threads subtract the block's outer products from the trailing lower
// triangle: three barriers per block, 24 in all.
constexpr float kPivotFloor = 1e-5f;
constexpr int kFb = 8;   // factor block

__global__ void __launch_bounds__(256) query_factor_kernel(int ncol, float* __restrict__ Bt)
{
    __shared__ float A[kL][kL + 1];   // lower triangle: G, updated in place into C
    __shared__ float gd[kL];          // diagonal of G (for the pivot floor)
    __shared__ float rinv[kL];        // 1 / C[j][j] (0 for a dropped pivot)
    const int t = threadIdx.x;
    float* G = Bt + (size_t)blockIdx.x * ncol * kL;
    for (int e = t; e < kL * kL; e += 256) A[e >> 6][e & 63] = G[e];
    __syncthreads();
    if (t < kL) gd[t] = A[t][t];
    __syncthreads();
#pragma unroll 1
    for (int j0 = 0; j0 < kL; j0 += kFb) {
        if (t == 0) {
            float a[kFb][kFb];
#pragma unroll
            for (int r = 0; r < kFb; ++r)
#pragma unroll
                for (int c = 0; c <= r; ++c) a[r][c] = A[j0 + r][j0 + c];
#pragma unroll
            for (int c = 0; c < kFb; ++c) {
                float s = a[c][c];
#pragma unroll
                for (int k = 0; k < c; ++k) s = fmaf(-a[c][k], a[c][k], s);
                // the pivot and its reciprocal from one reciprocal square root (a few ulp: C
                // feeds BF16 operands)
                const float ri = s > kPivotFloor * gd[j0 + c] ? rsqrtf(s) : 0.0f;
                const float d = s * ri;
                a[c][c] = d;
                rinv[j0 + c] = ri;
#pragma unroll
                for (int r = c + 1; r < kFb; ++r) {
                    float v = a[r][c];
#pragma unroll
                    for (int k = 0; k < c; ++k) v = fmaf(-a[r][k], a[c][k], v);
                    a[r][c] = v * ri;
                }
            }
#pragma unroll
            for (int r = 0; r < kFb; ++r)
#pragma unroll
                for (int c = 0; c <= r; ++c) A[j0 + r][j0 + c] = a[r][c];
        }
        __syncthreads();
        // rows below the block: x L_bb^T = A[i][j0 .. j0 + 7]
        const int i = j0 + kFb + t;
        if (i < kL) {
            float x[kFb];
#pragma unroll
            for (int c = 0; c < kFb; ++c) {
                float v = A[i][j0 + c];
#pragma unroll
                for (int k = 0; k < c; ++k) v = fmaf(-x[k], A[j0 + c][j0 + k], v);
                x[c] = v * rinv[j0 + c];
            }
#pragma unroll
            for (int c = 0; c < kFb; ++c) A[i][j0 + c] = x[c];
        }
        __syncthreads();
        // trailing lower triangle: A[r][c] -= sum_k C[r][j0 + k] C[c][j0 + k], j0 + 8 <= c <= r
        const int m = kL - j0 - kFb;
        for (int e = t; e < m * m; e += 256) {
            const int r = j0 + kFb + e / m, c = j0 + kFb + e % m;
            if (c <= r) {
                float v = A[r][c];
#pragma unroll
                for (int k = 0; k < kFb; ++k) v = fmaf(-A[r][j0 + k], A[c][j0 + k], v);
                A[r][c] = v;
            }
        }
        __syncthreads();
    }
    // every read of G is done: overwrite its rows with those of C^T (C's upper triangle is zero)
    for (int e = t; e < kL * kL; e += 256) {
        const int j = e >> 6, k = e & 63;
        G[e] = k >= j ? A[k][j] : 0.0f;
    }
}

// grid (ceil(P / 128), levels), 128 threads, dynamic smem = (64 + nt) * 64 floats.
__global__ void __launch_bounds__(128) query_f32_kernel(int64_t P, int Q, int n_neg, float tau,
                                                        const float* __restrict__ W, const float* __restrict__ Bt,
                                                        const float* __restrict__ tnorm, float* __restrict__ rel)
{
    extern __shared__ __align__(16) float sB[];
    const int lev = blockIdx.y, levels = gridDim.y;
    const int nt = Q * (1 + n_neg), ncol = kL + nt;
    const float* Bl = Bt + (size_t)lev * ncol * kL;
    for (int i = threadIdx.x * 4; i < ncol * kL; i += 512)
        *reinterpret_cast<float4*>(sB + i) = __ldg(reinterpret_cast<const float4*>(Bl + i));
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (p >= P) return;
    float w[kL];
    const float4* src = reinterpret_cast<const float4*>(W + ((size_t)lev * P + p) * kL);
#pragma unroll
    for (int i = 0; i < kL / 4; ++i) {
        const float4 v = __ldcs(src + i);
        w[4 * i] = v.x;
        w[4 * i + 1] = v.y;
        w[4 * i + 2] = v.z;
        w[4 * i + 3] = v.w;
    }
    float n2 = 0.0f;
#pragma unroll
    for (int j = 0; j < kL; ++j) {
        const float* col = sB + j * kL;
        float y = 0.0f;
#pragma unroll
        for (int k = 0; k < kL; k += 4) {
            const float4 b = *reinterpret_cast<const float4*>(col + k);
            y = fmaf(w[k], b.x, y);
            y = fmaf(w[k + 1], b.y, y);
            y = fmaf(w[k + 2], b.z, y);
            y = fmaf(w[k + 3], b.w, y);
        }
        n2 = fmaf(w[j], y, n2);
    }
    const float nf = sqrtf(fmaxf(n2, 0.0f));
    for (int q = 0; q < Q; ++q) {
        float best = -INFINITY, cpos = 0.0f;
        for (int t = 0; t <= n_neg; ++t) {
            const int tt = q * (1 + n_neg) + t;
            const float* col = sB + (kL + tt) * kL;
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < kL; k += 4) {
                const float4 b = *reinterpret_cast<const float4*>(col + k);
                s = fmaf(w[k], b.x, s);
                s = fmaf(w[k + 1], b.y, s);
                s = fmaf(w[k + 2], b.z, s);
                s = fmaf(w[k + 3], b.w, s);
            }
            const float c = nf < 1e-12f ? 0.0f : s / (nf * tnorm[tt]);
            if (t == 0) cpos = c;
            else best = fmaxf(best, c);
        }
        const float r = 1.0f / (1.0f + expf(-tau * (cpos - best)));
        rel[((size_t)q * levels + lev) * P + p] = r;
    }
}

}  // namespace

const float* query_ws_bt(const void* ws) { return static_cast<const float*>(ws); }

const float* query_ws_tnorm(const void* ws, int levels, int nt)
{
    return reinterpret_cast<const float*>(static_cast<const char*>(ws) +
                                          ((size_t)levels * (kL + nt) * kL * 4 + 255) / 256 * 256);
}

size_t query_workspace_bytes(int levels, int nt)
{
    return ((size_t)levels * (kL + nt) * kL * 4 + 255) / 256 * 256 + ((size_t)nt * 4 + 255) / 256 * 256;
}

cudaError_t launch_query_prepare(int levels, int D, int nt, const float* S, const float* text, void* ws,
                                 cudaStream_t stream)
{
    float* Bt = static_cast<float*>(ws);
    float* tnorm = reinterpret_cast<float*>(static_cast<char*>(ws) +
                                            ((size_t)levels * (kL + nt) * kL * 4 + 255) / 256 * 256);
    dim3 grid((unsigned)(kL + nt), (unsigned)levels);
    cudaError_t e = cudaFuncSetAttribute(query_prepare_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, D * 4);
    if (e != cudaSuccess) return e;
    query_prepare_kernel<<<grid, 256, (size_t)D * 4, stream>>>(D, nt, S, text, Bt, tnorm);
    return cudaGetLastError();
}

cudaError_t launch_query_factor(int levels, int nt, void* ws, cudaStream_t stream)
{
    query_factor_kernel<<<levels, 256, 0, stream>>>(kL + nt, static_cast<float*>(ws));
    return cudaGetLastError();
}

cudaError_t launch_query_f32(int levels, int64_t P, int Q, int n_neg, float tau, const float* W, const void* ws,
                             float* rel, cudaStream_t stream)
{
    if (P == 0) return cudaSuccess;
    const int nt = Q * (1 + n_neg);
    const float* Bt = static_cast<const float*>(ws);
    const float* tnorm = reinterpret_cast<const float*>(static_cast<const char*>(ws) +
                                                        ((size_t)levels * (kL + nt) * kL * 4 + 255) / 256 * 256);
    const size_t smem = (size_t)(kL + nt) * kL * 4;
    cudaError_t e = cudaFuncSetAttribute(query_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((P + 127) / 128), (unsigned)levels);
    query_f32_kernel<<<grid, 128, smem, stream>>>(P, Q, n_neg, tau, W, Bt, tnorm, rel);
    return cudaGetLastError();
}

}  // namespace lsv2
