// sparsify.cu -- the sparse coefficients of Sec. 3.3 and their gradient.
//
// Every Gaussian carries, per level, an L-dim parameter z: the paper normalises it with a
// softmax, keeps the K largest values as the nonzeros and renormalises them by their sum.  The
// kept weights are then a softmax over the K kept logits (the full softmax's denominator cancels),
// so the forward selects the K largest logits (the softmax is monotone; lower index first among
// equal logits) and takes the softmax of those, and the gradient is zero for the dropped logits
// and w_k (dw_k - sum_m w_m dw_m) for kept entry k (the selection is piecewise constant).
//
// Forward: a row of L logits is split over L / 16 adjacent threads of a warp, each loading its
// 16 logits straight from global memory (four 16-byte loads; no staging, no block barrier).  A
// thread sorts its two groups of 8 with Batcher's 19-comparator network and keeps the first K of
// their union; the row's threads then exchange their K by shuffles (butterfly: both partners end
// with the same K) until every thread holds the row's K.  One total order throughout (the larger
// value, then the lower index), so the selection is unique, and every step is branch-free.  The
// first thread of the row writes idx (K bytes) and w (K floats).  The backward (one row per
// thread) scatters the K gradients into a zeroed row staged in shared memory (rows padded by one
// word: conflict-free) and writes the rows out coalesced: it is HBM-bound (4 L bytes per row out).
#include "device.cuh"

namespace lsv2 {
namespace {

template <int L>
__host__ __device__ constexpr int rows_per_block() { return L <= 64 ? 128 : 32; }

// staged row i (stride L + 1) -> row r0 + i of a [rows][L] float array, coalesced
template <int L, int R>
__device__ __forceinline__ void stage_out(float* dst, int64_t r0, int nr, const float* zs)
{
    float* g = dst + r0 * L;
    for (int i = threadIdx.x; i < nr * L; i += R) g[i] = zs[(i / L) * (L + 1) + (i % L)];
}

// (value a, index ia) ranks before (value b, index ib): the larger value, the lower index on ties
__device__ __forceinline__ bool ranks_before(float a, int ia, float b, int ib) { return a > b || (a == b && ia < ib); }

// put the pair that ranks first in (a, ia)
__device__ __forceinline__ void order_pair(float& a, int& ia, float& b, int& ib)
{
    const bool sw = ranks_before(b, ib, a, ia);
    const float tv = sw ? b : a;
    const int ti = sw ? ib : ia;
    b = sw ? a : b;
    ib = sw ? ia : ib;
    a = tv;
    ia = ti;
}

template <int K>
__device__ __forceinline__ void store_row(uint8_t* idx, float* w, int64_t r, const int (&ix)[K], const float (&wv)[K])
{
    if constexpr (K == 4) {
        reinterpret_cast<uint32_t*>(idx)[r] =
            (uint32_t)ix[0] | ((uint32_t)ix[1] << 8) | ((uint32_t)ix[2] << 16) | ((uint32_t)ix[3] << 24);
        reinterpret_cast<float4*>(w)[r] = make_float4(wv[0], wv[1], wv[2], wv[3]);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            idx[r * K + k] = (uint8_t)ix[k];
            w[r * K + k] = wv[k];
        }
    }
}

// (v, ix) and (u, iu) each hold K entries in rank order; leave the K first of their union in
// (v, ix), in rank order: the better of v[i] and u[K-1-i] form a bitonic sequence, which the
// half-cleaners sort.
template <int K>
__device__ __forceinline__ void merge_first(float (&v)[K], int (&ix)[K], const float (&u)[K], const int (&iu)[K])
{
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const bool take = ranks_before(u[K - 1 - i], iu[K - 1 - i], v[i], ix[i]);
        v[i] = take ? u[K - 1 - i] : v[i];
        ix[i] = take ? iu[K - 1 - i] : ix[i];
    }
#pragma unroll
    for (int m = K / 2; m > 0; m >>= 1)
#pragma unroll
        for (int i = 0; i < K; ++i)
            if ((i & m) == 0) order_pair(v[i], ix[i], v[i | m], ix[i | m]);
}

// sort 8 (value, index) pairs into rank order with Batcher's odd-even merge network
__device__ __forceinline__ void sort8(float (&gv)[8], int (&gi)[8])
{
    constexpr int kNet8[19][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {1, 2}, {5, 6},
                                  {0, 4}, {1, 5}, {2, 6}, {3, 7}, {2, 4}, {3, 5}, {1, 2}, {3, 4}, {5, 6}};
#pragma unroll
    for (int c = 0; c < 19; ++c) order_pair(gv[kNet8[c][0]], gi[kNet8[c][0]], gv[kNet8[c][1]], gi[kNet8[c][1]]);
}

constexpr int kFwdThreads = 256;
constexpr int kPerThread = 16;   // logits per thread: two groups of 8

template <int L, int K>
__global__ void __launch_bounds__(kFwdThreads) sparsify_kernel(int64_t rows, const float* __restrict__ z,
                                                               uint8_t* __restrict__ idx, float* __restrict__ w)
{
    constexpr int T = L / kPerThread;   // threads per row, adjacent lanes of one warp
    static_assert(L % kPerThread == 0 && (T & (T - 1)) == 0 && T <= 32 && K <= 8, "row split");
    const int64_t t = (int64_t)blockIdx.x * kFwdThreads + threadIdx.x;
    const int64_t r = t / T;
    const int part = (int)(t % T);
    // threads past the last row work on the last row (their shuffles keep the warp converged)
    // and store nothing
    const float* src = z + (r < rows ? r : rows - 1) * L + part * kPerThread;
    float x[kPerThread];
    if ((reinterpret_cast<uintptr_t>(z) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < kPerThread / 4; ++j) {
            const float4 q = __ldcs(reinterpret_cast<const float4*>(src) + j);
            x[4 * j] = q.x;
            x[4 * j + 1] = q.y;
            x[4 * j + 2] = q.z;
            x[4 * j + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) x[j] = __ldcs(src + j);
    }
    const int base = part * kPerThread;
    float gv[8], hv[8];
    int gi[8], hi[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        gv[j] = x[j];
        gi[j] = base + j;
        hv[j] = x[8 + j];
        hi[j] = base + 8 + j;
    }
    sort8(gv, gi);
    sort8(hv, hi);
    float v[K], u[K];
    int ix[K], iu[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = gv[k];
        ix[k] = gi[k];
        u[k] = hv[k];
        iu[k] = hi[k];
    }
    merge_first<K>(v, ix, u, iu);
#pragma unroll
    for (int m = 1; m < T; m <<= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            u[k] = __shfl_xor_sync(0xffffffffu, v[k], m);
            iu[k] = __shfl_xor_sync(0xffffffffu, ix[k], m);
        }
        merge_first<K>(v, ix, u, iu);
    }
    if (part != 0 || r >= rows) return;
    // softmax over the kept logits (v[0] is the largest)
    float e[K], s = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        e[k] = expf(v[k] - v[0]);
        s += e[k];
    }
    float wv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) wv[k] = e[k] / s;
    store_row<K>(idx, w, r, ix, wv);
}

template <int L, int K>
__global__ void __launch_bounds__(rows_per_block<L>()) sparsify_backward_kernel(int64_t rows, const uint8_t* __restrict__ idx,
                                                                                const float* __restrict__ w,
                                                                                const float* __restrict__ dw,
                                                                                float* __restrict__ dz)
{
    constexpr int R = rows_per_block<L>();
    extern __shared__ float zs[];
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int nr = rows - r0 < R ? (int)(rows - r0) : R;
    for (int i = threadIdx.x; i < R * (L + 1); i += R) zs[i] = 0.0f;
    __syncthreads();
    if ((int)threadIdx.x < nr) {
        const int64_t r = r0 + threadIdx.x;
        float wv[K], g[K], dot = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            wv[k] = w[r * K + k];
            g[k] = dw[r * K + k];
            dot = fmaf(wv[k], g[k], dot);
        }
        float* row = zs + threadIdx.x * (L + 1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int c = idx[r * K + k];
            if (c < L) row[c] = wv[k] * (g[k] - dot);
        }
    }
    __syncthreads();
    stage_out<L, R>(dz, r0, nr, zs);
}

template <int L, int K>
cudaError_t launch_sparsify_t(int64_t rows, const float* z, uint8_t* idx, float* w, const float* dw, float* dz,
                              bool backward, cudaStream_t stream)
{
    constexpr int R = rows_per_block<L>();
    const size_t smem = (size_t)R * (L + 1) * sizeof(float);
    const int64_t blocks = (rows + R - 1) / R;
    if (blocks == 0) return cudaSuccess;
    if (backward) {
        cudaError_t e = cudaFuncSetAttribute(sparsify_backward_kernel<L, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        sparsify_backward_kernel<L, K><<<(unsigned)blocks, R, smem, stream>>>(rows, idx, w, dw, dz);
    } else {
        const int64_t fwd_blocks = (rows * (L / kPerThread) + kFwdThreads - 1) / kFwdThreads;
        sparsify_kernel<L, K><<<(unsigned)fwd_blocks, kFwdThreads, 0, stream>>>(rows, z, idx, w);
    }
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_sparsify_l(int K, int64_t rows, const float* z, uint8_t* idx, float* w, const float* dw, float* dz,
                              bool backward, cudaStream_t stream)
{
    switch (K) {
        case 1: return launch_sparsify_t<L, 1>(rows, z, idx, w, dw, dz, backward, stream);
        case 2: return launch_sparsify_t<L, 2>(rows, z, idx, w, dw, dz, backward, stream);
        case 4: return launch_sparsify_t<L, 4>(rows, z, idx, w, dw, dz, backward, stream);
        case 8: return launch_sparsify_t<L, 8>(rows, z, idx, w, dw, dz, backward, stream);
        default: return cudaErrorInvalidValue;
    }
}

bool sparsify_supported(int L, int K)
{
    const bool l_ok = L == 16 || L == 32 || L == 64 || L == 128 || L == 256;
    return l_ok && (K == 1 || K == 2 || K == 4 || K == 8) && K <= L;
}

cudaError_t launch_sparsify(int L, int K, int64_t rows, const float* z, uint8_t* idx, float* w, const float* dw,
                            float* dz, bool backward, cudaStream_t stream)
{
    if (rows > 0 && (!idx || !w || (backward ? (!dw || !dz) : !z))) return cudaErrorInvalidValue;
    switch (L) {
        case 16: return launch_sparsify_l<16>(K, rows, z, idx, w, dw, dz, backward, stream);
        case 32: return launch_sparsify_l<32>(K, rows, z, idx, w, dw, dz, backward, stream);
        case 64: return launch_sparsify_l<64>(K, rows, z, idx, w, dw, dz, backward, stream);
        case 128: return launch_sparsify_l<128>(K, rows, z, idx, w, dw, dz, backward, stream);
        case 256: return launch_sparsify_l<256>(K, rows, z, idx, w, dw, dz, backward, stream);
        default: return cudaErrorInvalidValue;
    }
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace
}  // namespace lsv2

using namespace lsv2;

extern "C" lsv2_status lsv2_sparsify(int64_t rows, int32_t L, int32_t K, const float* logits, uint8_t* idx, float* w,
                                     void* stream)
{
    if (rows < 0 || (rows > 0 && (!logits || !idx || !w))) return LSV2_ERR_INVALID_ARGUMENT;
    if (!sparsify_supported(L, K)) return LSV2_ERR_UNSUPPORTED;
    if (!aligned(logits, 4) || !aligned(w, K == 4 ? 16 : 4) || !aligned(idx, K == 4 ? 4 : 1))
        return LSV2_ERR_INVALID_ARGUMENT;
    const cudaError_t e = launch_sparsify(L, K, rows, logits, idx, w, nullptr, nullptr, false,
                                          static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LSV2_OK : LSV2_ERR_CUDA;
}

extern "C" lsv2_status lsv2_sparsify_backward(int64_t rows, int32_t L, int32_t K, const uint8_t* idx, const float* w,
                                              const float* dw, float* dlogits, void* stream)
{
    if (rows < 0 || (rows > 0 && (!idx || !w || !dw || !dlogits))) return LSV2_ERR_INVALID_ARGUMENT;
    if (!sparsify_supported(L, K)) return LSV2_ERR_UNSUPPORTED;
    if (!aligned(w, 4) || !aligned(dw, 4) || !aligned(dlogits, 4)) return LSV2_ERR_INVALID_ARGUMENT;
    const cudaError_t e = launch_sparsify(L, K, rows, nullptr, const_cast<uint8_t*>(idx), const_cast<float*>(w), dw,
                                          dlogits, true, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LSV2_OK : LSV2_ERR_CUDA;
}
