// post.cu -- post-processing of relevancy maps on the GPU (paper appendix, "Evaluation
// Details"; Sec. 3.2 notes that LangSplat ran this stage on the CPU and LangSplat* moved it to
// the GPU).
//
// For every query q and level l the relevancy map M (H x W) is smoothed with a k x k mean
// filter (the mean over the in-image part of the window; k odd, at most kMaxWindow):
//   mode LSV2_POST_LERF:    S = Avg(M); the selected level has the highest value of S; the
//                           localisation point is the first pixel (row-major) where it is
//                           attained; the mask is (S - min S) / (max S - min S) > thr.
//   mode LSV2_POST_BLENDED: S = 0.5 (M + Avg(M)) (3D-OVS, Mip-NeRF360); the selected level has
//                           the highest mean of S over its own mask (an empty mask ranks
//                           lowest); point and mask as above.
// Kernels: workspace init -> box filter over all (q, l) maps, which also reduces each map's
// (value, first index) maximum and its minimum with one atomic per block -> [blended: masked
// sums] -> selection (one thread per query) -> mask of the selected level.  All are stream
// ordered and capturable in a CUDA graph.  HBM-bound: one read of M, one write of S, one or
// two reads of S.
#include <cuda_bf16.h>

#include "device.cuh"

namespace lsv2 {
namespace {

constexpr int kMaxWindow = 63;
constexpr int kTX = 64, kTY = 32;  // output tile of one box-filter CTA
constexpr int kPostThreads = 256;

// Per (q, l) map statistics in the workspace.
struct MapStats {
    unsigned long long max_key;    // orderable(value) << 32 | (0xFFFFFFFF - pixel)
    unsigned int min_key;          // orderable(value)
    unsigned int pad;
    double masked_sum;             // blended mode: sum of S over the mask
    unsigned long long masked_count;
};

// Order-preserving map of a float to an unsigned int (larger float -> larger key).
__device__ __forceinline__ unsigned int orderable(float v)
{
    const unsigned int b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_orderable(unsigned int k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ float load_rel(const void* rel, bool bf16, size_t i)
{
    return bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(rel)[i]) : static_cast<const float*>(rel)[i];
}

__global__ void post_init_kernel(MapStats* st, int maps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < maps) st[i] = MapStats{0ull, 0xFFFFFFFFu, 0u, 0.0, 0ull};
}

struct BoxArgs {
    int H, W, k, mode;
    const void* rel;
    bool bf16;
    float* smoothed;
    MapStats* st;
};

// One kTX x kTY output tile of map blockIdx.z.  The input tile with its halo (r = (k - 1) / 2 on
// each side) is staged in shared memory; the column pass slides a k-row sum down each half of
// each staged column (k loads in four partial sums to start, then one added and one dropped row
// per output row), the row pass slides a k-column sum along 8 outputs per thread; each sum is divided by the number of
// in-image pixels of its window.  (Sliding sums round differently from direct sums by a few
// ulps of a window sum.)
__global__ void __launch_bounds__(kPostThreads) box_filter_kernel(BoxArgs a)
{
    extern __shared__ float sm[];
    const int r = (a.k - 1) / 2;
    const int EX = kTX + 2 * r, EY = kTY + 2 * r;  // staged extents (EX <= 128)
    float* in = sm;                                // [EY][EX]
    float* vs = sm + EX * EY;                      // [kTY][EX] column sums
    const int map = blockIdx.z;
    const size_t P = (size_t)a.H * a.W;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int c = threadIdx.x & 127, xx = x0 - r + c;
    const bool col_in = c < EX && xx >= 0 && xx < a.W;
    if (!a.bf16) {
        // FP32 maps: staged column c = thread % 128, rows thread / 128 + 2 j, every element by an
        // asynchronous 4-byte copy (all of them in flight at once; zero-filled outside the image)
        const float* rel = static_cast<const float*>(a.rel) + map * P;
        for (int row = threadIdx.x >> 7; row < EY; row += 2) {
            const int yy = y0 - r + row;
            const bool ok = col_in && yy >= 0 && yy < a.H;
            const float* src = ok ? rel + (size_t)yy * a.W + xx : rel;
            if (c < EX)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(in + row * EX + c)),
                             "l"(src), "r"(ok ? 4 : 0)
                             : "memory");
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    } else {
        // BF16 maps: eight loads in flight per thread, converted on the way to shared memory
        for (int row0 = threadIdx.x >> 7; row0 < EY; row0 += 16) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int row = row0 + 2 * j, yy = y0 - r + row;
                v[j] = (col_in && row < EY && yy >= 0 && yy < a.H) ? load_rel(a.rel, a.bf16, map * P + (size_t)yy * a.W + xx)
                                                                  : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (c < EX && row0 + 2 * j < EY) in[(row0 + 2 * j) * EX + c] = v[j];
        }
    }
    __syncthreads();
    // column pass: thread -> (column c, output rows h * 16 .. h * 16 + 15)
    if (threadIdx.x < 2 * EX) {
        const int h = threadIdx.x < EX ? 0 : 1, c = threadIdx.x - h * EX, t0 = h * (kTY / 2);
        const float* col = in + t0 * EX + c;
        float p[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int d = 0;
        for (; d + 4 <= a.k; d += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] += col[(d + u) * EX];
        for (; d < a.k; ++d) p[0] += col[d * EX];
        float s = (p[0] + p[1]) + (p[2] + p[3]);
        vs[t0 * EX + c] = s;
        for (int ty = 1; ty < kTY / 2; ++ty) {
            s += col[(ty + a.k - 1) * EX] - col[(ty - 1) * EX];
            vs[(t0 + ty) * EX + c] = s;
        }
    }
    __syncthreads();
    unsigned long long best = 0ull;
    unsigned int lo = 0xFFFFFFFFu;
    {
        // thread -> (row ty, outputs tx0 .. tx0 + 7); kTY x kTX / 8 = kPostThreads segments
        const int ty = threadIdx.x >> 3, tx0 = (threadIdx.x & 7) * 8;
        const int y = y0 + ty;
        const float* row = vs + ty * EX + tx0;
        float p[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int d = 0;
        for (; d + 4 <= a.k; d += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] += row[d + u];
        for (; d < a.k; ++d) p[0] += row[d];
        float s = (p[0] + p[1]) + (p[2] + p[3]);
        const int cy = min(y + r, a.H - 1) - max(y - r, 0) + 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j > 0) s += row[j + a.k - 1] - row[j - 1];
            const int x = x0 + tx0 + j;
            if (x < a.W && y < a.H) {
                const int cx = min(x + r, a.W - 1) - max(x - r, 0) + 1;
                float v = s / (float)(cx * cy);
                if (a.mode == LSV2_POST_BLENDED) v = 0.5f * (in[(ty + r) * EX + tx0 + j + r] + v);
                const size_t pix = (size_t)y * a.W + x;
                a.smoothed[map * P + pix] = v;
                const unsigned int kv = orderable(v);
                const unsigned long long key = ((unsigned long long)kv << 32) | (0xFFFFFFFFull - pix);
                best = key > best ? key : best;
                lo = kv < lo ? kv : lo;
            }
        }
    }
    // block reduction, then one atomic per block and quantity
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        best = ob > best ? ob : best;
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    }
    __shared__ unsigned long long s_best[kPostThreads / 32];
    __shared__ unsigned int s_lo[kPostThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_best[warp] = best;
        s_lo[warp] = lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kPostThreads / 32; ++w) {
            best = s_best[w] > best ? s_best[w] : best;
            lo = min(lo, s_lo[w]);
        }
        if (best != 0ull) atomicMax(&a.st[map].max_key, best);
        if (lo != 0xFFFFFFFFu) atomicMin(&a.st[map].min_key, lo);
    }
}

__device__ __forceinline__ bool in_mask(float v, const MapStats& s, float thr)
{
    const float mx = from_orderable((unsigned int)(s.max_key >> 32)), mn = from_orderable(s.min_key);
    const float nrm = mx > mn ? (v - mn) / (mx - mn) : 0.0f;
    return nrm > thr;
}

// Blended mode: sum and count of S over each map's mask.
__global__ void __launch_bounds__(kPostThreads) masked_sum_kernel(const float* smoothed, size_t P, float thr,
                                                                  MapStats* st)
{
    const int map = blockIdx.y;
    const MapStats s = st[map];
    double sum = 0.0;
    unsigned long long cnt = 0;
    for (size_t p = (size_t)blockIdx.x * kPostThreads + threadIdx.x; p < P; p += (size_t)gridDim.x * kPostThreads) {
        const float v = smoothed[map * P + p];
        if (in_mask(v, s, thr)) {
            sum += (double)v;
            ++cnt;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0) {
        atomicAdd(&st[map].masked_sum, sum);
        atomicAdd(&st[map].masked_count, cnt);
    }
}

__global__ void select_kernel(int Q, int levels, int W, int mode, const MapStats* st, int32_t* point, int32_t* level,
                              float* score)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    int sel = 0;
    double best = 0.0;
    for (int l = 0; l < levels; ++l) {
        const MapStats& s = st[q * levels + l];
        double crit;
        if (mode == LSV2_POST_LERF)
            crit = (double)from_orderable((unsigned int)(s.max_key >> 32));
        else
            crit = s.masked_count > 0 ? s.masked_sum / (double)s.masked_count : -INFINITY;
        if (l == 0 || crit > best) {
            best = crit;
            sel = l;
        }
    }
    const MapStats& s = st[q * levels + sel];
    const unsigned long long pix = 0xFFFFFFFFull - (s.max_key & 0xFFFFFFFFull);
    point[2 * q] = (int32_t)(pix % (unsigned long long)W);
    point[2 * q + 1] = (int32_t)(pix / (unsigned long long)W);
    level[q] = sel;
    score[q] = from_orderable((unsigned int)(s.max_key >> 32));
}

__global__ void __launch_bounds__(kPostThreads) mask_kernel(const float* smoothed, size_t P, int levels, float thr,
                                                            const MapStats* st, const int32_t* level, uint8_t* mask)
{
    const int q = blockIdx.y;
    const int l = level[q];
    const MapStats s = st[q * levels + l];
    const float* src = smoothed + ((size_t)q * levels + l) * P;
    for (size_t p = (size_t)blockIdx.x * kPostThreads + threadIdx.x; p < P; p += (size_t)gridDim.x * kPostThreads)
        mask[(size_t)q * P + p] = in_mask(src[p], s, thr) ? 1 : 0;
}

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

int grid_cap(size_t P)
{
    const size_t b = (P + kPostThreads - 1) / kPostThreads;
    return (int)(b < 4096 ? b : 4096);
}

}  // namespace
}  // namespace lsv2

using namespace lsv2;

extern "C" size_t lsv2_postprocess_workspace_bytes(int32_t Q, int32_t levels)
{
    if (Q < 1 || levels < 1 || levels > 8) return 0;
    return a256((size_t)Q * levels * sizeof(MapStats));
}

extern "C" lsv2_status lsv2_postprocess(int32_t Q, int32_t levels, int32_t H, int32_t W, const void* rel,
                                        lsv2_dtype rel_dtype, int32_t k, int32_t mode, float threshold,
                                        void* workspace, size_t workspace_bytes, float* smoothed, int32_t* point,
                                        int32_t* level, float* score, uint8_t* mask, int32_t* dev_status,
                                        void* stream)
{
    (void)dev_status;
    if (Q < 1 || levels < 1 || levels > 8 || H < 1 || W < 1 || (int64_t)H * W > 0xFFFFFFFFll) return LSV2_ERR_INVALID_ARGUMENT;
    if (k < 1 || k > kMaxWindow || (k & 1) == 0) return LSV2_ERR_INVALID_ARGUMENT;
    if (mode != LSV2_POST_LERF && mode != LSV2_POST_BLENDED) return LSV2_ERR_INVALID_ARGUMENT;
    if (!(threshold >= 0.0f && threshold <= 1.0f)) return LSV2_ERR_INVALID_ARGUMENT;
    if (rel_dtype != LSV2_F32 && rel_dtype != LSV2_BF16) return LSV2_ERR_INVALID_ARGUMENT;
    if (!rel || !smoothed || !point || !level || !score) return LSV2_ERR_INVALID_ARGUMENT;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 15u) ||
        workspace_bytes < lsv2_postprocess_workspace_bytes(Q, levels))
        return LSV2_ERR_INVALID_ARGUMENT;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int maps = Q * levels;
    MapStats* ms = static_cast<MapStats*>(workspace);
    const size_t P = (size_t)H * W;
    post_init_kernel<<<(maps + 255) / 256, 256, 0, st>>>(ms, maps);
    const int r = (k - 1) / 2, EX = kTX + 2 * r, EY = kTY + 2 * r;
    const size_t smem = (size_t)(EX * EY + kTY * EX) * sizeof(float);
    BoxArgs ba{H, W, k, mode, rel, rel_dtype == LSV2_BF16, smoothed, ms};
    if (cudaFuncSetAttribute(box_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LSV2_ERR_CUDA;
    box_filter_kernel<<<dim3((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, maps), kPostThreads, smem, st>>>(ba);
    if (mode == LSV2_POST_BLENDED)
        masked_sum_kernel<<<dim3(grid_cap(P), maps), kPostThreads, 0, st>>>(smoothed, P, threshold, ms);
    select_kernel<<<(Q + 127) / 128, 128, 0, st>>>(Q, levels, W, mode, ms, point, level, score);
    if (mask) mask_kernel<<<dim3(grid_cap(P), Q), kPostThreads, 0, st>>>(smoothed, P, levels, threshold, ms, level, mask);
    return cudaGetLastError() == cudaSuccess ? LSV2_OK : LSV2_ERR_CUDA;
}
