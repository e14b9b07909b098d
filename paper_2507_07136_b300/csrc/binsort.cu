// binsort.cu -- tile binning and per-tile depth order ("ordered Gaussian points within a
// tile", Eq. 3).  One instance per (visible Gaussian, tile of its rectangle), ordered by
// (tile, depth key bits, Gaussian id).
//
// Instead of one global radix sort over (tile, depth) keys, the instances are bucketed by
// tile with a counting pass (atomic counts -> exclusive scan -> atomic scatter) and each
// bucket is then sorted on its own by one CTA on the 64-bit key (depth bits << 32 | id):
// small buckets by a bitonic sort in shared memory, large buckets by bitonic-sorted chunks
// merged pairwise (each element's output slot = own index + rank in the other run; keys
// are unique).  The scatter order is nondeterministic, the sorted result is not.
// Capacity overflow is reported in the status word and every range is clipped to capacity,
// so nothing downstream can read out of bounds.
#include "device.cuh"
#include "binsort.cuh"

namespace lsv2 {
namespace {

constexpr int kSmallCap = 2048;   // keys per bucket sorted in one shared-memory bitonic pass
constexpr int kChunk = 8192;      // chunk size of the large-bucket path (64 KB of keys)

__global__ void __launch_bounds__(256) count_kernel(int64_t n, const int32_t* rect, const uint32_t* touched,
                                                    int GX, uint32_t* count)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || touched[g] == 0) return;
    const int4 r = reinterpret_cast<const int4*>(rect)[g];
    for (int ty = r.y; ty < r.w; ++ty)
        for (int tx = r.x; tx < r.z; ++tx) atomicAdd(&count[ty * GX + tx], 1u);
}

// Single CTA: exclusive scan of the bucket sizes, clipped ranges, capacity check; resets
// the counters for the scatter pass.
__global__ void __launch_bounds__(1024) scan_kernel(int T, uint32_t* count, uint32_t* start,
                                                    uint32_t* tile_ranges, int64_t capacity,
                                                    int64_t* num_instances, int32_t* status)
{
    __shared__ unsigned long long warp_sums[32];
    const int tid = threadIdx.x;
    const int per = (T + 1023) / 1024;
    const int b = tid * per, e = min(T, b + per);
    unsigned long long local = 0;
    for (int t = b; t < e; ++t) local += count[t];
    // inclusive scan of `local` across the block
    unsigned long long x = local;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if ((tid & 31) >= o) x += y;
    }
    if ((tid & 31) == 31) warp_sums[tid >> 5] = x;
    __syncthreads();
    if (tid < 32) {
        unsigned long long w = warp_sums[tid];
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (tid >= o) w += y;
        }
        warp_sums[tid] = w;
    }
    __syncthreads();
    unsigned long long run = x - local + ((tid >> 5) ? warp_sums[(tid >> 5) - 1] : 0ull);
    const unsigned long long cap = (unsigned long long)capacity;
    for (int t = b; t < e; ++t) {
        const unsigned long long c = count[t];
        start[t] = (uint32_t)min(run, cap);
        tile_ranges[2 * t] = (uint32_t)min(run, cap);
        tile_ranges[2 * t + 1] = (uint32_t)min(run + c, cap);
        run += c;
        count[t] = 0;
    }
    if (tid == 1023) {
        *num_instances = (int64_t)run;
        if (run > cap) report(status, LSV2_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(256) scatter_kernel(int64_t n, const int32_t* rect, const uint32_t* touched,
                                                      const float* depth, int GX, uint32_t* count,
                                                      const uint32_t* start, int64_t capacity,
                                                      unsigned long long* keys)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n || touched[g] == 0) return;
    const int4 r = reinterpret_cast<const int4*>(rect)[g];
    const unsigned long long key = ((unsigned long long)__float_as_uint(depth[g]) << 32) | (unsigned long long)g;
    for (int ty = r.y; ty < r.w; ++ty)
        for (int tx = r.x; tx < r.z; ++tx) {
            const int t = ty * GX + tx;
            const unsigned long long dst = (unsigned long long)start[t] + atomicAdd(&count[t], 1u);
            if (dst < (unsigned long long)capacity) keys[dst] = key;
        }
}

__device__ void bitonic_smem(unsigned long long* s, int npow2)
{
    for (int k = 2; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = s[i], b = s[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) sort_small_kernel(const uint32_t* tile_ranges,
                                                         const unsigned long long* keys, uint32_t* ids)
{
    __shared__ unsigned long long s[kSmallCap];
    const uint32_t b = tile_ranges[2 * blockIdx.x], e = tile_ranges[2 * blockIdx.x + 1];
    const int n = (int)(e - b);
    if (n <= 1) {
        if (n == 1 && threadIdx.x == 0) ids[b] = (uint32_t)keys[b];
        return;
    }
    if (n > kSmallCap) return;
    int np = 2;
    while (np < n) np <<= 1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s[i] = i < n ? keys[b + i] : ~0ull;
    __syncthreads();
    bitonic_smem(s, np);
    for (int i = threadIdx.x; i < n; i += blockDim.x) ids[b + i] = (uint32_t)s[i];
}

// rank of `key` in the sorted run r[0, len): number of elements smaller than key
__device__ __forceinline__ int lower_rank(const unsigned long long* r, int len, unsigned long long key)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (r[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(1024) sort_large_kernel(const uint32_t* tile_ranges, unsigned long long* keys,
                                                          unsigned long long* alt, uint32_t* ids)
{
    extern __shared__ unsigned long long sk[];
    const uint32_t b = tile_ranges[2 * blockIdx.x], e = tile_ranges[2 * blockIdx.x + 1];
    const int n = (int)(e - b);
    if (n <= kSmallCap) return;
    unsigned long long* src = keys + b;
    unsigned long long* dst = alt + b;
    // 1. sort chunks in shared memory
    for (int c0 = 0; c0 < n; c0 += kChunk) {
        const int len = min(kChunk, n - c0);
        int np = 2;
        while (np < len) np <<= 1;
        for (int i = threadIdx.x; i < np; i += blockDim.x) sk[i] = i < len ? src[c0 + i] : ~0ull;
        __syncthreads();
        bitonic_smem(sk, np);
        for (int i = threadIdx.x; i < len; i += blockDim.x) src[c0 + i] = sk[i];
        __syncthreads();
    }
    // 2. merge runs pairwise until one run remains
    for (int run = kChunk; run < n; run <<= 1) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int r0 = (i / (2 * run)) * 2 * run;      // start of this pair of runs
            const int a_len = min(run, n - r0);
            const int b0 = r0 + a_len, b_len = max(0, min(run, n - b0));
            const unsigned long long k = src[i];
            int pos;
            if (i < b0) pos = (i - r0) + lower_rank(src + b0, b_len, k);
            else pos = (i - b0) + lower_rank(src + r0, a_len, k);
            dst[r0 + pos] = k;
        }
        __syncthreads();
        unsigned long long* t = src;
        src = dst;
        dst = t;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) ids[b + i] = (uint32_t)src[i];
}

}  // namespace

size_t binsort_workspace_bytes(int64_t capacity, int32_t num_tiles)
{
    const size_t t4 = ((size_t)num_tiles * 4 + 255) / 256 * 256;
    return 2 * t4 + 2 * (((size_t)capacity * 8 + 255) / 256 * 256);
}

cudaError_t launch_binsort(const BinSortArgs& a, cudaStream_t stream)
{
    const size_t t4 = ((size_t)a.num_tiles * 4 + 255) / 256 * 256;
    const size_t kbytes = ((size_t)a.capacity * 8 + 255) / 256 * 256;
    char* ws = static_cast<char*>(a.workspace);
    uint32_t* count = reinterpret_cast<uint32_t*>(ws);
    uint32_t* start = reinterpret_cast<uint32_t*>(ws + t4);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + 2 * t4);
    unsigned long long* alt = reinterpret_cast<unsigned long long*>(ws + 2 * t4 + kbytes);
    cudaError_t e = cudaMemsetAsync(count, 0, (size_t)a.num_tiles * 4, stream);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
    if (a.n > 0) count_kernel<<<blocks, threads, 0, stream>>>(a.n, a.rect, a.touched, a.GX, count);
    scan_kernel<<<1, 1024, 0, stream>>>(a.num_tiles, count, start, a.tile_ranges, a.capacity,
                                        a.num_instances, a.status);
    if (a.n > 0)
        scatter_kernel<<<blocks, threads, 0, stream>>>(a.n, a.rect, a.touched, a.depth, a.GX, count, start,
                                                      a.capacity, keys);
    sort_small_kernel<<<a.num_tiles, 256, 0, stream>>>(a.tile_ranges, keys, a.gauss_ids);
    const int large_smem = kChunk * 8;
    e = cudaFuncSetAttribute(sort_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, large_smem);
    if (e != cudaSuccess) return e;
    sort_large_kernel<<<a.num_tiles, 1024, large_smem, stream>>>(a.tile_ranges, keys, alt, a.gauss_ids);
    return cudaGetLastError();
}

}  // namespace lsv2
