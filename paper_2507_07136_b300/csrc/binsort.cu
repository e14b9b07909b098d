// binsort.cu -- tile binning and per-tile depth order ("ordered Gaussian points within a
// tile", Eq. 3), for one view or several views at once.  One instance per (visible Gaussian,
// tile of its rectangle), ordered by (tile, depth key bits, Gaussian id); tiles of view v are
// numbered tile_base[v] + ty * GX_v + tx.
//
// Counting sort by tile with no global atomics (same-address atomics on the densest tiles
// serialise in L2):
//   1. hist:    block b of view v counts its Gaussians' tiles in shared memory and writes the
//               histogram row hist_v[b][t]
//   2. columns: one thread per tile scans hist_v[.][t] over blocks (exclusive, in place) and
//               writes the tile's total
//   3. scan:    exclusive scan of the totals -> tile ranges (clipped to capacity), instance
//               count, capacity check, list of tiles too large for the shared-memory sort
//   4. scatter: block b starts per-tile shared-memory cursors at tile_start[t] + hist_v[b][t]
//               and writes each instance's 64-bit key (depth bits << 32 | id) at its cursor
//   5. sort:    per tile, bitonic sort in shared memory (<= 2048 keys); larger tiles (from the
//               list) by bitonic-sorted chunks merged pairwise (output slot = own index + rank
//               in the other run; keys are unique)
// Slot assignment within a block is nondeterministic, the sorted lists are not.
#include "binsort.cuh"
#include "device.cuh"

namespace lsv2 {
namespace {

constexpr int kGB = 1024;          // Gaussians per histogram block
constexpr int kSmallCap = 2048;    // keys sorted in one shared-memory bitonic pass
constexpr int kChunk = 8192;       // chunk of the large-tile path (64 KB of keys)

struct ViewsDev {                  // per-view tables (device copies live in the workspace)
    int32_t GX[kMaxViews];
    int32_t T[kMaxViews];
    int32_t tile_base[kMaxViews + 1];
    int64_t hist_base[kMaxViews];
};

__device__ __forceinline__ int view_of_tile(const ViewsDev& vd, int V, int tg)
{
    int v = 0;
    while (v + 1 < V && tg >= vd.tile_base[v + 1]) ++v;
    return v;
}

__global__ void __launch_bounds__(kGB) hist_kernel(BinSortViews a, ViewsDev vd, uint32_t* hist)
{
    extern __shared__ uint32_t cnt[];
    const int v = blockIdx.y, b = blockIdx.x, T = vd.T[v], GX = vd.GX[v];
    for (int t = threadIdx.x; t < T; t += kGB) cnt[t] = 0;
    __syncthreads();
    const int64_t g = (int64_t)b * kGB + threadIdx.x;
    if (g < a.n) {
        const size_t o = (size_t)v * a.n + g;
        if (a.touched[o] != 0) {
            const int4 r = reinterpret_cast<const int4*>(a.rect)[o];
            for (int ty = r.y; ty < r.w; ++ty)
                for (int tx = r.x; tx < r.z; ++tx) atomicAdd(&cnt[ty * GX + tx], 1u);
        }
    }
    __syncthreads();
    uint32_t* row = hist + vd.hist_base[v] + (size_t)b * T;
    for (int t = threadIdx.x; t < T; t += kGB) row[t] = cnt[t];
}

__global__ void __launch_bounds__(256) column_kernel(int V, int nblk, ViewsDev vd, uint32_t* hist, uint32_t* total,
                                                     int T_total)
{
    const int tg = blockIdx.x * blockDim.x + threadIdx.x;
    if (tg >= T_total) return;
    const int v = view_of_tile(vd, V, tg);
    const int t = tg - vd.tile_base[v], T = vd.T[v];
    uint32_t* col = hist + vd.hist_base[v] + t;
    uint32_t run = 0;
    // 16 block counts are loaded before any is overwritten, so their latencies overlap
    constexpr int kU = 16;
    int b = 0;
    for (; b + kU <= nblk; b += kU) {
        uint32_t c[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) c[u] = col[(size_t)(b + u) * T];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            col[(size_t)(b + u) * T] = run;
            run += c[u];
        }
    }
    for (; b < nblk; ++b) {
        const uint32_t c = col[(size_t)b * T];
        col[(size_t)b * T] = run;
        run += c;
    }
    total[tg] = run;
}

// Single CTA: exclusive scan of the per-tile totals, clipped ranges, capacity check, and the list
// of tiles that need the large-tile sort (count in big[0], ids from big[1]).
__global__ void __launch_bounds__(1024) scan_kernel(int T, const uint32_t* total, uint32_t* start,
                                                    uint32_t* tile_ranges, int64_t capacity, int64_t* num_instances,
                                                    uint32_t* big, int32_t* status)
{
    __shared__ unsigned long long warp_sums[32];
    __shared__ uint32_t nbig;
    const int tid = threadIdx.x;
    if (tid == 0) nbig = 0;
    const int per = (T + 1023) / 1024;
    const int b = tid * per, e = min(T, b + per);
    unsigned long long local = 0;
    for (int t = b; t < e; ++t) local += total[t];
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
        const unsigned long long c = total[t];
        const uint32_t s = (uint32_t)min(run, cap), en = (uint32_t)min(run + c, cap);
        start[t] = s;
        tile_ranges[2 * t] = s;
        tile_ranges[2 * t + 1] = en;
        if (en - s > (uint32_t)kSmallCap) big[1 + atomicAdd(&nbig, 1u)] = (uint32_t)t;
        run += c;
    }
    __syncthreads();
    if (tid == 0) big[0] = nbig;
    if (tid == 1023) {
        *num_instances = (int64_t)run;
        if (run > cap) report(status, LSV2_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kGB) scatter_kernel(BinSortViews a, ViewsDev vd, const uint32_t* hist,
                                                      const uint32_t* start, unsigned long long* keys)
{
    extern __shared__ uint32_t cur[];
    const int v = blockIdx.y, b = blockIdx.x, T = vd.T[v], GX = vd.GX[v], tb = vd.tile_base[v];
    const uint32_t* row = hist + vd.hist_base[v] + (size_t)b * T;
    for (int t = threadIdx.x; t < T; t += kGB) cur[t] = start[tb + t] + row[t];
    __syncthreads();
    const int64_t g = (int64_t)b * kGB + threadIdx.x;
    if (g >= a.n) return;
    const size_t o = (size_t)v * a.n + g;
    if (a.touched[o] == 0) return;
    const int4 r = reinterpret_cast<const int4*>(a.rect)[o];
    const unsigned long long key = ((unsigned long long)__float_as_uint(a.depth[o]) << 32) | (unsigned long long)g;
    for (int ty = r.y; ty < r.w; ++ty)
        for (int tx = r.x; tx < r.z; ++tx) {
            const uint32_t dst = atomicAdd(&cur[ty * GX + tx], 1u);
            if ((int64_t)dst < a.capacity) keys[dst] = key;
        }
}

// Bitonic sorting network over 32 K keys held by one warp, key i = lane * K + j in register j:
// partners i ^ m with m < K are registers of the same lane, the others (m >= K) are exchanged
// with lane ^ (m / K) by shuffles.  Ascending on return.
template <int K>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&x)[K], int lane)
{
#pragma unroll
    for (int k = 2; k <= 32 * K; k <<= 1) {
#pragma unroll
        for (int m = k >> 1; m > 0; m >>= 1) {
            if (m < K) {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    if ((j & m) == 0) {
                        const bool up = (((lane * K) | j) & k) == 0;
                        const unsigned long long lo = x[j], hi = x[j | m];
                        const bool sw = (lo > hi) == up;
                        x[j] = sw ? hi : lo;
                        x[j | m] = sw ? lo : hi;
                    }
                }
            } else {
                const int ml = m / K;
                const bool lower = (lane & ml) == 0;       // this lane holds the pair's lower index
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const bool up = (((lane * K) | j) & k) == 0;
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, x[j], ml);
                    x[j] = (lower == up) ? (o < x[j] ? o : x[j]) : (o > x[j] ? o : x[j]);
                }
            }
        }
    }
}

template <int K>
__device__ __forceinline__ void warp_sort_tile(const unsigned long long* keys, uint32_t* ids, uint32_t b, int n, int lane)
{
    unsigned long long x[K];
#pragma unroll
    for (int j = 0; j < K; ++j) x[j] = lane * K + j < n ? keys[b + lane * K + j] : ~0ull;
    warp_bitonic<K>(x, lane);
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (lane * K + j < n) ids[b + lane * K + j] = (uint32_t)x[j];
}

// One warp per tile of at most kWarpCap keys (the common case), four tiles per block; the key
// (depth bits, Gaussian id) is unique, so the sorted order is.
constexpr int kWarpCap = 512;
__global__ void __launch_bounds__(128) sort_warp_kernel(int T, const uint32_t* tile_ranges,
                                                        const unsigned long long* keys, uint32_t* ids)
{
    const int tile = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (tile >= T) return;
    const uint32_t b = tile_ranges[2 * tile], e = tile_ranges[2 * tile + 1];
    const int n = (int)(e - b);
    if (n <= 1) {
        if (n == 1 && lane == 0) ids[b] = (uint32_t)keys[b];
    } else if (n <= 64) {
        warp_sort_tile<2>(keys, ids, b, n, lane);
    } else if (n <= 128) {
        warp_sort_tile<4>(keys, ids, b, n, lane);
    } else if (n <= 256) {
        warp_sort_tile<8>(keys, ids, b, n, lane);
    } else if (n <= kWarpCap) {
        warp_sort_tile<16>(keys, ids, b, n, lane);
    }
}

// Tiles of kWarpCap < n <= kSmallCap keys: one block of four warps.  Warp r sorts keys
// [512 r, 512 r + 512) of the tile in registers (warp_bitonic), the runs go to shared memory, and
// each key's place in the tile is its index in its run plus the number of smaller keys in each
// other run (a binary search per run; keys are unique, so the places are).  Two barriers in all.
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

__global__ void __launch_bounds__(128) sort_small_kernel(const uint32_t* tile_ranges,
                                                         const unsigned long long* keys, uint32_t* ids)
{
    __shared__ unsigned long long s[kSmallCap];
    const uint32_t b = tile_ranges[2 * blockIdx.x], e = tile_ranges[2 * blockIdx.x + 1];
    const int n = (int)(e - b);
    if (n <= kWarpCap || n > kSmallCap) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nruns = (n + kWarpCap - 1) / kWarpCap;
    if (warp < nruns) {
        unsigned long long x[kWarpCap / 32];
#pragma unroll
        for (int j = 0; j < kWarpCap / 32; ++j) {
            const int i = warp * kWarpCap + lane * (kWarpCap / 32) + j;
            x[j] = i < n ? keys[b + i] : ~0ull;
        }
        warp_bitonic<kWarpCap / 32>(x, lane);
#pragma unroll
        for (int j = 0; j < kWarpCap / 32; ++j) s[warp * kWarpCap + lane * (kWarpCap / 32) + j] = x[j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // the i-th key in run order (runs hold n keys in all, padding at the end of the last run)
        const int r = i / kWarpCap, p = i - r * kWarpCap;
        const unsigned long long k = s[i];
        int place = p;
        for (int q = 0; q < nruns; ++q) {
            if (q == r) continue;
            const int len = q == nruns - 1 ? n - q * kWarpCap : kWarpCap;
            place += lower_rank(s + q * kWarpCap, len, k);
        }
        ids[b + place] = (uint32_t)k;
    }
}


// Persistent over the list of large tiles.
__global__ void __launch_bounds__(1024) sort_large_kernel(const uint32_t* tile_ranges, const uint32_t* big,
                                                          unsigned long long* keys, unsigned long long* alt,
                                                          uint32_t* ids)
{
    extern __shared__ unsigned long long sk[];
    const uint32_t nbig = big[0];
    for (uint32_t it = blockIdx.x; it < nbig; it += gridDim.x) {
        const uint32_t tile = big[1 + it];
        const uint32_t b = tile_ranges[2 * tile], e = tile_ranges[2 * tile + 1];
        const int n = (int)(e - b);
        unsigned long long* src = keys + b;
        unsigned long long* dst = alt + b;
        // each chunk: runs of kWarpCap keys sorted by warps in registers, then every key placed at
        // its index in its run plus the count of smaller keys in the chunk's other runs
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int c0 = 0; c0 < n; c0 += kChunk) {
            const int len = min(kChunk, n - c0);
            const int nruns = (len + kWarpCap - 1) / kWarpCap;
            if (warp < nruns) {
                unsigned long long x[kWarpCap / 32];
#pragma unroll
                for (int j = 0; j < kWarpCap / 32; ++j) {
                    const int i = warp * kWarpCap + lane * (kWarpCap / 32) + j;
                    x[j] = i < len ? src[c0 + i] : ~0ull;
                }
                warp_bitonic<kWarpCap / 32>(x, lane);
#pragma unroll
                for (int j = 0; j < kWarpCap / 32; ++j) sk[warp * kWarpCap + lane * (kWarpCap / 32) + j] = x[j];
            }
            __syncthreads();
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const int r = i / kWarpCap, p = i - r * kWarpCap;
                const unsigned long long k = sk[i];
                int place = p;
                for (int q = 0; q < nruns; ++q) {
                    if (q == r) continue;
                    const int qlen = q == nruns - 1 ? len - q * kWarpCap : kWarpCap;
                    place += lower_rank(sk + q * kWarpCap, qlen, k);
                }
                src[c0 + place] = k;
            }
            __syncthreads();
        }
        for (int run = kChunk; run < n; run <<= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int r0 = (i / (2 * run)) * 2 * run;
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
        __syncthreads();
    }
}

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

struct Layout {
    size_t total, start, big, hist, keys, alt, bytes;
};

Layout layout(int64_t n, int64_t capacity, const int32_t* T, int V)
{
    int64_t nblk = (n + kGB - 1) / kGB;
    if (nblk < 1) nblk = 1;
    int64_t Tt = 0, hist = 0;
    for (int v = 0; v < V; ++v) {
        Tt += T[v];
        hist += nblk * T[v];
    }
    Layout L{};
    L.total = 0;
    L.start = L.total + a256((size_t)Tt * 4);
    L.big = L.start + a256((size_t)Tt * 4);
    L.hist = L.big + a256((size_t)(Tt + 1) * 4);
    L.keys = L.hist + a256((size_t)hist * 4);
    L.alt = L.keys + a256((size_t)capacity * 8);
    L.bytes = L.alt + a256((size_t)capacity * 8);
    return L;
}

}  // namespace

size_t binsort_views_workspace_bytes(int64_t n, int64_t capacity, const int32_t* num_tiles, int V)
{
    return layout(n, capacity, num_tiles, V).bytes;
}

size_t binsort_workspace_bytes(int64_t n, int64_t capacity, int32_t num_tiles)
{
    return layout(n, capacity, &num_tiles, 1).bytes;
}

int binsort_max_tiles_per_view() { return 56 * 1024; }

cudaError_t launch_binsort_views(const BinSortViews& a, cudaStream_t stream)
{
    const int V = a.V;
    ViewsDev vd{};
    int Tt = 0, Tmax = 0;
    int64_t nblk = (a.n + kGB - 1) / kGB;
    if (nblk < 1) nblk = 1;
    int64_t hb = 0;
    for (int v = 0; v < V; ++v) {
        vd.GX[v] = a.GX[v];
        vd.T[v] = a.T[v];
        vd.tile_base[v] = Tt;
        vd.hist_base[v] = hb;
        hb += nblk * a.T[v];
        Tt += a.T[v];
        Tmax = a.T[v] > Tmax ? a.T[v] : Tmax;
    }
    vd.tile_base[V] = Tt;
    const Layout L = layout(a.n, a.capacity, a.T, V);
    char* ws = static_cast<char*>(a.workspace);
    uint32_t* total = reinterpret_cast<uint32_t*>(ws + L.total);
    uint32_t* start = reinterpret_cast<uint32_t*>(ws + L.start);
    uint32_t* big = reinterpret_cast<uint32_t*>(ws + L.big);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
    unsigned long long* alt = reinterpret_cast<unsigned long long*>(ws + L.alt);
    const size_t cnt_smem = (size_t)Tmax * 4;
    cudaError_t e = cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cnt_smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)nblk, (unsigned)V);
    hist_kernel<<<grid, kGB, cnt_smem, stream>>>(a, vd, hist);
    column_kernel<<<(Tt + 255) / 256, 256, 0, stream>>>(V, (int)nblk, vd, hist, total, Tt);
    scan_kernel<<<1, 1024, 0, stream>>>(Tt, total, start, a.tile_ranges, a.capacity, a.num_instances, big, a.status);
    scatter_kernel<<<grid, kGB, cnt_smem, stream>>>(a, vd, hist, start, keys);
    sort_warp_kernel<<<(Tt + 3) / 4, 128, 0, stream>>>((int)Tt, a.tile_ranges, keys, a.gauss_ids);
    sort_small_kernel<<<Tt, 128, 0, stream>>>(a.tile_ranges, keys, a.gauss_ids);
    const int large_smem = kChunk * 8;
    e = cudaFuncSetAttribute(sort_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, large_smem);
    if (e != cudaSuccess) return e;
    sort_large_kernel<<<64, 1024, large_smem, stream>>>(a.tile_ranges, big, keys, alt, a.gauss_ids);
    return cudaGetLastError();
}

}  // namespace lsv2
