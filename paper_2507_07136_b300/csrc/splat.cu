// splat.cu -- efficient sparse-coefficient splatting (Sec. 3.4, Algorithm 1) on sm_103a.
//
// Per pixel, front to back over its tile's depth-ordered list (Eq. 3), with the weights
// e_i = alpha_i prod_{j<i} (1 - alpha_j) of Eq. 7, only the K nonzero coefficients of each
// level are blended: W_lev[idx_k] += w_k e_i.  Blending stays in FP32.
//
// Layout on the SM (warps independent within a tile, no block barrier in the blend):
//  * One producer warp per CTA gathers the tile's records, 32 per batch, with bulk async copies
//    into a ring of shared-memory stages (full / empty mbarriers, every wait bounded) and writes
//    a compact culling box per record.
//  * Each consumer warp covers an 8 x 4 pixel block, one pixel per lane.  Its FP32 accumulators
//    are columns, col = lev * L + idx: in shared memory (acc[col][lane], a stride of 33 floats)
//    or, for consumer warps 4-7 of the 16 x 16 CTA of splat_tm_kernel, in the warp's TMEM lane
//    quarter (lane = pixel, TMEM column = col), so twice as many warps hide the blend's latency.
//    The codebook index of a Gaussian is the same for every pixel of the tile, so a pair update is
//    one conflict-free load / FFMA / store on a warp-uniform column.  (Registers cannot be
//    indexed by a runtime value; a jump table would cost a uniform indirect branch per pair.)
//  * A warp tests each record's alpha >= 1/255 box against its block; a ballot keeps the records
//    that can touch it, walked in list order four at a time: alpha of the four in parallel (with
//    the records' column offsets), the transmittance scan, then the accumulation of the records
//    some lane takes.  Culling skips only work whose alpha is below 1/255 everywhere on the
//    block, so it changes no result.
//  * A pre-pass packs per-Gaussian records (2D mean pair, principal frame of the conic,
//    opacity, weights, column offsets, culling extents).  Repeated indices within one level are
//    merged into one pair, and the emptied repeats and invalid indices point at a dummy column,
//    so a record's pairs carrying weight have distinct columns and all their loads can be issued
//    before any store.
#include "device.cuh"
#include "splat.cuh"
#include "splat_core.cuh"
#include "tc.cuh"

namespace lsv2 {

// One thread per (view, Gaussian): the record in registers (fully unrolled over the pairs, so no
// local memory), written with 16-byte stores.
template <int LEVELS, int K, int LW = 64>
__global__ void __launch_bounds__(256) pack_records_kernel(PackArgs a)
{
    constexpr int P = LEVELS * K;
    constexpr int kRecFloats = record_bytes(P) / 4;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // Gaussian
    if (g >= a.n) return;
    const int64_t o = (int64_t)blockIdx.y * a.n + g;                     // projection slot of this view
    float r[kRecFloats];
#pragma unroll
    for (int i = 0; i < kRecFloats; ++i) r[i] = 0.0f;
    const float4 m = reinterpret_cast<const float4*>(a.xy)[o];
    const float4 ax0 = reinterpret_cast<const float4*>(a.axes)[2 * o];
    const float4 ax1 = reinterpret_cast<const float4*>(a.axes)[2 * o + 1];
    const float op = reinterpret_cast<const float4*>(a.conic_o)[o].w;
    r[0] = m.x, r[1] = m.y, r[2] = m.z, r[3] = m.w;
    r[4] = ax0.x, r[5] = ax0.y, r[6] = ax0.z, r[7] = ax0.w;
    r[8] = ax1.x, r[9] = ax1.y, r[10] = ax1.z, r[11] = op;
    // gather the pairs; merge repeats of a column within a level into the first occurrence
    float wv[P];
    int col[P];
    bool real[P];
    bool bad = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int lev = p / K;
        const size_t src = (size_t)g * P + p;
        const int ix = a.idx[src];
        bad |= ix >= LW;
        col[p] = lev * LW + (ix < LW ? ix : 0);
        wv[p] = ix < LW ? a.w[src] : 0.0f;
        real[p] = ix < LW;
    }
    if (bad) report(a.status, LSV2_ERR_INVALID_ARGUMENT);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        bool merged = false;
#pragma unroll
        for (int p2 = (p / K) * K; p2 < p; ++p2) {
            const bool m2 = !merged && real[p] && real[p2] && col[p2] == col[p];
            wv[p2] = m2 ? wv[p2] + wv[p] : wv[p2];
            merged |= m2;
        }
        wv[p] = merged ? 0.0f : wv[p];
        real[p] = real[p] && !merged;
    }
    // within each level: emptied pairs first (pointing at the dummy column), real pairs last;
    // slot of each pair, then a gather
#pragma unroll
    for (int lev = 0; lev < LEVELS; ++lev) {
        int seen = 0, n_empty = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) n_empty += real[lev * K + k] ? 0 : 1;
        int slot[K];
        int e = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool rk = real[lev * K + k];
            slot[k] = rk ? n_empty + seen : e;
            seen += rk ? 1 : 0;
            e += rk ? 0 : 1;
        }
#pragma unroll
        for (int s2 = 0; s2 < K; ++s2) {
            float wsel = 0.0f;
            uint32_t csel = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const bool hit = slot[k] == s2;
                const bool rk = real[lev * K + k];
                wsel = hit ? (rk ? wv[lev * K + k] : 0.0f) : wsel;
                csel = hit ? (uint32_t)(rk ? col[lev * K + k] : LEVELS * LW) * 132u : csel;
            }
            r[12 + lev * K + s2] = wsel;
            r[12 + P + lev * K + s2] = __uint_as_float(csel);
        }
    }
    const float2 ex = reinterpret_cast<const float2*>(a.extent)[o];
    r[kRecFloats - 4] = ex.x;
    r[kRecFloats - 3] = ex.y;
    float4* dst = reinterpret_cast<float4*>(a.recs + (size_t)o * kRecFloats);
#pragma unroll
    for (int v = 0; v < kRecFloats / 4; ++v) dst[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
}

// Dense records for the comparison blend: the header of the sparse record, then every level's 64
// coefficients (the K pairs scattered, repeats summed in pair order, zeros elsewhere).
template <int LEVELS>
__global__ void __launch_bounds__(256) pack_dense_kernel(PackArgs a)
{
    constexpr int kRecFloats = dense_record_bytes(LEVELS) / 4;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    float* rec = a.recs + (size_t)g * kRecFloats;
    const float4 m = reinterpret_cast<const float4*>(a.xy)[g];
    const float4 ax0 = reinterpret_cast<const float4*>(a.axes)[2 * g];
    const float4 ax1 = reinterpret_cast<const float4*>(a.axes)[2 * g + 1];
    const float op = reinterpret_cast<const float4*>(a.conic_o)[g].w;
    reinterpret_cast<float4*>(rec)[0] = m;
    reinterpret_cast<float4*>(rec)[1] = ax0;
    reinterpret_cast<float4*>(rec)[2] = make_float4(ax1.x, ax1.y, ax1.z, op);
    for (int i = 12; i < kRecFloats; i += 4) *reinterpret_cast<float4*>(rec + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    bool bad = false;
    for (int lev = 0; lev < LEVELS; ++lev)
        for (int k = 0; k < a.K; ++k) {
            const size_t src = ((size_t)g * LEVELS + lev) * a.K + k;
            const int ix = a.idx[src];
            bad |= ix >= 64;
            if (ix < 64) rec[12 + lev * 64 + ix] += a.w[src];
        }
    if (bad) report(a.status, LSV2_ERR_INVALID_ARGUMENT);
    const float2 ex = reinterpret_cast<const float2*>(a.extent)[g];
    reinterpret_cast<float4*>(rec + kRecFloats - 4)[0] = make_float4(ex.x, ex.y, 0.f, 0.f);
}

// One CTA per TW x TH pixel block; SUB blocks stacked vertically share one bin tile of
// TW x (TH SUB) pixels (and its list), so a bin tile's halves can run as two CTAs per SM.
template <int LEVELS, int K, int TW, int TH, bool DENSE = false, int SUB = 1, int LW = 64>
__global__ void __launch_bounds__(TW* TH + 32, (TW * TH <= 128 && LW <= 64) ? 2 : 1) splat_kernel(SplatArgs a)
{
    using C = SplatCfg<LEVELS, K, TW, TH, 0, DENSE, LW>;
    extern __shared__ __align__(16) unsigned char smem[];
    const SplatSmem<C> sm(smem);
    if (threadIdx.x == 0) {
        sm.init();
        // after a wait ran out anywhere, the remaining tiles are skipped
        *sm.skip = a.status && *reinterpret_cast<volatile int32_t*>(a.status) == LSV2_ERR_TIMEOUT;
    }
    __syncthreads();
    if (*sm.skip) return;
    const int tile = blockIdx.x / SUB, sub = blockIdx.x % SUB;
    const int GX = (a.cam.width + TW - 1) / TW;
    TileJob j{a.cam.width, a.cam.height, (tile % GX) * TW, (tile / GX) * (TH * SUB) + sub * TH, a.tile_ranges[2 * tile],
              a.tile_ranges[2 * tile + 1], a.gauss_ids, a.recs, a.coeff, a.final_T, a.n_last, a.status,
              a.coeff_bf16};
    j.wait_ns = a.wait_ns;
    (void)splat_tile<LEVELS, K, TW, TH, 0, true, DENSE, LW>(j, sm, 0u);
}

// One CTA per 16 x 16 tile with eight consumer warps, the last four accumulating in TMEM (at
// L = 64: 256 columns per CTA, two CTAs per SM, the whole of the SM's TMEM), so an SM runs 16
// consumer warps where shared memory alone holds the accumulators of 8 (at L = 128: one CTA and
// 512 columns per SM, 8 consumer warps where shared memory alone holds those of 4).
template <int LEVELS, int K, int BATCH, int LW = 64>
__global__ void __launch_bounds__(16 * 16 + 32, LW <= 64 ? 2 : 1) splat_tm_kernel(SplatArgs a)
{
    using C = SplatCfg<LEVELS, K, 16, 16, BATCH, false, LW, 4>;
    constexpr uint32_t kSplatTmemCols = C::kTmemCols;
    extern __shared__ __align__(16) unsigned char smem[];
    const SplatSmem<C> sm(smem);
    if (threadIdx.x == 0) {
        sm.init();
        *sm.skip = a.status && *reinterpret_cast<volatile int32_t*>(a.status) == LSV2_ERR_TIMEOUT;
    }
    __syncthreads();
    if (*sm.skip) return;
    const int warp = threadIdx.x >> 5;
    if (warp == C::kSmemAccWarps) tc::tmem_alloc(tc::smem_u32(sm.tmem_slot), kSplatTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const int tile = blockIdx.x;
    const int GX = (a.cam.width + 15) / 16;
    TileJob j{a.cam.width, a.cam.height, (tile % GX) * 16, (tile / GX) * 16, a.tile_ranges[2 * tile],
              a.tile_ranges[2 * tile + 1], a.gauss_ids, a.recs, a.coeff, a.final_T, a.n_last, a.status,
              a.coeff_bf16};
    j.wait_ns = a.wait_ns;
    (void)splat_tile_tm<C, LEVELS, K>(j, sm, 0u);
    // every TMEM access of the tile completed before splat_tile_tm's barrier
    if (warp == C::kSmemAccWarps) tc::tmem_dealloc(*sm.tmem_slot, kSplatTmemCols);
}

// Persistent over the (view, tile) work items of several views: each CTA takes the next work
// item from an atomic counter (largest views first, as they come first in the numbering); a
// TW x (TH SUB) bin tile is SUB items of TW x TH pixels.
template <int LEVELS, int K, int TW, int TH, int BATCH, int SUB = 1>
__global__ void __launch_bounds__(TW* TH + 32, 1) splat_views_kernel(SplatViewsArgs a)
{
    using C = SplatCfg<LEVELS, K, TW, TH, BATCH>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tile;
    const SplatSmem<C> sm(smem);
    if (threadIdx.x == 0) sm.init();
    uint32_t bbase = 0;
    while (true) {
        if (threadIdx.x == 0) {
            s_tile = (int)atomicAdd(a.queue, 1u);
            *sm.skip = *sm.abort || (a.status && *reinterpret_cast<volatile int32_t*>(a.status) == LSV2_ERR_TIMEOUT);
        }
        __syncthreads();
        const int item = s_tile;
        const bool stop = *sm.skip;
        __syncthreads();
        const int tg = item / SUB, sub = item % SUB;
        if (tg >= a.total_tiles || stop) break;
        int v = 0;
        while (v + 1 < a.V && tg >= a.view[v + 1].tile_base) ++v;
        const SplatView& w = a.view[v];
        const int tl = tg - w.tile_base;
        TileJob j{w.width, w.height, (tl % w.GX) * TW, (tl / w.GX) * (TH * SUB) + sub * TH, a.tile_ranges[2 * tg],
                  a.tile_ranges[2 * tg + 1],
                  a.gauss_ids, a.recs + w.rec_off,
                  a.coeff_bf16 ? reinterpret_cast<float*>(reinterpret_cast<__nv_bfloat16*>(a.coeff) + w.coeff_off)
                               : a.coeff + w.coeff_off,
                  a.final_T + w.pix_off, a.n_last + w.pix_off, a.status, a.coeff_bf16};
        j.wait_ns = a.wait_ns;
        bbase += splat_tile<LEVELS, K, TW, TH, BATCH>(j, sm, bbase);
    }
}

// The multi-view splat over 16 x 16 tiles with TMEM accumulators for consumer warps 4-7 (as
// splat_tm_kernel), persistent: the CTA allocates its TMEM once and takes tiles from the queue.
template <int LEVELS, int K, int BATCH>
__global__ void __launch_bounds__(16 * 16 + 32, 2) splat_views_tm_kernel(SplatViewsArgs a)
{
    using C = SplatCfg<LEVELS, K, 16, 16, BATCH, false, 64, 4>;
    constexpr uint32_t kSplatTmemCols = C::kTmemCols;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tile;
    const SplatSmem<C> sm(smem);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) sm.init();
    if (warp == C::kSmemAccWarps) tc::tmem_alloc(tc::smem_u32(sm.tmem_slot), kSplatTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    uint32_t bbase = 0;
    while (true) {
        if (threadIdx.x == 0) {
            s_tile = (int)atomicAdd(a.queue, 1u);
            *sm.skip = *sm.abort || (a.status && *reinterpret_cast<volatile int32_t*>(a.status) == LSV2_ERR_TIMEOUT);
        }
        __syncthreads();
        const int tg = s_tile;
        const bool stop = *sm.skip;
        __syncthreads();
        if (tg >= a.total_tiles || stop) break;
        int v = 0;
        while (v + 1 < a.V && tg >= a.view[v + 1].tile_base) ++v;
        const SplatView& w = a.view[v];
        const int tl = tg - w.tile_base;
        TileJob j{w.width, w.height, (tl % w.GX) * 16, (tl / w.GX) * 16, a.tile_ranges[2 * tg], a.tile_ranges[2 * tg + 1],
                  a.gauss_ids, a.recs + w.rec_off,
                  a.coeff_bf16 ? reinterpret_cast<float*>(reinterpret_cast<__nv_bfloat16*>(a.coeff) + w.coeff_off)
                               : a.coeff + w.coeff_off,
                  a.final_T + w.pix_off, a.n_last + w.pix_off, a.status, a.coeff_bf16};
        j.wait_ns = a.wait_ns;
        bbase += splat_tile_tm<C, LEVELS, K>(j, sm, bbase);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == C::kSmemAccWarps) tc::tmem_dealloc(*sm.tmem_slot, kSplatTmemCols);
}

namespace {

// CTAs per 16 x 16 bin tile (two CTAs of 16 x 8 pixels share an SM)
constexpr int kSub16 = 2;

// Bin tiles of TW x TH pixels, each run as SUB CTAs of TW x (TH / SUB) pixels.
template <int LEVELS, int K, int TW, int TH, bool DENSE = false, int SUB = 1, int LW = 64>
cudaError_t launch_t(const SplatArgs& a, cudaStream_t stream)
{
    constexpr int kTHc = TH / SUB;
    using C = SplatCfg<LEVELS, K, TW, kTHc, 0, DENSE, LW>;
    static_assert(C::kSmemBytes <= 232448, "shared memory budget");
    auto kern = splat_kernel<LEVELS, K, TW, kTHc, DENSE, SUB, LW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    const int GX = (a.cam.width + TW - 1) / TW, GY = (a.cam.height + TH - 1) / TH;
    if (GX * GY == 0) return cudaSuccess;
    kern<<<GX * GY * SUB, C::kThreads, C::kSmemBytes, stream>>>(a);
    return cudaGetLastError();
}

template <int LEVELS, int K, int LW = 64>
cudaError_t launch_tm(const SplatArgs& a, cudaStream_t stream)
{
    // 32 records per stage, 16 for the larger records of K >= 6 (two stages must fit twice per SM)
    constexpr int kBatch = record_bytes(LEVELS * K) <= 160 ? 32 : 16;
    using C = SplatCfg<LEVELS, K, 16, 16, kBatch, false, LW, 4>;
    // the CTAs an SM holds (by shared memory) must fit its 512 TMEM columns together
    constexpr int kPerSm = 233472 / (C::kSmemBytes + 1024);
    static_assert(kPerSm >= 1 && kPerSm * C::kTmemCols <= 512, "TMEM of the resident CTAs");
    auto kern = splat_tm_kernel<LEVELS, K, kBatch, LW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    const int GX = (a.cam.width + 15) / 16, GY = (a.cam.height + 15) / 16;
    if (GX * GY == 0) return cudaSuccess;
    kern<<<GX * GY, C::kThreads, C::kSmemBytes, stream>>>(a);
    return cudaGetLastError();
}

template <int LEVELS, int K, int BATCH>
cudaError_t launch_views_tm(const SplatViewsArgs& a, int num_sms, cudaStream_t stream)
{
    using C = SplatCfg<LEVELS, K, 16, 16, BATCH, false, 64, 4>;
    static_assert(2 * (C::kSmemBytes + 1024) <= 233472 && 3 * (C::kSmemBytes + 1024) > 233472, "two CTAs per SM");
    auto kern = splat_views_tm_kernel<LEVELS, K, BATCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    if (a.total_tiles == 0) return cudaSuccess;
    e = cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    kern<<<num_sms * 2, C::kThreads, C::kSmemBytes, stream>>>(a);
    return cudaGetLastError();
}

template <int LEVELS, int K, int TW, int TH, int BATCH, int SUB = 1>
cudaError_t launch_views_t(const SplatViewsArgs& a, int num_sms, cudaStream_t stream)
{
    using C = SplatCfg<LEVELS, K, TW, TH, BATCH>;
    static_assert(C::kSmemBytes <= 232448, "shared memory budget");
    auto kern = splat_views_kernel<LEVELS, K, TW, TH, BATCH, SUB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::kThreads, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (a.total_tiles == 0) return cudaSuccess;
    e = cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    kern<<<num_sms * per_sm, C::kThreads, C::kSmemBytes, stream>>>(a);
    return cudaGetLastError();
}

// TW x TH bin tiles as SUB CTAs of TW x (TH / SUB) pixels
template <int LEVELS, int K, int TW, int TH, int SUB = 1>
cudaError_t launch_views_b(const SplatViewsArgs& a, int batch, int num_sms, cudaStream_t stream)
{
    constexpr int kTHc = TH / SUB;
    using Auto = SplatCfg<LEVELS, K, TW, kTHc>;
    if (batch == 16) return launch_views_t<LEVELS, K, TW, kTHc, 16, SUB>(a, num_sms, stream);
    if (batch == 0 || batch == Auto::kBatch)
        return launch_views_t<LEVELS, K, TW, kTHc, Auto::kBatch, SUB>(a, num_sms, stream);
    return cudaErrorInvalidValue;
}

template <int LEVELS, int K>
cudaError_t launch_views_tile(const SplatViewsArgs& a, int tw, int th, int batch, int num_sms, cudaStream_t stream)
{
    if (tw == 16 && th == 16) {
        if constexpr (LEVELS == 3 && K == 4) {   // TMEM accumulators for half the consumer warps
            if (batch == 16) return launch_views_tm<LEVELS, K, 16>(a, num_sms, stream);
            if (batch == 0 || batch == 32) return launch_views_tm<LEVELS, K, 32>(a, num_sms, stream);
            return cudaErrorInvalidValue;
        }
        return launch_views_b<LEVELS, K, 16, 16, kSub16>(a, batch, num_sms, stream);
    }
    if (tw == 8 && th == 8) return launch_views_b<LEVELS, K, 8, 8>(a, batch, num_sms, stream);
    if (tw == 32 && th == 8) return launch_views_b<LEVELS, K, 32, 8>(a, batch, num_sms, stream);
    return cudaErrorInvalidValue;
}

template <int LEVELS, int K>
cudaError_t launch_tile(const SplatArgs& a, cudaStream_t stream)
{
    if (a.cam.tile_w == 16 && a.cam.tile_h == 16) return launch_t<LEVELS, K, 16, 16, false, kSub16>(a, stream);
    if (a.cam.tile_w == 8 && a.cam.tile_h == 8) return launch_t<LEVELS, K, 8, 8>(a, stream);
    if (a.cam.tile_w == 32 && a.cam.tile_h == 8) return launch_t<LEVELS, K, 32, 8>(a, stream);
    return cudaErrorInvalidValue;
}

}  // namespace

bool splat_supported(int levels, int K, int L, int tw, int th)
{
    // the L sweep: codebooks of 32 and 128 entries at three levels, K = 4, 16 x 16 tiles; and an
    // 8-column map at three levels (the low-dimensional latent of the decoder-based comparison path)
    if (L == 8 || L == 32 || L == 128) return levels == 3 && K == 4 && tw == 16 && th == 16;
    if (L != 64) return false;
    const bool tile_ok = (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 32 && th == 8);
    if (!tile_ok) return false;
    if (levels == 1) return K == 2 || K == 4 || K == 6 || K == 8;
    if (levels == 2) return K == 4;
    if (levels == 3) return K == 4 || (tw == 16 && th == 16 && (K == 2 || K == 6 || K == 8));
    return false;
}

bool splat_dense_supported(int levels, int L, int tw, int th)
{
    return L == 64 && (levels == 1 || levels == 3) && tw == 16 && th == 16;
}

int splat_dense_record_bytes(int levels) { return dense_record_bytes(levels); }

cudaError_t launch_pack_dense(const PackArgs& a, cudaStream_t stream)
{
    if (a.n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((a.n + 255) / 256);
    if (a.levels == 3) pack_dense_kernel<3><<<blocks, 256, 0, stream>>>(a);
    else if (a.levels == 1) pack_dense_kernel<1><<<blocks, 256, 0, stream>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_splat_dense(int levels, const SplatArgs& args, cudaStream_t stream)
{
    SplatArgs a = args;
    a.wait_ns = wait_limit_ns();
    if (levels == 3) return launch_t<3, 4, 16, 16, true>(a, stream);
    if (levels == 1) return launch_t<1, 4, 16, 16, true>(a, stream);
    return cudaErrorInvalidValue;
}

int splat_record_bytes(int levels, int K) { return record_bytes(levels * K); }


cudaError_t launch_pack(const PackArgs& a, cudaStream_t stream, int V)
{
    if (a.n == 0 || V == 0) return cudaSuccess;
    const int threads = 256;
    const dim3 grid((unsigned)((a.n + threads - 1) / threads), (unsigned)V);
    if (a.L != 64) {   // the L sweep: three levels, K = 4
        if (a.levels == 3 && a.K == 4 && a.L == 8) pack_records_kernel<3, 4, 8><<<grid, threads, 0, stream>>>(a);
        else if (a.levels == 3 && a.K == 4 && a.L == 32) pack_records_kernel<3, 4, 32><<<grid, threads, 0, stream>>>(a);
        else if (a.levels == 3 && a.K == 4 && a.L == 128) pack_records_kernel<3, 4, 128><<<grid, threads, 0, stream>>>(a);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    if (a.levels == 3 && a.K == 4) pack_records_kernel<3, 4><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 3 && a.K == 2) pack_records_kernel<3, 2><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 3 && a.K == 6) pack_records_kernel<3, 6><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 3 && a.K == 8) pack_records_kernel<3, 8><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 2 && a.K == 4) pack_records_kernel<2, 4><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 1 && a.K == 2) pack_records_kernel<1, 2><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 1 && a.K == 4) pack_records_kernel<1, 4><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 1 && a.K == 6) pack_records_kernel<1, 6><<<grid, threads, 0, stream>>>(a);
    else if (a.levels == 1 && a.K == 8) pack_records_kernel<1, 8><<<grid, threads, 0, stream>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_splat_views(int levels, int K, int tw, int th, int batch, const SplatViewsArgs& args, int num_sms,
                               cudaStream_t stream)
{
    SplatViewsArgs a = args;
    a.wait_ns = wait_limit_ns();
    if (levels == 1 && K == 4) return launch_views_tile<1, 4>(a, tw, th, batch, num_sms, stream);
    if (levels == 2 && K == 4) return launch_views_tile<2, 4>(a, tw, th, batch, num_sms, stream);
    if (levels == 3 && K == 4) return launch_views_tile<3, 4>(a, tw, th, batch, num_sms, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_splat(int levels, int K, const SplatArgs& args, cudaStream_t stream)
{
    SplatArgs a = args;
    a.wait_ns = wait_limit_ns();
    if (levels == 1) {
        switch (K) {
            case 2: return launch_tile<1, 2>(a, stream);
            case 4: return launch_tile<1, 4>(a, stream);
            case 6: return launch_tile<1, 6>(a, stream);
            case 8: return launch_tile<1, 8>(a, stream);
        }
    }
    if (levels == 2 && K == 4) return launch_tile<2, 4>(a, stream);
    if (levels == 3 && K == 4 && a.L == 8) return launch_t<3, 4, 16, 16, false, kSub16, 8>(a, stream);
    if (levels == 3 && K == 4 && a.L == 32) return launch_t<3, 4, 16, 16, false, kSub16, 32>(a, stream);
    if (levels == 3 && K == 4 && a.L == 128 && a.cam.tile_w == 16 && a.cam.tile_h == 16)
        return launch_tm<3, 4, 128>(a, stream);
    if (a.L != 64) return cudaErrorInvalidValue;
    if (levels == 3 && K == 4) {
        if (a.cam.tile_w == 16 && a.cam.tile_h == 16) return launch_tm<3, 4>(a, stream);
        return launch_tile<3, 4>(a, stream);
    }
    if (levels == 3 && a.cam.tile_w == 16 && a.cam.tile_h == 16) {   // K sweep at three levels
        // TMEM accumulators pay at K = 2 (as at K = 4); at K = 6 and 8 the 18-24 TMEM loads and
        // stores per record and the smaller stages make them slower than one CTA of eight
        // shared-memory warps per tile (1.28 and 1.86 ms against 1.06 and 1.26 ms)
        if (K == 2) return launch_tm<3, 2>(a, stream);
        if (K == 6) return launch_t<3, 6, 16, 16>(a, stream);
        if (K == 8) return launch_t<3, 8, 16, 16>(a, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lsv2
