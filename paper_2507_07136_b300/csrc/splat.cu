// splat.cu -- efficient sparse-coefficient splatting (Sec. 3.4, Algorithm 1) on sm_103a.
//
// Per pixel, front to back over its tile's depth-ordered list (Eq. 3), with the weights
// e_i = alpha_i prod_{j<i} (1 - alpha_j) of Eq. 7, only the K nonzero coefficients of each
// level are blended: W_lev[idx_k] += w_k e_i.  Blending stays in FP32.
//
// Layout on the SM (one CTA per tile, one thread per pixel, warps independent):
//  * Every warp owns the FP32 accumulators of its 32 pixels in shared memory as columns:
//    acc[col][lane] with col = lev * 64 + idx and a stride of 33 floats.  The codebook index
//    of a Gaussian is the same for every pixel of the tile, so a pair update is one
//    conflict-free LDS / FFMA / STS on a warp-uniform column.  (Registers cannot be indexed
//    by a runtime value on this architecture; a jump table would cost a uniform indirect
//    branch per pair.)
//  * Gaussians are staged per warp in batches of 32 records (one 16-byte-vector gather per
//    lane, issued one batch ahead into registers).  Each lane tests its record's alpha >= 1/255 bounding box
//    against the warp's pixel strip; a ballot keeps only the records that can touch the strip
//    and the warp walks the set bits in list order ("warp-ballot culling").  Culling skips
//    only work whose alpha is below 1/255 everywhere on the strip, so it changes no result.
//  * A pre-pass packs per-Gaussian records (2D mean pair, principal frame of the conic,
//    opacity, weights, columns).  Repeated indices within one level are merged into one pair
//    and the emptied repeats are stored first, so the loads of a record's pairs can all be
//    issued before any store.
#include "device.cuh"
#include "splat.cuh"

namespace lsv2 {

__global__ void __launch_bounds__(256) pack_records_kernel(PackArgs a)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // Gaussian
    if (g >= a.n) return;
    const int64_t o = (int64_t)blockIdx.y * a.n + g;                     // projection slot of this view
    const int P = a.levels * a.K;
    const int rec_floats = a.rec_bytes / 4;
    float* rec = a.recs + (size_t)o * rec_floats;
    const float4 ax1 = reinterpret_cast<const float4*>(a.axes)[2 * o + 1];
    reinterpret_cast<float4*>(rec)[0] = reinterpret_cast<const float4*>(a.xy)[o];
    reinterpret_cast<float4*>(rec)[1] = reinterpret_cast<const float4*>(a.axes)[2 * o];
    reinterpret_cast<float4*>(rec)[2] = make_float4(ax1.x, ax1.y, ax1.z, reinterpret_cast<const float4*>(a.conic_o)[o].w);
    // gather pairs, merge repeats of a column into the first occurrence
    float wv[kMaxPairs];
    int col[kMaxPairs];
    bool real[kMaxPairs];
    for (int lev = 0; lev < a.levels; ++lev)
        for (int k = 0; k < a.K; ++k) {
            const int p = lev * a.K + k;
            const size_t src = ((size_t)g * a.levels + lev) * a.K + k;
            const int ix = a.idx[src];
            col[p] = lev * 64 + (ix < 64 ? ix : 0);
            wv[p] = ix < 64 ? a.w[src] : 0.0f;
            real[p] = ix < 64;
            if (ix >= 64) report(a.status, LSV2_ERR_INVALID_ARGUMENT);
            for (int p2 = lev * a.K; p2 < p; ++p2)
                if (real[p] && real[p2] && col[p2] == col[p]) {
                    wv[p2] += wv[p];
                    wv[p] = 0.0f;
                    real[p] = false;
                    break;
                }
        }
    // within each level: emptied pairs first (pointing at the level's first real column), real
    // pairs last, so every level's K slots stay contiguous
    uint8_t* cb = reinterpret_cast<uint8_t*>(rec + 12 + P);
    for (int lev = 0; lev < a.levels; ++lev) {
        const int p0 = lev * a.K;
        int first_real = -1;
        for (int p = p0; p < p0 + a.K; ++p)
            if (real[p]) {
                first_real = p;
                break;
            }
        int slot = p0;
        for (int p = p0; p < p0 + a.K; ++p)
            if (!real[p]) {
                rec[12 + slot] = 0.0f;
                cb[slot] = (uint8_t)(first_real >= 0 ? col[first_real] : lev * 64);
                ++slot;
            }
        for (int p = p0; p < p0 + a.K; ++p)
            if (real[p]) {
                rec[12 + slot] = wv[p];
                cb[slot] = (uint8_t)col[p];
                ++slot;
            }
    }
    reinterpret_cast<float2*>(rec + rec_floats - 4)[0] = reinterpret_cast<const float2*>(a.extent)[o];
}

// One tile of one view.  Only this warp's shared-memory region is touched, so the warps of a
// CTA need no barrier between them.
struct TileJob {
    int width, height, GX, tile, lev0;   // lev0: first level accumulated by this CTA
    uint32_t beg, end;
    const uint32_t* gauss_ids;
    const float* recs;
    float* coeff;
    float* final_T;
    uint32_t* n_last;
};

template <int LEVELS, int K, int TW, int TH, int BATCH = 0, int LCTA = LEVELS>
__device__ __forceinline__ void splat_tile(const TileJob& a, float* smem)
{
    using C = SplatCfg<LEVELS, K, TW, TH, BATCH, LCTA>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* acc = smem + warp * C::kAccFloats;
    float* stage = smem + C::kWarps * C::kAccFloats + warp * (C::kBatch * C::kSmemRecFloats);

    const int GX = a.GX;
    const int tile = a.tile;
    const int tx = tile % GX, ty = tile / GX;
    const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
    const int px = tx * TW + lx, py = ty * TH + ly;
    const bool inside = px < a.width && py < a.height;
    // pixel strip covered by this warp
    constexpr int kRows = 32 / TW;
    const float wx0 = (float)(tx * TW), wx1 = (float)(tx * TW + TW - 1);
    const float wy0 = (float)(ty * TH + warp * kRows), wy1 = wy0 + (float)(kRows - 1);

    for (int i = lane * 4; i < C::kAccFloats; i += 128)
        *reinterpret_cast<float4*>(acc + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();

    const uint32_t beg = a.beg, end = a.end;
    float T = 1.0f;
    uint32_t last = 0;
    bool done = !inside;
    const float pxf = (float)px, pyf = (float)py;

    // Next batch's record for this lane, fetched into registers while the current batch is
    // processed (the gather from L2 is the other latency the warp would otherwise wait on).
    constexpr int kV = C::kSmemRecFloats / 4;
    float4 nx[kV];
    float2 nex = make_float2(-1.0f, -1.0f);
    bool nvalid = false;
    auto fetch = [&](uint32_t b) {
        const uint32_t j = b + lane;
        nvalid = lane < C::kBatch && j < end;
        if (nvalid) {
            const uint32_t g = a.gauss_ids[j];
            const float4* src = reinterpret_cast<const float4*>(a.recs + (size_t)g * C::kRecFloats);
#pragma unroll
            for (int v = 0; v < kV; ++v) nx[v] = __ldg(src + v);
            nex = __ldg(reinterpret_cast<const float2*>(a.recs + (size_t)g * C::kRecFloats + C::kRecFloats - 4));
        }
    };
    if (beg < end) fetch(beg);

    for (uint32_t base = beg; base < end; base += C::kBatch) {
        if (__all_sync(0xffffffffu, done)) break;
        const bool keep = nvalid && nex.x >= 0.0f && nx[0].x + nex.x >= wx0 && nx[0].x - nex.x <= wx1 &&
                          nx[0].y + nex.y >= wy0 && nx[0].y - nex.y <= wy1;
        if (keep) {
            float4* dst = reinterpret_cast<float4*>(stage + lane * C::kSmemRecFloats);
#pragma unroll
            for (int v = 0; v < kV; ++v) dst[v] = nx[v];
        }
        uint32_t mask = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (base + C::kBatch < end) fetch(base + C::kBatch);
        if (mask) {
            // software pipeline: the next record's power and 2^power (independent of T) are
            // formed before this record's transmittance update and accumulation
            int i = __ffs(mask) - 1;
            mask &= mask - 1;
            const float* r = stage + i * C::kSmemRecFloats;
            float p2 = eval_power2(*reinterpret_cast<const float4*>(r), *reinterpret_cast<const float4*>(r + 4),
                                   *reinterpret_cast<const float4*>(r + 8), pxf, pyf);
            float o = r[11];
            float ex2;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex2) : "f"(p2));
            while (true) {
                int jn = -1;
                const float* rn = r;
                float p2n = 0.0f, on = 0.0f, exn = 0.0f;
                if (mask) {
                    jn = __ffs(mask) - 1;
                    mask &= mask - 1;
                    rn = stage + jn * C::kSmemRecFloats;
                    p2n = eval_power2(*reinterpret_cast<const float4*>(rn), *reinterpret_cast<const float4*>(rn + 4),
                                      *reinterpret_cast<const float4*>(rn + 8), pxf, pyf);
                    on = rn[11];
                    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(exn) : "f"(p2n));
                }
                float e = 0.0f;
                if (!done && p2 <= 0.0f) {
                    const float alpha = fminf(kAlphaMax, o * ex2);
                    if (alpha >= kAlphaMin) {
                        const float test_T = T * one_minus_alpha(alpha, o, p2);
                        if (test_T < kTMin) {
                            done = true;
                        } else {
                            e = alpha * T;
                            T = test_T;
                            last = base + i - beg + 1;
                        }
                    }
                }
                if (__any_sync(0xffffffffu, e > 0.0f)) {
                    const float* wr = r + 12 + a.lev0 * K;
                    const uint8_t* cr = reinterpret_cast<const uint8_t*>(r + 12 + C::kPairs) + a.lev0 * K;
                    const int cbase = a.lev0 * 64;
                    float v[C::kCtaPairs];
                    int off[C::kCtaPairs];
#pragma unroll
                    for (int p = 0; p < C::kCtaPairs; ++p) {
                        off[p] = ((int)cr[p] - cbase) * 33 + lane;
                        v[p] = acc[off[p]];
                    }
#pragma unroll
                    for (int p = 0; p < C::kCtaPairs; ++p) v[p] = fmaf(e, wr[p], v[p]);
#pragma unroll
                    for (int p = 0; p < C::kCtaPairs; ++p) acc[off[p]] = v[p];
                }
                if (jn < 0) break;
                i = jn;
                r = rn;
                p2 = p2n;
                o = on;
                ex2 = exn;
            }
        }
        __syncwarp();
    }

    if (inside && a.lev0 == 0) {
        const size_t pix = (size_t)py * a.width + px;
        a.final_T[pix] = T;
        a.n_last[pix] = last;
    }
    __syncwarp();
    // write this warp's 32 pixels: per row segment TW pixels x 64 floats (contiguous in HBM)
    const size_t P = (size_t)a.width * a.height;
#pragma unroll
    for (int lc = 0; lc < LCTA; ++lc) {
        const int lev = a.lev0 + lc;
        for (int q = lane; q < 32 * 16; q += 32) {
            const int pl = q >> 4;  // pixel within the warp (row-major over the strip)
            const int c4 = (q & 15) * 4;
            const int gx = tx * TW + (pl % TW), gy = ty * TH + warp * kRows + pl / TW;
            if (gx < a.width && gy < a.height) {
                const float* col = acc + (lc * 64 + c4) * 33 + pl;
                float4 val = make_float4(col[0], col[33], col[66], col[99]);
                __stcs(reinterpret_cast<float4*>(a.coeff + ((size_t)lev * P + (size_t)gy * a.width + gx) * 64 + c4), val);
            }
        }
    }
}

template <int LEVELS, int K, int TW, int TH, int LCTA>
__global__ void __launch_bounds__(TW* TH) splat_kernel(SplatArgs a)
{
    extern __shared__ __align__(16) float smem[];
    const int tile = blockIdx.x;
    TileJob j{a.cam.width, a.cam.height, (a.cam.width + TW - 1) / TW, tile, (int)blockIdx.y * LCTA,
              a.tile_ranges[2 * tile], a.tile_ranges[2 * tile + 1], a.gauss_ids, a.recs, a.coeff, a.final_T,
              a.n_last};
    splat_tile<LEVELS, K, TW, TH, 0, LCTA>(j, smem);
}

// Persistent over the (view, tile) work items of several views: each CTA takes the next global
// tile id from an atomic counter (largest views first, as they come first in the numbering).
template <int LEVELS, int K, int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW* TH) splat_views_kernel(SplatViewsArgs a)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_tile;
    while (true) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int tg = s_tile;
        __syncthreads();
        if (tg >= a.total_tiles) break;
        int v = 0;
        while (v + 1 < a.V && tg >= a.view[v + 1].tile_base) ++v;
        const SplatView& w = a.view[v];
        TileJob j{w.width, w.height, w.GX, tg - w.tile_base, 0, a.tile_ranges[2 * tg], a.tile_ranges[2 * tg + 1],
                  a.gauss_ids, a.recs + w.rec_off, a.coeff + w.coeff_off, a.final_T + w.pix_off,
                  a.n_last + w.pix_off};
        splat_tile<LEVELS, K, TW, TH, BATCH>(j, smem);
    }
}

namespace {

template <int LEVELS, int K, int TW, int TH, int LCTA>
cudaError_t launch_t(const SplatArgs& a, cudaStream_t stream)
{
    using C = SplatCfg<LEVELS, K, TW, TH, 0, LCTA>;
    static_assert(C::kSmemBytes <= 232448, "shared memory budget");
    auto kern = splat_kernel<LEVELS, K, TW, TH, LCTA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    const int GX = (a.cam.width + TW - 1) / TW, GY = (a.cam.height + TH - 1) / TH;
    if (GX * GY == 0) return cudaSuccess;
    kern<<<dim3(GX * GY, LEVELS / LCTA), TW * TH, C::kSmemBytes, stream>>>(a);
    return cudaGetLastError();
}

template <int LEVELS, int K, int TW, int TH>
cudaError_t launch_split(const SplatArgs& a, cudaStream_t stream)
{
    return launch_t<LEVELS, K, TW, TH, LEVELS>(a, stream);
}

template <int LEVELS, int K, int TW, int TH, int BATCH>
cudaError_t launch_views_t(const SplatViewsArgs& a, int num_sms, cudaStream_t stream)
{
    using C = SplatCfg<LEVELS, K, TW, TH, BATCH>;
    static_assert(C::kSmemBytes <= 232448, "shared memory budget");
    auto kern = splat_views_kernel<LEVELS, K, TW, TH, BATCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TW * TH, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (a.total_tiles == 0) return cudaSuccess;
    e = cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    kern<<<num_sms * per_sm, TW * TH, C::kSmemBytes, stream>>>(a);
    return cudaGetLastError();
}

template <int LEVELS, int K, int TW, int TH>
cudaError_t launch_views_b(const SplatViewsArgs& a, int batch, int num_sms, cudaStream_t stream)
{
    using Auto = SplatCfg<LEVELS, K, TW, TH>;
    if (batch == 16) return launch_views_t<LEVELS, K, TW, TH, 16>(a, num_sms, stream);
    if (batch == 0 || batch == Auto::kBatch) return launch_views_t<LEVELS, K, TW, TH, Auto::kBatch>(a, num_sms, stream);
    return cudaErrorInvalidValue;   // 32 does not fit this configuration's shared memory
}

template <int LEVELS, int K>
cudaError_t launch_views_tile(const SplatViewsArgs& a, int tw, int th, int batch, int num_sms, cudaStream_t stream)
{
    if (tw == 16 && th == 16) return launch_views_b<LEVELS, K, 16, 16>(a, batch, num_sms, stream);
    if (tw == 8 && th == 8) return launch_views_b<LEVELS, K, 8, 8>(a, batch, num_sms, stream);
    if (tw == 32 && th == 8) return launch_views_b<LEVELS, K, 32, 8>(a, batch, num_sms, stream);
    return cudaErrorInvalidValue;
}

template <int LEVELS, int K>
cudaError_t launch_tile(const SplatArgs& a, cudaStream_t stream)
{
    if (a.cam.tile_w == 16 && a.cam.tile_h == 16) return launch_split<LEVELS, K, 16, 16>(a, stream);
    if (a.cam.tile_w == 8 && a.cam.tile_h == 8) return launch_split<LEVELS, K, 8, 8>(a, stream);
    if (a.cam.tile_w == 32 && a.cam.tile_h == 8) return launch_split<LEVELS, K, 32, 8>(a, stream);
    return cudaErrorInvalidValue;
}

}  // namespace

bool splat_supported(int levels, int K, int L, int tw, int th)
{
    if (L != 64) return false;
    const bool tile_ok = (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 32 && th == 8);
    if (!tile_ok) return false;
    if (levels == 1) return K == 2 || K == 4 || K == 6 || K == 8;
    if (levels == 2 || levels == 3) return K == 4;
    return false;
}

int splat_record_bytes(int levels, int K) { return record_bytes(levels * K); }


cudaError_t launch_pack(const PackArgs& a, cudaStream_t stream, int V)
{
    if (a.n == 0 || V == 0) return cudaSuccess;
    const int threads = 256;
    pack_records_kernel<<<dim3((unsigned)((a.n + threads - 1) / threads), (unsigned)V), threads, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_splat_views(int levels, int K, int tw, int th, int batch, const SplatViewsArgs& a, int num_sms,
                               cudaStream_t stream)
{
    if (levels == 1 && K == 4) return launch_views_tile<1, 4>(a, tw, th, batch, num_sms, stream);
    if (levels == 2 && K == 4) return launch_views_tile<2, 4>(a, tw, th, batch, num_sms, stream);
    if (levels == 3 && K == 4) return launch_views_tile<3, 4>(a, tw, th, batch, num_sms, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_splat(int levels, int K, const SplatArgs& a, cudaStream_t stream)
{
    if (levels == 1) {
        switch (K) {
            case 2: return launch_tile<1, 2>(a, stream);
            case 4: return launch_tile<1, 4>(a, stream);
            case 6: return launch_tile<1, 6>(a, stream);
            case 8: return launch_tile<1, 8>(a, stream);
        }
    }
    if (levels == 2 && K == 4) return launch_tile<2, 4>(a, stream);
    if (levels == 3 && K == 4) return launch_tile<3, 4>(a, stream);
    return cudaErrorInvalidValue;
}

}  // namespace lsv2
