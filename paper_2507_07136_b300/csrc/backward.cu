// backward.cu -- gradients of an L1 feature loss through decode, splat and projection.
//
// The paper trains the coefficient field (Sec. 3.3, Sec. 4.1) but gives no gradient; this
// is the adjoint of the forward path implemented here.
//
// 1. The decode adjoint (Loss = mean |F - target|, F = W S, Eq. 7) is in backward_tc.cu.
// 2. splat_backward: per pixel, back to front from its last contributor.  The transmittance
//    is recomputed from final_T as T_i = T_{i+1} / (1 - alpha_i).  Because each Gaussian has
//    only K nonzeros per level, the running sum of later contributions is one scalar:
//        g_i = sum_pairs dW[col] w,   dalpha_i = T_i (g_i - B),   B <- alpha_i g_i + (1 - alpha_i) B.
//    Gaussians are taken two at a time where their quantities fit 32 lanes (independent
//    evaluations; the transmittance and running sum pass from one to the next); the per-Gaussian
//    sums over the 32 pixels of a warp use one butterfly reduce-scatter (31 shuffles for up to 32
//    quantities), then one atomic per quantity.  The list entries and records of the next batch
//    are loaded while the current batch is evaluated.
// 3. project_backward: one thread per Gaussian, chain rule from (u, v, conic) to (mean,
//    scale, quaternion) through Sigma' = N N^T + 0.3 I, N = J W R diag(s).
#include "device.cuh"
#include "backward.cuh"
#include "tc.cuh"

#include <algorithm>

namespace lsv2 {
namespace {

// ------------------------------------------------------------------------------------ 2
// Backward splat record (global, per Gaussian): g0 = (u_hi, v_hi, u_lo, v_lo), the principal
// frame and opacity exactly as in the forward record (so alpha is recomputed bit for bit), the
// conic (a, b, c) and the culling half-width ex.x, then P weights and P column bytes (no merging),
// and the culling half-height ex.y in the record's last float.
__host__ __device__ constexpr int bwd_record_floats(int P) { return (64 + 5 * P + 15) / 16 * 4; }
// floats in use before the last one: header 16, P weights, P column bytes
__host__ __device__ constexpr bool bwd_record_last_free(int P) { return 16 + P + (P + 3) / 4 < bwd_record_floats(P); }

__global__ void __launch_bounds__(256) pack_bwd_kernel(int64_t n, int levels, int K, const float* xy,
                                                       const float* axes, const float* conic_o, const float* extent,
                                                       const uint8_t* idx, const float* w, float* recs)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int P = levels * K;
    float* rec = recs + (size_t)g * bwd_record_floats(P);
    const float4 cn = reinterpret_cast<const float4*>(conic_o)[g];
    const float4 ax1 = reinterpret_cast<const float4*>(axes)[2 * g + 1];
    reinterpret_cast<float4*>(rec)[0] = reinterpret_cast<const float4*>(xy)[g];
    reinterpret_cast<float4*>(rec)[1] = reinterpret_cast<const float4*>(axes)[2 * g];
    reinterpret_cast<float4*>(rec)[2] = make_float4(ax1.x, ax1.y, ax1.z, cn.w);
    const float2 ex = reinterpret_cast<const float2*>(extent)[g];
    reinterpret_cast<float4*>(rec)[3] = make_float4(cn.x, cn.y, cn.z, ex.x);
    rec[bwd_record_floats(P) - 1] = ex.y;
    uint8_t* cb = reinterpret_cast<uint8_t*>(rec + 16 + P);
    for (int p = 0; p < P; ++p) {
        const int lev = p / K;
        const size_t src = (size_t)g * P + p;
        const int ix = idx[src];
        const bool ok = ix < 64;
        rec[16 + p] = ok ? w[src] : 0.0f;
        cb[p] = (uint8_t)(lev * 64 + (ok ? ix : 0));
    }
}

// lane L ends with the warp-wide sum of v[L]
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = upper ? v[i] : v[i + o];
            const float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// 16-byte asynchronous copy global -> shared (cp.async, L2 only), its group commit and wait
__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int LEVELS, int K, int TW, int TH>
struct BwdCfg {
    static constexpr int kWarps = TW * TH / 32;
    static constexpr int kPairs = LEVELS * K;
    static constexpr int kCols = LEVELS * 64;
    static constexpr int kGFloats = (kCols * 33 + 3) / 4 * 4;
    static constexpr int kRecFloats = bwd_record_floats(kPairs);
    static constexpr int kSmemRecFloats = kRecFloats - 4;  // staged without the 2D mean
    static constexpr int kSmemBytes = kWarps * (kGFloats + 32 * kSmemRecFloats) * 4;
    // lane -> pixel as in the forward splat: each warp covers an 8 x 4 block, warps row-major
    static constexpr int kWarpW = 8, kWarpH = 4, kWarpsX = TW / kWarpW;
    __host__ __device__ static constexpr int lane_x(int warp, int lane) { return (warp % kWarpsX) * kWarpW + lane % kWarpW; }
    __host__ __device__ static constexpr int lane_y(int warp, int lane) { return (warp / kWarpsX) * kWarpH + lane / kWarpW; }
    static_assert(kPairs + 6 <= 32, "quantities per Gaussian");
    static constexpr int kQ = kPairs + 6;              // gradient quantities per Gaussian and pixel
    // Gaussians evaluated per step: as many as their quantities fit the 32 lanes of one reduce-scatter
    static constexpr int kPer = 32 / kQ > 4 ? 4 : 32 / kQ;
    static_assert(bwd_record_last_free(kPairs), "the record's last float holds the culling half-height");
    static_assert(TW % 8 == 0 && TH % 4 == 0 && (TW * TH) % 32 == 0, "warps cover 8 x 4 blocks of a tile");
};

// The adjoint of one warp's 8 x 4 pixel block `warp` of bin tile `tile`: its pixels' dLoss/dW
// staged as columns gW[col][lane] in shared memory, or (TM) in this warp's 64 TMEM columns at tcol;
// then the tile's list back to front.  stage: 32 staged records (without TM); rbuf: TM's
// double-buffered records.
template <int LEVELS, int K, int TW, int TH, bool TM>
__device__ __forceinline__ void bwd_warp_block(const SplatBwdArgs& a, int tile, int warp, int lane, float* gW,
                                               uint32_t tcol, float* stage, float* rbuf)
{
    using C = BwdCfg<LEVELS, K, TW, TH>;
    const int GX = (a.cam.width + TW - 1) / TW;
    const int tx = tile % GX, ty = tile / GX;
    const int px = tx * TW + C::lane_x(warp, lane), py = ty * TH + C::lane_y(warp, lane);
    const bool inside = px < a.cam.width && py < a.cam.height;
    const size_t P = (size_t)a.cam.width * a.cam.height;
    const size_t pix = (size_t)py * a.cam.width + px;
    const float wx0 = (float)(tx * TW + C::lane_x(warp, 0)), wx1 = wx0 + (float)(C::kWarpW - 1);
    const float wy0 = (float)(ty * TH + C::lane_y(warp, 0)), wy1 = wy0 + (float)(C::kWarpH - 1);

    if constexpr (TM) {
        // each lane's pixel row of dLoss/dW (64 floats) into its TMEM lane (the previous block's
        // TMEM loads completed at their waits)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t v[32];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (inside) x = __ldg(reinterpret_cast<const float4*>(a.dcoeff + pix * 64 + 32 * h) + i);
                v[4 * i] = __float_as_uint(x.x);
                v[4 * i + 1] = __float_as_uint(x.y);
                v[4 * i + 2] = __float_as_uint(x.z);
                v[4 * i + 3] = __float_as_uint(x.w);
            }
            tc::tmem_st32(tcol + 32u * h, v);
        }
        tc::tmem_wait_st();
    }
    // stage dLoss/dW of this warp's pixels as columns gW[col][lane]
    for (int lev = 0; lev < (TM ? 0 : LEVELS); ++lev)
        for (int q = lane; q < 32 * 16; q += 32) {
            const int pl = q >> 4, c4 = (q & 15) * 4;
            const int gx = tx * TW + C::lane_x(warp, pl), gy = ty * TH + C::lane_y(warp, pl);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gx < a.cam.width && gy < a.cam.height)
                v = __ldg(reinterpret_cast<const float4*>(a.dcoeff + ((size_t)lev * P + (size_t)gy * a.cam.width + gx) * 64 + c4));
            float* col = gW + (lev * 64 + c4) * 33 + pl;
            col[0] = v.x;
            col[33] = v.y;
            col[66] = v.z;
            col[99] = v.w;
        }
    __syncwarp();

    const uint32_t beg = a.tile_ranges[2 * tile];
    const uint32_t my_last = inside ? a.n_last[pix] : 0u;
    float T = inside ? a.final_T[pix] : 1.0f;
    float Bsum = 0.0f;
    uint32_t wmax = my_last;
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    const float pxf = (float)px, pyf = (float)py;

    // The list back to front in batches of 32 positions [top - 32, top): lane i <-> position
    // top - 32 + i (negative positions are empty).  Each lane's record (2D mean, culling extent
    // and the rest) is loaded one batch ahead and its list entry two batches ahead, so the loads
    // are in flight while the current batch is evaluated; kept records are staged in shared
    // memory, the 2D mean and the id stay in the staging lane's registers.
    constexpr int kR = C::kRecFloats / 4;
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    // (every load is inside its condition: no address outside the list or the records is formed)
    auto load_id = [&](int t) -> uint32_t {
        const int pos = t - 32 + lane;
        uint32_t id = kNone;
        if (t > 0 && pos >= 0) id = __ldg(a.gauss_ids + beg + pos);
        return id;
    };
    auto load_rec = [&](uint32_t id, float4 (&r)[kR]) {
        if (id != kNone) {
            const float4* src = reinterpret_cast<const float4*>(a.recs + (size_t)id * C::kRecFloats);
#pragma unroll
            for (int v = 0; v < kR; ++v) r[v] = __ldg(src + v);
        } else {
#pragma unroll
            for (int v = 0; v < kR; ++v) r[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto fetch = [&](uint32_t id, int slot) {   // TM: this lane's record into rbuf[slot] (one copy group)
        if (id != kNone) {
            const float* src = a.recs + (size_t)id * C::kRecFloats;
            float* dst = rbuf + (slot * 32 + lane) * C::kRecFloats;
#pragma unroll
            for (int v = 0; v < kR; ++v) cp_async16(dst + 4 * v, src + 4 * v);
        }
        cp_async_commit();
    };
    int top = (int)wmax;
    uint32_t my_g = load_id(top), id_nxt = load_id(top - 32);
    float4 rc[TM ? 1 : kR];
    if constexpr (TM) fetch(my_g, 0);
    else load_rec(my_g, rc);
    int slot = 0;
    for (; top > 0; top -= 32) {
        float4 rn[TM ? 1 : kR];
        if constexpr (TM) {
            fetch(id_nxt, slot ^ 1);
            cp_async_wait<1>();   // this lane's copies of the current batch have landed
            __syncwarp();         // ... and every lane's, for the reads of other lanes' records below
        } else {
            load_rec(id_nxt, rn);
        }
        const uint32_t id_nn = load_id(top - 64);
        const int lo = top - 32;
        const float* myrec = TM ? rbuf + (slot * 32 + lane) * C::kRecFloats : nullptr;
        const float4 my_xy = TM ? *reinterpret_cast<const float4*>(myrec) : rc[0];
        const float exx = TM ? myrec[15] : rc[3].w, exy = TM ? myrec[C::kRecFloats - 1] : rc[kR - 1].w;
        const bool keep = my_g != kNone && exx >= 0.0f && my_xy.x + exx >= wx0 && my_xy.x - exx <= wx1 &&
                          my_xy.y + exy >= wy0 && my_xy.y - exy <= wy1;
        if (!TM && keep) {
            float4* dst = reinterpret_cast<float4*>(stage + lane * C::kSmemRecFloats);
#pragma unroll
            for (int v = 1; v < kR; ++v) dst[v - 1] = rc[v];
        }
        uint32_t mask = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        // kPer Gaussians per step (as many as kPer kQ <= 32 allows), back to front: the first is the one further
        // back in the list.  Their evaluations are independent; the transmittance and the running
        // sum pass from one to the next; one reduce-scatter of all their quantities serves both.
        constexpr int kPer = C::kPer;
        while (mask) {
            int idx[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                idx[u] = mask ? 31 - __clz(mask) : -1;   // (warp-uniform)
                if (mask) mask &= ~(1u << idx[u]);
            }
            uint32_t gid[kPer];
            float p2[kPer], dx[kPer], dy[kPer];
            float4 axl[kPer], g2[kPer];
            const float* rr[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int i = idx[u] < 0 ? idx[0] : idx[u];   // an absent second Gaussian re-reads the first (unused)
                gid[u] = __shfl_sync(0xffffffffu, my_g, i);
                float4 g0;
                if constexpr (TM) {
                    const float* ri = rbuf + (slot * 32 + i) * C::kRecFloats;
                    g0 = *reinterpret_cast<const float4*>(ri);
                    rr[u] = ri + 4;
                } else {
                    g0.x = __shfl_sync(0xffffffffu, my_xy.x, i);
                    g0.y = __shfl_sync(0xffffffffu, my_xy.y, i);
                    g0.z = __shfl_sync(0xffffffffu, my_xy.z, i);
                    g0.w = __shfl_sync(0xffffffffu, my_xy.w, i);
                    rr[u] = stage + i * C::kSmemRecFloats;
                }
                const float4 ax = *reinterpret_cast<const float4*>(rr[u]);
                axl[u] = *reinterpret_cast<const float4*>(rr[u] + 4);
                g2[u] = *reinterpret_cast<const float4*>(rr[u] + 8);
                dx[u] = __fadd_rn(__fsub_rn(g0.x, pxf), g0.z);
                dy[u] = __fadd_rn(__fsub_rn(g0.y, pyf), g0.w);
                p2[u] = eval_power2(g0, ax, axl[u], pxf, pyf);
            }
            // TM: the dLoss/dW columns of every pair of the step's Gaussians (warp-uniform columns,
            // loaded by all lanes together before the per-lane conditions)
            uint32_t gwt[TM ? kPer : 1][TM ? C::kPairs : 1];
            if constexpr (TM) {
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    const uint8_t* cr = reinterpret_cast<const uint8_t*>(rr[u] + 12 + C::kPairs);
#pragma unroll
                    for (int p = 0; p < C::kPairs; ++p) tc::tmem_ld1(tcol + (uint32_t)cr[p], gwt[u][p]);
                }
                tc::tmem_wait_ld();
            }
            float vals[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) vals[k] = 0.0f;
            bool contrib = false;
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                if (idx[u] >= 0 && lo + idx[u] < (int)my_last && p2[u] <= 0.0f) {
                    float ex2;
                    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex2) : "f"(p2[u]));
                    const float raw = axl[u].w * ex2;
                    const float alpha = fminf(kAlphaMax, raw);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        float oma = 1.0f - alpha;   // exact to within alpha's own error up to alpha = 1/2
                        if (alpha > 0.5f) oma = one_minus_alpha(alpha, axl[u].w, p2[u]);
                        const float Ti = __fdividef(T, oma);   // within 2 ulp: far below the gradients' error bound
                        const float e = alpha * Ti;
                        const float* wr = rr[u] + 12;
                        const uint8_t* cr = reinterpret_cast<const uint8_t*>(rr[u] + 12 + C::kPairs);
                        float gsum = 0.0f;
#pragma unroll
                        for (int p = 0; p < C::kPairs; ++p) {
                            float gw;
                            if constexpr (TM) gw = __uint_as_float(gwt[u][p]);
                            else gw = gW[(int)cr[p] * 33 + lane];
                            vals[u * C::kQ + p] = gw * e;
                            gsum = fmaf(gw, wr[p], gsum);
                        }
                        const float dalpha = Ti * (gsum - Bsum);
                        Bsum = fmaf(alpha, gsum, oma * Bsum);
                        T = Ti;
                        if (!(raw > kAlphaMax)) {
                            const float dpow = dalpha * alpha;
                            const float ca = g2[u].x, cb = g2[u].y, cc = g2[u].z, x = dx[u], y = dy[u];
                            float* v = vals + u * C::kQ + C::kPairs;
                            v[0] = dpow * -(ca * x + cb * y);   // d/du
                            v[1] = dpow * -(cb * x + cc * y);   // d/dv
                            v[2] = dpow * (-0.5f * x * x);      // d/da
                            v[3] = dpow * (-x * y);             // d/db
                            v[4] = dpow * (-0.5f * y * y);      // d/dc
                            v[5] = dalpha * ex2;                // d/dopacity
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                // lane L holds quantity L % kQ of Gaussian L / kQ of the step
                const float tot = reduce_scatter32(vals, lane);
                const int u = lane / C::kQ, q = lane - u * C::kQ;
                bool here = false;
                uint32_t g = 0;
#pragma unroll
                for (int v = 0; v < kPer; ++v)
                    if (u == v) {
                        here = idx[v] >= 0;
                        g = gid[v];
                    }
                if (here) {
                    if (q < C::kPairs) {
                        atomicAdd(a.dw + (size_t)g * C::kPairs + q, tot);
                    } else if (q < C::kPairs + 5) {
                        atomicAdd(a.grad2d + (size_t)g * 8 + (q - C::kPairs), tot);
                    } else {
                        atomicAdd(a.dopacity + g, tot);
                    }
                }
            }
        }
        __syncwarp();
        if constexpr (TM) {
            slot ^= 1;
        } else {
#pragma unroll
            for (int v = 0; v < kR; ++v) rc[v] = rn[v];
        }
        my_g = id_nxt;
        id_nxt = id_nn;
    }
    if constexpr (TM) {
        cp_async_wait<0>();   // the last prefetch has landed before rbuf is reused
        __syncwarp();
    }
}

template <int LEVELS, int K, int TW, int TH>
__global__ void __launch_bounds__(TW* TH) splat_backward_kernel(SplatBwdArgs a)
{
    using C = BwdCfg<LEVELS, K, TW, TH>;
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bwd_warp_block<LEVELS, K, TW, TH, false>(a, blockIdx.x, warp, lane, smem + warp * C::kGFloats, 0u,
                                             smem + C::kWarps * C::kGFloats + warp * 32 * C::kSmemRecFloats, nullptr);
}

// One level, 16 x 16 tiles: dLoss/dW of each warp's 32 pixels in tensor memory (8 warps, two per TMEM
// lane quarter, 64 columns each, 128 per CTA) and each lane's records double-buffered in shared
// memory by asynchronous copies, so three CTAs (24 warps) share an SM (registers), where the
// shared-memory columns allowed two.  Persistent: every warp takes (tile, 8 x 4 block) work items
// from a queue on its own, so a warp that finishes early starts the next block instead of waiting
// for the slowest warp of its tile.
template <int K>
__global__ void __launch_bounds__(256, 3) splat_backward_tm_kernel(SplatBwdArgs a, uint32_t items)
{
    using C = BwdCfg<1, K, 16, 16>;
    constexpr uint32_t kTmCols = 128;
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tslot), kTmCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tcol = tslot + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(64 * (warp >> 2));
    float* rbuf = smem + warp * 2 * 32 * C::kRecFloats;
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(a.queue, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= items) break;
        bwd_warp_block<1, K, 16, 16, true>(a, (int)(item / C::kWarps), (int)(item % C::kWarps), lane, nullptr, tcol,
                                           nullptr, rbuf);
    }
    // every warp's TMEM loads completed at their waits
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tslot, kTmCols);
    }
}

template <int LEVELS, int K, int TW, int TH>
cudaError_t launch_bwd_t(const SplatBwdArgs& a, cudaStream_t stream)
{
    using C = BwdCfg<LEVELS, K, TW, TH>;
    static_assert(C::kSmemBytes <= 232448, "shared memory budget");
    auto kern = splat_backward_kernel<LEVELS, K, TW, TH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    const int GX = (a.cam.width + TW - 1) / TW, GY = (a.cam.height + TH - 1) / TH;
    if (GX * GY == 0) return cudaSuccess;
    kern<<<GX * GY, TW * TH, C::kSmemBytes, stream>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_bwd_tm(const SplatBwdArgs& a, cudaStream_t stream)
{
    using C = BwdCfg<1, K, 16, 16>;
    // the double-buffered records, padded so that at most four CTAs (4 x 128 TMEM columns) could
    // share an SM: a CTA's TMEM allocation never waits
    constexpr int kRecBytes = C::kWarps * 2 * 32 * C::kRecFloats * 4;
    constexpr int kSmem = kRecBytes > 49152 ? kRecBytes : 49152;
    static_assert(5 * (kSmem + 1024 + 16) > 233472, "at most four CTAs per SM");
    auto kern = splat_backward_tm_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    const int GX = (a.cam.width + 15) / 16, GY = (a.cam.height + 15) / 16;
    const uint32_t items = (uint32_t)(GX * GY) * C::kWarps;
    if (items == 0) return cudaSuccess;
    e = cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    int grid = 3 * (a.num_sms > 0 ? a.num_sms : 1);
    if ((uint32_t)grid * C::kWarps > items) grid = (int)((items + C::kWarps - 1) / C::kWarps);
    kern<<<grid, 256, kSmem, stream>>>(a, items);
    return cudaGetLastError();
}

template <int LEVELS, int K>
cudaError_t launch_bwd_tile(const SplatBwdArgs& a, cudaStream_t stream)
{
    if (a.cam.tile_w == 16 && a.cam.tile_h == 16) {
        if constexpr (LEVELS == 1) return launch_bwd_tm<K>(a, stream);
        return launch_bwd_t<LEVELS, K, 16, 16>(a, stream);
    }
    if (a.cam.tile_w == 8 && a.cam.tile_h == 8) return launch_bwd_t<LEVELS, K, 8, 8>(a, stream);
    if (a.cam.tile_w == 32 && a.cam.tile_h == 8) return launch_bwd_t<LEVELS, K, 32, 8>(a, stream);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------ 3
__global__ void __launch_bounds__(256) project_backward_kernel(ProjBwdArgs a)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= a.n || !(a.flags[gi] & 1)) return;
    const lsv2_camera& c = a.cam;
    const float* gr = a.grad2d + (size_t)gi * 8;
    const float du = gr[0], dv = gr[1], dA = gr[2], dB = gr[3], dC = gr[4];
    const float m[3] = {a.means[3 * gi], a.means[3 * gi + 1], a.means[3 * gi + 2]};
    const float s[3] = {a.scales[3 * gi], a.scales[3 * gi + 1], a.scales[3 * gi + 2]};
    const float4 q4 = reinterpret_cast<const float4*>(a.quats)[gi];
    // forward quantities (float32)
    float t[3];
    for (int i = 0; i < 3; ++i) t[i] = c.R[3 * i] * m[0] + c.R[3 * i + 1] * m[1] + c.R[3 * i + 2] * m[2] + c.t[i];
    const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x / qn, x = q4.y / qn, y = q4.z / qn, z = q4.w / qn;
    float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                  2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                  2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float M[9];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) M[3 * k + j] = R[3 * k + j] * s[j];
    const float limx = kGuard * ((float)c.width / (2.0f * c.fx)), limy = kGuard * ((float)c.height / (2.0f * c.fy));
    const float tz = t[2], itz = 1.0f / tz;
    const float txz = t[0] * itz, tyz = t[1] * itz;
    const bool clx = txz > limx || txz < -limx, cly = tyz > limy || tyz < -limy;
    const float cxz = fminf(limx, fmaxf(-limx, txz)), cyz = fminf(limy, fmaxf(-limy, tyz));
    const float J00 = c.fx * itz, J11 = c.fy * itz, J02 = -c.fx * cxz * itz, J12 = -c.fy * cyz * itz;
    float T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * c.R[j] + J02 * c.R[6 + j];
        T[3 + j] = J11 * c.R[3 + j] + J12 * c.R[6 + j];
    }
    float N[6];
    for (int r = 0; r < 2; ++r)
        for (int j = 0; j < 3; ++j) N[3 * r + j] = T[3 * r] * M[j] + T[3 * r + 1] * M[3 + j] + T[3 * r + 2] * M[6 + j];
    const float c00 = N[0] * N[0] + N[1] * N[1] + N[2] * N[2] + kDilation;
    const float c11 = N[3] * N[3] + N[4] * N[4] + N[5] * N[5] + kDilation;
    const float c01 = N[0] * N[3] + N[1] * N[4] + N[2] * N[5];
    const float idet = 1.0f / (c00 * c11 - c01 * c01);
    const float qa = c11 * idet, qb = -c01 * idet, qc = c00 * idet;  // conic
    // dL/dSigma' = -Q Ghat Q, Ghat = [[dA, dB/2], [dB/2, dC]]
    const float g01 = 0.5f * dB;
    const float X00 = dA * qa + g01 * qb, X01 = dA * qb + g01 * qc;   // Ghat Q
    const float X10 = g01 * qa + dC * qb, X11 = g01 * qb + dC * qc;
    const float H00 = -(qa * X00 + qb * X10), H01 = -(qa * X01 + qb * X11), H11 = -(qb * X01 + qc * X11);
    // Sigma' = N N^T + d I  ->  dN = 2 H N
    float dN[6];
    for (int j = 0; j < 3; ++j) {
        dN[j] = 2.0f * (H00 * N[j] + H01 * N[3 + j]);
        dN[3 + j] = 2.0f * (H01 * N[j] + H11 * N[3 + j]);
    }
    // N = T M
    float dT[6], dM[9];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) dT[3 * r + k] = dN[3 * r] * M[3 * k] + dN[3 * r + 1] * M[3 * k + 1] + dN[3 * r + 2] * M[3 * k + 2];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) dM[3 * k + j] = T[k] * dN[j] + T[3 + k] * dN[3 + j];
    float ds[3], dR[9];
    for (int j = 0; j < 3; ++j) ds[j] = dM[j] * R[j] + dM[3 + j] * R[3 + j] + dM[6 + j] * R[6 + j];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) dR[3 * k + j] = dM[3 * k + j] * s[j];
    // rotation matrix of the unit quaternion (w, x, y, z)
    float dw_ = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    float dx_ = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2.f * x * dR[8]);
    float dy_ = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
    float dz_ = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
    const float dot = w * dw_ + x * dx_ + y * dy_ + z * dz_;
    const float iq = 1.0f / qn;
    // T = J W:  dJ
    const float dJ00 = dT[0] * c.R[0] + dT[1] * c.R[1] + dT[2] * c.R[2];
    const float dJ02 = dT[0] * c.R[6] + dT[1] * c.R[7] + dT[2] * c.R[8];
    const float dJ11 = dT[3] * c.R[3] + dT[4] * c.R[4] + dT[5] * c.R[5];
    const float dJ12 = dT[3] * c.R[6] + dT[4] * c.R[7] + dT[5] * c.R[8];
    float dt[3] = {0.f, 0.f, 0.f};
    const float itz2 = itz * itz;
    dt[2] += -c.fx * itz2 * dJ00 - c.fy * itz2 * dJ11;
    if (!clx) {
        dt[0] += -c.fx * itz2 * dJ02;
        dt[2] += 2.0f * c.fx * t[0] * itz2 * itz * dJ02;
    } else {
        dt[2] += c.fx * cxz * itz2 * dJ02;
    }
    if (!cly) {
        dt[1] += -c.fy * itz2 * dJ12;
        dt[2] += 2.0f * c.fy * t[1] * itz2 * itz * dJ12;
    } else {
        dt[2] += c.fy * cyz * itz2 * dJ12;
    }
    // u = fx tx / tz + cx
    dt[0] += du * c.fx * itz;
    dt[1] += dv * c.fy * itz;
    dt[2] += -(du * c.fx * t[0] + dv * c.fy * t[1]) * itz2;
    for (int j = 0; j < 3; ++j)
        a.dmeans[3 * gi + j] += c.R[j] * dt[0] + c.R[3 + j] * dt[1] + c.R[6 + j] * dt[2];
    for (int j = 0; j < 3; ++j) a.dscales[3 * gi + j] += ds[j];
    a.dquats[4 * gi + 0] += (dw_ - w * dot) * iq;
    a.dquats[4 * gi + 1] += (dx_ - x * dot) * iq;
    a.dquats[4 * gi + 2] += (dy_ - y * dot) * iq;
    a.dquats[4 * gi + 3] += (dz_ - z * dot) * iq;
}

}  // namespace

size_t splat_backward_workspace_bytes(int64_t n, int levels, int K)
{
    const size_t g2 = ((size_t)n * 8 * 4 + 255) / 256 * 256;
    const size_t recs = ((size_t)n * bwd_record_floats(levels * K) * 4 + 255) / 256 * 256;
    return g2 + recs + 256;   // + the work queue of the persistent kernel
}

cudaError_t launch_splat_backward(int levels, int K, const SplatBwdArgs& args, const ProjBwdArgs& pargs,
                                  const uint8_t* idx, const float* w, cudaStream_t stream)
{
    SplatBwdArgs a = args;
    const size_t g2 = ((size_t)pargs.n * 8 * 4 + 255) / 256 * 256;
    a.grad2d = static_cast<float*>(a.workspace);
    a.recs = reinterpret_cast<float*>(static_cast<char*>(a.workspace) + g2);
    a.queue = reinterpret_cast<uint32_t*>(static_cast<char*>(a.workspace) + g2 +
                                          ((size_t)pargs.n * bwd_record_floats(levels * K) * 4 + 255) / 256 * 256);
    cudaError_t e = cudaMemsetAsync(a.grad2d, 0, (size_t)pargs.n * 8 * 4, stream);
    if (e != cudaSuccess) return e;
    if (pargs.n > 0)
        pack_bwd_kernel<<<(unsigned)((pargs.n + 255) / 256), 256, 0, stream>>>(pargs.n, levels, K, a.xy, a.axes,
                                                                              a.conic_o, a.extent, idx, w, a.recs);
    if (levels == 1 && K == 4) e = launch_bwd_tile<1, 4>(a, stream);
    else if (levels == 1 && K == 2) e = launch_bwd_tile<1, 2>(a, stream);
    else if (levels == 1 && K == 8) e = launch_bwd_tile<1, 8>(a, stream);
    else if (levels == 2 && K == 4) e = launch_bwd_tile<2, 4>(a, stream);
    else if (levels == 3 && K == 4) e = launch_bwd_tile<3, 4>(a, stream);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    ProjBwdArgs pa = pargs;
    pa.grad2d = a.grad2d;
    if (pa.n > 0) project_backward_kernel<<<(unsigned)((pa.n + 255) / 256), 256, 0, stream>>>(pa);
    return cudaGetLastError();
}

bool splat_backward_supported(int levels, int K)
{
    return (levels == 1 && (K == 2 || K == 4 || K == 8)) || ((levels == 2 || levels == 3) && K == 4);
}

}  // namespace lsv2
