// splat_core.cuh -- the sparse-coefficient splat of one tile (Sec. 3.4, Algorithm 1; Eq. 3 and
// Eq. 7 weights), shared by the splat kernels and the fused render kernel.  See splat.cu for the
// design (producer warp + shared-memory ring of records, consumer warps with accumulator columns
// in shared memory or TMEM).
#pragma once

#include "device.cuh"
#include "splat.cuh"
#include "tc.cuh"

namespace lsv2 {
namespace {

// One tile of one view.
struct TileJob {
    int width, height, x0, y0;   // image size; first pixel of this CTA's TW x TH block
    uint32_t beg, end;
    const uint32_t* gauss_ids;
    const float* recs;
    float* coeff;                // F32 coefficient map, or BF16 when coeff_bf16
    float* final_T;
    uint32_t* n_last;
    int32_t* status;
    int coeff_bf16 = 0;
    uint64_t wait_ns = kDefaultWaitNs;   // bound of every wait on a stage barrier
};

// Shared memory of one CTA: accumulators [kWarps][kAccFloats], stage barriers and flags, then
// kStages stages of [kBatch records][kBatch culling boxes (u, v, ex, ey)].  The barriers are
// initialised once per CTA; batches are numbered across the CTA's tiles (stage = batch %
// kStages, phase parity = (batch / kStages) & 1), so a persistent CTA never re-initialises them.
template <class C>
struct SplatSmem {
    float* acc;
    uint64_t* full;    // a stage's batch has landed (32 producer arrivals + the copies' bytes)
    uint64_t* empty;   // every consumer warp is done with the stage (kWarps arrivals)
    int* done_warps;   // consumer warps of the current tile whose pixels have all terminated
    int* abort;        // a wait of this CTA ran out: every later wait gives up at once
    uint32_t* issued;  // batches the producer issued for the current tile
    int* skip;         // a wait ran out somewhere (status word): skip the remaining tiles
    uint32_t* tmem_slot;   // TMEM base address of the CTA's allocation (TMEM accumulators)
    unsigned char* stages;
    __device__ explicit SplatSmem(unsigned char* base)
        : acc(reinterpret_cast<float*>(base)),
          full(reinterpret_cast<uint64_t*>(base + C::kAccBytes)),
          empty(reinterpret_cast<uint64_t*>(base + C::kAccBytes) + 8),
          done_warps(reinterpret_cast<int*>(base + C::kAccBytes + 128)),
          abort(reinterpret_cast<int*>(base + C::kAccBytes + 132)),
          issued(reinterpret_cast<uint32_t*>(base + C::kAccBytes + 136)),
          skip(reinterpret_cast<int*>(base + C::kAccBytes + 140)),
          tmem_slot(reinterpret_cast<uint32_t*>(base + C::kAccBytes + 144)),
          stages(base + C::kFixedBytes)
    {
    }
    __device__ const unsigned char* rec(int s) const { return stages + s * C::kStageBytes; }
    __device__ float4* box(int s) const
    {
        return reinterpret_cast<float4*>(stages + s * C::kStageBytes + C::kBatch * C::kRecBytes);
    }
    // once per CTA, by one thread, before a __syncthreads
    __device__ void init() const
    {
        for (int s = 0; s < C::kStages; ++s) {
            tc::mbar_init(tc::smem_u32(full + s), 32);
            tc::mbar_init(tc::smem_u32(empty + s), C::kWarps);
        }
        *done_warps = 0;
        *abort = 0;
        *skip = 0;
    }
};

constexpr int kWaitDone = 1, kWaitStopped = 0, kWaitTimeout = -1, kWaitAborted = -2;

// A pair's accumulator reference: the record's shared-memory byte offset (col * 132), or with
// TMEM accumulators the column col = (offset / 4) / 33, as (x * 1986) >> 16, exact for x = 33 col
// with col < 32768.
template <bool kTM>
__device__ __forceinline__ uint32_t acc_ref(uint32_t off)
{
    return kTM ? ((off >> 2) * 1986u) >> 16 : off;
}

// Warp-uniform bounded wait for a barrier phase.  `done_warps` (optional) ends the wait early
// once all_done consumer warps have finished; a wait that is still unfinished `limit_ns` after
// it began raises the CTA's abort flag (and the caller reports LSV2_ERR_TIMEOUT), after which
// every other wait returns at once.  The first check is a non-blocking test (a try_wait may
// suspend the warp until the phase completes), so with limit 0 the wait gives up unless the
// phase is complete when it starts.
__device__ __forceinline__ int warp_wait(uint64_t* bar, uint32_t parity, const volatile int* done_warps,
                                         int all_done, volatile int* abort, uint64_t limit_ns)
{
    const uint64_t t0 = tc::globaltimer();
    for (bool first = true;; first = false) {
        const bool ready = first ? tc::mbar_test(tc::smem_u32(bar), parity) : tc::mbar_try(tc::smem_u32(bar), parity);
        if (__all_sync(0xffffffffu, ready)) return kWaitDone;
        if (__shfl_sync(0xffffffffu, *abort, 0)) return kWaitAborted;
        if (done_warps && __shfl_sync(0xffffffffu, *done_warps, 0) >= all_done) return kWaitStopped;
        if (__any_sync(0xffffffffu, tc::globaltimer() - t0 >= limit_ns)) {
            *abort = 1;
            return kWaitTimeout;
        }
    }
}

// Warp-uniform wait for a phase that this warp's own copies complete (they always land): used
// to drain a CTA that is giving up, so it ignores the abort flag; bounded by kDrainNs.
__device__ __forceinline__ bool warp_drain(uint64_t* bar, uint32_t parity)
{
    const uint64_t t0 = tc::globaltimer();
    while (!__all_sync(0xffffffffu, tc::mbar_try(tc::smem_u32(bar), parity)))
        if (__any_sync(0xffffffffu, tc::globaltimer() - t0 > kDrainNs)) return false;
    return true;
}

// Producer warp: the tile's batch b is CTA batch g = bbase + b and goes to stage g % kStages
// once every consumer warp has released the stage's previous batch; each lane copies one
// record (bulk async copy, completing on the stage's barrier) and writes its culling box.
// Before returning it waits until every copy it issued has landed (also after a wait of the CTA
// ran out), so no copy is in flight into shared memory that is reused or released, and
// publishes the number of batches it issued.
template <class C>
__device__ void splat_produce(const TileJob& a, const SplatSmem<C>& sm, int lane, uint32_t bbase)
{
    const uint32_t n = a.end - a.beg;
    const uint32_t nb = (n + C::kBatch - 1) / C::kBatch;
    const volatile int* done_warps = sm.done_warps;
    uint32_t issued = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        const uint32_t g = bbase + b;
        const int s = (int)(g % C::kStages);
        if (g >= (uint32_t)C::kStages) {
            const int w =
                warp_wait(sm.empty + s, ((g / C::kStages) - 1u) & 1u, done_warps, C::kWarps, sm.abort, a.wait_ns);
            if (w == kWaitTimeout && lane == 0) report(a.status, LSV2_ERR_TIMEOUT);
            if (w != kWaitDone) break;
        }
        if (__shfl_sync(0xffffffffu, *done_warps, 0) >= C::kWarps) break;
        const uint32_t cnt = min((uint32_t)C::kBatch, n - b * C::kBatch);
        const uint32_t full = tc::smem_u32(sm.full + s);
        if (lane == 0) tc::mbar_expect_tx(full, cnt * (uint32_t)C::kRecBytes);
        __syncwarp();
        float4 box = make_float4(0.0f, 0.0f, -1.0f, -1.0f);
        if ((uint32_t)lane < cnt) {
            const uint32_t id = a.gauss_ids[a.beg + b * C::kBatch + lane];
            const float* src = a.recs + (size_t)id * C::kRecFloats;
            tc::bulk_load(tc::smem_u32(sm.rec(s) + lane * C::kRecBytes), src, (uint32_t)C::kRecBytes, full);
            const float2 xy = __ldg(reinterpret_cast<const float2*>(src));
            const float2 ex = __ldg(reinterpret_cast<const float2*>(src + C::kRecFloats - 4));
            box = make_float4(xy.x, xy.y, ex.x, ex.y);
        }
        if (lane < C::kBatch) sm.box(s)[lane] = box;
        tc::mbar_arrive(full);
        issued = b + 1;
    }
    // the last kStages batches' copies (each stage's earlier batches completed before its reuse)
    const uint32_t first = issued > (uint32_t)C::kStages ? issued - C::kStages : 0u;
    for (uint32_t b = first; b < issued; ++b) {
        const uint32_t g = bbase + b;
        if (!warp_drain(sm.full + (int)(g % C::kStages), (g / C::kStages) & 1u)) {
            if (lane == 0) report(a.status, LSV2_ERR_TIMEOUT);
            *sm.abort = 1;
        }
    }
    if (lane == 0) *sm.issued = issued;
}

// Consumer warp: 32 pixels (one per lane), front to back over the tile's batches.
// kWriteCoeff: write the warp's coefficients to a.coeff at the end (false: they stay in the
// warp's shared-memory columns for a fused consumer).  kTM: the accumulators are TMEM columns
// of this warp's lane quarter (lane = pixel, column = accumulator column) instead of
// shared-memory columns; the arithmetic and its order are the same.
template <class C, int LEVELS, int K, int TW, int TH, bool kWriteCoeff = true, bool kTM = false>
__device__ uint32_t splat_consume(const TileJob& a, const SplatSmem<C>& sm, int warp, int lane, uint32_t bbase)
{
    constexpr int kB = C::kBatch;
    constexpr int kChunk = 4;   // kept records evaluated together
    static_assert(!kTM || (C::kLW % 32 == 0 && !C::kDense && C::kPairs % 6 == 0 && kWriteCoeff), "TMEM accumulators");
    float* acc = sm.acc + (kTM ? 0 : warp) * C::kAccFloats;
    unsigned char* acc_lane = reinterpret_cast<unsigned char*>(acc + lane);
    const uint32_t tbase = kTM ? *sm.tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) : 0u;

    const int px = a.x0 + C::lane_x(warp, lane), py = a.y0 + C::lane_y(warp, lane);
    const bool inside = px < a.width && py < a.height;
    // pixel block covered by this warp
    const float wx0 = (float)(a.x0 + C::lane_x(warp, 0)), wx1 = wx0 + (float)(C::kWarpW - 1);
    const float wy0 = (float)(a.y0 + C::lane_y(warp, 0)), wy1 = wy0 + (float)(C::kWarpH - 1);

    if constexpr (kTM) {
        uint32_t zero[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) zero[i] = 0u;
#pragma unroll
        for (int c = 0; c < C::kCols + 1; c += 32) tc::tmem_st32(tbase + (uint32_t)c, zero);
        tc::tmem_wait_st();
    } else {
        for (int i = lane * 4; i < C::kAccFloats; i += 128)
            *reinterpret_cast<float4*>(acc + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();

    const uint32_t n = a.end - a.beg;
    const uint32_t nb = (n + kB - 1) / kB;
    float T = 1.0f;
    uint32_t last = 0;
    bool done = !inside, wdone = false;
    const float pxf = (float)px, pyf = (float)py;
    const volatile int* done_warps = sm.done_warps;

    uint32_t consumed = 0;   // batches this warp has released
    for (uint32_t b = 0; b < nb; ++b) {
        const uint32_t g = bbase + b;
        const int s = (int)(g % C::kStages);
        if (!wdone && __all_sync(0xffffffffu, done)) {
            wdone = true;
            if (lane == 0) atomicAdd(sm.done_warps, 1);
        }
        if (wdone && __shfl_sync(0xffffffffu, *done_warps, 0) >= C::kWarps) break;
        // (the producer issues no further batch once every warp is done)
        const int w = warp_wait(sm.full + s, (g / C::kStages) & 1u, done_warps, C::kWarps, sm.abort, a.wait_ns);
        if (w != kWaitDone) {
            if (w == kWaitTimeout && lane == 0) report(a.status, LSV2_ERR_TIMEOUT);
            if (!wdone && lane == 0) atomicAdd(sm.done_warps, 1);
            break;
        }
        if (!wdone) {
            const float4 box = lane < kB ? sm.box(s)[lane] : make_float4(0.0f, 0.0f, -1.0f, -1.0f);
            const bool keep = box.z >= 0.0f && box.x + box.z >= wx0 && box.x - box.z <= wx1 &&
                              box.y + box.w >= wy0 && box.y - box.w <= wy1;
            const unsigned char* recs = sm.rec(s);
            // kept records in list order, kChunk at a time
            uint32_t m = __ballot_sync(0xffffffffu, keep);
            while (m != 0u) {
                if (__all_sync(0xffffffffu, done)) break;
                int sl[kChunk];
#pragma unroll
                for (int j = 0; j < kChunk; ++j) {
                    sl[j] = m ? __ffs(m) - 1 : -1;
                    m &= m - 1u;
                }
                // (A) alpha_j and 1 - alpha_j of the chunk's records at this pixel: independent
                // of one another (instruction-level parallelism across the chunk); the records'
                // column offsets are loaded here too, so the accumulation's loads need not wait
                float al[kChunk], om[kChunk], p2s[kChunk], os[kChunk];
                // (records of up to 12 pairs: larger ones load their offsets in step C, so the
                // hoisted copies do not spill)
                constexpr bool kHoist = !C::kDense && C::kPairs <= 12;
                uint32_t offs[kChunk][kHoist ? C::kPairs : 1];
                bool high = false;
#pragma unroll
                for (int j = 0; j < kChunk; ++j) {
                    const float* r = reinterpret_cast<const float*>(recs + max(sl[j], 0) * C::kRecBytes);
                    const float4 g0 = *reinterpret_cast<const float4*>(r);
                    const float4 ax = *reinterpret_cast<const float4*>(r + 4);
                    const float4 axl = *reinterpret_cast<const float4*>(r + 8);
                    if constexpr (kHoist) {
                        const uint32_t* cw = reinterpret_cast<const uint32_t*>(r + 12 + C::kPairs);
                        if constexpr (C::kPairs % 4 == 0) {
#pragma unroll
                            for (int i = 0; i < C::kPairs / 4; ++i) {
                                const uint4 v4 = reinterpret_cast<const uint4*>(cw)[i];
                                offs[j][4 * i] = acc_ref<kTM>(v4.x);
                                offs[j][4 * i + 1] = acc_ref<kTM>(v4.y);
                                offs[j][4 * i + 2] = acc_ref<kTM>(v4.z);
                                offs[j][4 * i + 3] = acc_ref<kTM>(v4.w);
                            }
                        } else {
#pragma unroll
                            for (int p = 0; p < C::kPairs; ++p) offs[j][p] = acc_ref<kTM>(cw[p]);
                        }
                    }
                    const float p2 = eval_power2(g0, ax, axl, pxf, pyf);
                    float ex2;
                    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex2) : "f"(p2));
                    const float alpha = fminf(kAlphaMax, axl.w * ex2);
                    al[j] = (sl[j] >= 0 && p2 <= 0.0f && alpha >= kAlphaMin) ? alpha : 0.0f;
                    om[j] = 1.0f - al[j];
                    p2s[j] = p2;
                    os[j] = axl.w;
                    high = high || al[j] > 0.5f;
                }
                // 1 - alpha without cancellation where some pixel of the warp has alpha > 1/2
                // (rare: the plain difference is exact to within alpha's own error otherwise)
                if (__any_sync(0xffffffffu, high)) {
#pragma unroll
                    for (int j = 0; j < kChunk; ++j) om[j] = one_minus_alpha(al[j], os[j], p2s[j]);
                }
                // (B) front-to-back transmittance (Eq. 3): e_j = alpha_j T_j, the serial part;
                // al[j] becomes e_j (0 where the pixel skips or has terminated)
                uint32_t take_bits = 0;
                int li = -1;
#pragma unroll
                for (int j = 0; j < kChunk; ++j) {
                    const bool act = !done && al[j] > 0.0f;
                    const float test_T = T * om[j];
                    const bool stop = act && test_T < kTMin;
                    const bool take = act && !stop;
                    done = done || stop;
                    al[j] = take ? al[j] * T : 0.0f;
                    T = take ? test_T : T;
                    take_bits |= take ? (1u << j) : 0u;
                    li = take ? sl[j] : li;
                }
                if (li >= 0) last = b * kB + (uint32_t)li + 1u;
                // (C) W_col += w e_j for the pairs of every record some pixel of the warp takes
                const uint32_t used = __reduce_or_sync(0xffffffffu, take_bits);
#pragma unroll
                for (int j = 0; j < kChunk; ++j) {
                    if (used & (1u << j)) {
                        const float* r = reinterpret_cast<const float*>(recs + sl[j] * C::kRecBytes);
                        const float* wr = r + 12;
                        if constexpr (C::kDense) {
                            // every column of every level (zeros included)
#pragma unroll 4
                            for (int c4 = 0; c4 < C::kCols; c4 += 4) {
                                const float4 w4 = *reinterpret_cast<const float4*>(wr + c4);
                                float* a0 = acc + c4 * 33 + lane;
                                a0[0] = fmaf(al[j], w4.x, a0[0]);
                                a0[33] = fmaf(al[j], w4.y, a0[33]);
                                a0[66] = fmaf(al[j], w4.z, a0[66]);
                                a0[99] = fmaf(al[j], w4.w, a0[99]);
                            }
                        } else if constexpr (kTM) {
                            const uint32_t* cw = reinterpret_cast<const uint32_t*>(r + 12 + C::kPairs);
                            auto col = [&](int p) -> uint32_t {
                                if constexpr (kHoist) return offs[j][p];
                                else return acc_ref<true>(cw[p]);
                            };
                            // the pairs' columns are distinct (repeats and invalid indices sit
                            // in the dummy column), so all loads go before the stores; the
                            // stores land before the next record's loads
                            uint32_t v[C::kPairs];
#pragma unroll
                            for (int p = 0; p < C::kPairs; ++p) tc::tmem_ld1(tbase + col(p), v[p]);
                            tc::tmem_wait_ld_regs(v);
#pragma unroll
                            for (int p = 0; p < C::kPairs; ++p)
                                tc::tmem_st1(tbase + col(p), __float_as_uint(fmaf(al[j], wr[p], __uint_as_float(v[p]))));
                            tc::tmem_wait_st();
                        } else {
                            const uint32_t* cw = reinterpret_cast<const uint32_t*>(r + 12 + C::kPairs);
                            float v[C::kPairs];
                            float* addr[C::kPairs];
#pragma unroll
                            for (int p = 0; p < C::kPairs; ++p) {
                                uint32_t o;
                                if constexpr (kHoist) o = offs[j][p];
                                else o = cw[p];
                                addr[p] = reinterpret_cast<float*>(acc_lane + o);
                                v[p] = *addr[p];
                            }
#pragma unroll
                            for (int p = 0; p < C::kPairs; ++p) v[p] = fmaf(al[j], wr[p], v[p]);
#pragma unroll
                            for (int p = 0; p < C::kPairs; ++p) *addr[p] = v[p];
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tc::smem_u32(sm.empty + s));
        consumed = b + 1;
    }

    if (inside) {
        const size_t pix = (size_t)py * a.width + px;
        a.final_T[pix] = T;
        a.n_last[pix] = last;
    }
    __syncwarp();
    if (!kWriteCoeff) return consumed;
    // write this warp's 32 pixels (each pixel's L = C::kLW coefficients of a level are contiguous
    // in HBM)
    constexpr int LW = C::kLW;
    const size_t P = (size_t)a.width * a.height;
    if constexpr (kTM) {
        // each lane writes its own pixel's row of a level, read from TMEM 32 columns at a time
#pragma unroll 1
        for (int lev = 0; lev < LEVELS; ++lev) {
#pragma unroll 1
            for (int h = 0; h < LW / 32; ++h) {
                uint32_t r[32];
                tc::tmem_ld32(tbase + (uint32_t)(lev * LW + h * 32), r);
                tc::tmem_wait_ld_regs(r);
                if (inside) {
                    const size_t o = ((size_t)lev * P + (size_t)py * a.width + px) * LW + h * 32;
                    if (a.coeff_bf16) {
                        uint4* out = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.coeff) + o);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            __stcs(out + i, make_uint4(tc::pack_bf16(__uint_as_float(r[8 * i]), __uint_as_float(r[8 * i + 1])),
                                                       tc::pack_bf16(__uint_as_float(r[8 * i + 2]), __uint_as_float(r[8 * i + 3])),
                                                       tc::pack_bf16(__uint_as_float(r[8 * i + 4]), __uint_as_float(r[8 * i + 5])),
                                                       tc::pack_bf16(__uint_as_float(r[8 * i + 6]), __uint_as_float(r[8 * i + 7]))));
                    } else {
                        float4* out = reinterpret_cast<float4*>(a.coeff + o);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            __stcs(out + i, make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]),
                                                        __uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3])));
                    }
                }
            }
        }
        return consumed;
    }
    if (a.coeff_bf16) {
        __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(a.coeff);
        constexpr int G8 = LW / 8;   // 8-coefficient groups per pixel
#pragma unroll 1
        for (int lev = 0; lev < LEVELS; ++lev) {
            for (int q = lane; q < 32 * G8; q += 32) {
                const int pl = q / G8;  // pixel within the warp (its lane)
                const int c8 = (q % G8) * 8;
                const int gx = a.x0 + C::lane_x(warp, pl), gy = a.y0 + C::lane_y(warp, pl);
                if (gx < a.width && gy < a.height) {
                    const float* col = acc + (lev * LW + c8) * 33 + pl;
                    const uint4 val = make_uint4(tc::pack_bf16(col[0], col[33]), tc::pack_bf16(col[66], col[99]),
                                                 tc::pack_bf16(col[132], col[165]), tc::pack_bf16(col[198], col[231]));
                    __stcs(reinterpret_cast<uint4*>(out + ((size_t)lev * P + (size_t)gy * a.width + gx) * LW + c8), val);
                }
            }
        }
        return consumed;
    }
    constexpr int G4 = LW / 4;       // 4-coefficient groups per pixel
#pragma unroll 1
    for (int lev = 0; lev < LEVELS; ++lev) {
        for (int q = lane; q < 32 * G4; q += 32) {
            const int pl = q / G4;  // pixel within the warp (its lane)
            const int c4 = (q % G4) * 4;
            const int gx = a.x0 + C::lane_x(warp, pl), gy = a.y0 + C::lane_y(warp, pl);
            if (gx < a.width && gy < a.height) {
                const float* col = acc + (lev * LW + c4) * 33 + pl;
                float4 val = make_float4(col[0], col[33], col[66], col[99]);
                __stcs(reinterpret_cast<float4*>(a.coeff + ((size_t)lev * P + (size_t)gy * a.width + gx) * LW + c4), val);
            }
        }
    }
    return consumed;
}

// One tile by all threads of the CTA: kWarps consumer warps and the producer warp (the last
// one).  Precondition: the CTA's barriers are initialised, no tile is in progress and every
// thread is synchronised.  Returns the number of batches the tile used (the caller adds it to
// bbase).
template <int LEVELS, int K, int TW, int TH, int BATCH, bool kWriteCoeff = true, bool DENSE = false, int LW = 64>
__device__ __forceinline__ uint32_t splat_tile(const TileJob& a,
                                               const SplatSmem<SplatCfg<LEVELS, K, TW, TH, BATCH, DENSE, LW>>& sm,
                                               uint32_t bbase)
{
    using C = SplatCfg<LEVELS, K, TW, TH, BATCH, DENSE, LW>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t consumed = 0;
    if (warp == C::kWarps)
        splat_produce<C>(a, sm, lane, bbase);
    else
        consumed = splat_consume<C, LEVELS, K, TW, TH, kWriteCoeff>(a, sm, warp, lane, bbase);
    __syncthreads();
    const uint32_t issued = *sm.issued;
    if (threadIdx.x == 0) *sm.done_warps = 0;
    // Warps that stopped early release the stages of the batches they skipped (every one of
    // them lies within the last kStages batches, whose predecessors all warps released), so
    // each stage's barriers stay in step for the next tile.
    if (warp < C::kWarps && lane == 0 && !*reinterpret_cast<volatile int*>(sm.abort))
        for (uint32_t b = consumed; b < issued; ++b) tc::mbar_arrive(tc::smem_u32(sm.empty + (int)((bbase + b) % C::kStages)));
    return issued;
}

// One 16 x 16 tile with TMEM accumulators for consumer warps 4-7 (SplatCfg with TM = 4): warps
// 0-3 (rows 0-7) accumulate in shared memory, warps 4-7 (rows 8-15) in TMEM lane quarters 0-3,
// warp 8 produces.  Same contract as splat_tile; the CTA's TMEM allocation is in *sm.tmem_slot.
template <class C, int LEVELS, int K>
__device__ __forceinline__ uint32_t splat_tile_tm(const TileJob& a, const SplatSmem<C>& sm, uint32_t bbase)
{
    static_assert(C::kTmemWarps == 4 && C::kWarps == 8, "warps 4-7 in TMEM");
    constexpr int TW = 16, TH = 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t consumed = 0;
    if (warp == C::kWarps)
        splat_produce<C>(a, sm, lane, bbase);
    else if (warp < C::kSmemAccWarps)
        consumed = splat_consume<C, LEVELS, K, TW, TH, true, false>(a, sm, warp, lane, bbase);
    else
        consumed = splat_consume<C, LEVELS, K, TW, TH, true, true>(a, sm, warp, lane, bbase);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t issued = *sm.issued;
    if (threadIdx.x == 0) *sm.done_warps = 0;
    if (warp < C::kWarps && lane == 0 && !*reinterpret_cast<volatile int*>(sm.abort))
        for (uint32_t b = consumed; b < issued; ++b) tc::mbar_arrive(tc::smem_u32(sm.empty + (int)((bbase + b) % C::kStages)));
    return issued;
}

}  // namespace
}  // namespace lsv2
