// backward_tc.cu -- the decode adjoint of Loss = mean |F - target|, F = W S (Eq. 7), on the
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM).
//
// The adjoint is three contractions per 128-pixel tile of one level:
//     F = W S           (128 x 64) (64 x D)    only to decide G = sign(F - target)
//     dW = G S^T        (128 x D) (D x 64)
//     dS^T += G^T W     (D x 128) (128 x 64)    summed over every tile of the CTA
// G is -1, 0 or +1, exact in BF16; the scale 1 / (levels P D) multiplies the sums once.  W and
// S are split into BF16 high and low parts (x = hi + lo to within 2^-18 |x|): dW uses
// G (S_hi + S_lo)^T, dS^T uses G^T (W_hi + W_lo), F uses W_hi S_hi + W_hi S_lo + W_lo S_hi.
//
// Sign decisions.  The split products leave |F_tc - F| below about 1.2e-5 sum_l |W_l| |S_ld|.
// Where |F_tc - target| < tau_p = 1.3e-5 (sum_l |W_pl|) max|S| (a few elements per tile), the
// sign is provisional: it goes into G, the element is listed, and at the end of the kernel the
// residual is evaluated from the FP32 inputs as if in twice FP32 precision (Dot2); where its
// sign differs, dW and dS get the difference of the two signs' terms.  So every sign is the sign
// of the exact F - target, and the loss takes the accurate residual of the listed elements.
//
// One CTA per SM, persistent over the level's tiles; 224 KB of shared memory:
//  * S resident as blocks of 64 features, each S_hi (64 codebook rows x 128 bytes, 128-byte
//    swizzle) followed by S_lo: the MN-major B operand of F (K = codebook row, N = feature) and,
//    the same bytes, the K-major B operand of dW with N = 128 rows (S_hi rows then S_lo rows, so
//    one MMA forms G S_hi^T and G S_lo^T side by side).
//  * W_hi, W_lo of the tile (128 pixel rows x 64 BF16): the K-major A operand of F and the
//    MN-major B operand of dS^T (K = pixel, N = codebook row).
//  * G of one 128-feature chunk as two 64-feature atoms (128 pixel rows x 128 bytes): the
//    K-major A operand of dW and the MN-major A operand of dS^T (K = pixel, M = feature).
//  * the target through a two-stage ring of TMA tensor loads (128 pixels x 32 features FP32,
//    128-byte swizzle), with L2 prefetches of the boxes eight stages ahead.
//  * TMEM: the F chunk in columns [0, 128), dW [128, 256) (G S_hi^T, then G S_lo^T), dS^T
//    [256, 256 + D / 2) (one 64-column block per 128 features, lane = feature).
// Warps: 0 TMA producer; 1 MMA issuer (and TMEM owner); 2-9 epilogue (warp w reads TMEM lane
// quarter w % 4, i.e. 32 pixels; warps 2-5 take features 0-15 and warps 6-9 features 16-31 of
// each ring stage; all eight load and split the next tile's W).  Per chunk the MMA warp issues F
// of the chunk, then dS^T and dW of the previous chunk once its G is written, so the next F
// overlaps the epilogue.  The epilogue keeps a chunk's signs in registers while it drains the
// ring and writes G once the previous chunk's MMAs have read it, so the target stream does not
// wait for the tensor cores.  Every wait is bounded (the caller's limit); a CTA that gives up
// records LSV2_ERR_TIMEOUT, lets its TMA loads and MMAs complete and frees TMEM.
#include <cuda_bf16.h>

#include "backward.cuh"
#include "tc.cuh"
#include "tmap.cuh"

namespace lsv2 {
namespace {

constexpr int kM = 128;                          // pixels per tile (MMA rows)
constexpr int kL = 64;                           // codebook size
constexpr int kDC = 128;                         // features per chunk (F MMA N)
constexpr int kSD = 32;                          // features per ring stage
constexpr int kStagesPerChunk = kDC / kSD;
constexpr int kStageBytes = kSD * kM * 4;        // 16 KB
constexpr int kStages = 2;
constexpr int kPrefetch = 8;                     // ring stages prefetched into L2 ahead of their load
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kSBlock = kL * 128;                // 64 codebook rows x 64 features BF16 (8 KB)
constexpr int kSStride = 2 * kSBlock;            // a feature block: S_hi then S_lo
constexpr int kMaxD = 512;
constexpr int kS = 0;
constexpr int kWHi = kS + (kMaxD / 64) * kSStride;
constexpr int kWLo = kWHi + kM * 128;
constexpr int kGAtom = kM * 128;                 // 64 features of G (16 KB)
constexpr int kG = kWLo + kM * 128;
constexpr int kRing = kG + 2 * kGAtom;
constexpr int kMisc = kRing + kStages * kStageBytes;
constexpr int kFixCap = 160;                     // listed near-tie elements per CTA
constexpr int kWsumOff = 128, kFixOff = kWsumOff + kM * 4;
constexpr int kSmemBytes = 1024 + kMisc + kFixOff + 8 * kFixCap;   // alignment slack; barriers, sums, list
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColF = 0, kColDW = 128, kColDS = 256;
constexpr float kTieRel = 1.3e-5f;
static_assert(kSmemBytes <= 232448, "shared memory budget");
static_assert(kRing % 1024 == 0 && kG % 1024 == 0 && kWHi % 1024 == 0, "swizzled buffers are 1024-byte aligned");

struct L1TcArgs {
    int64_t P;
    int D;
    float inv_n;
    const float* W;        // [levels][P][64]
    const float* S;        // [levels][64][D]
    const float* target;   // [levels][P][D] (also read through the tensor map)
    float* loss;
    float* dW;
    float* dS;
    int32_t* status;
    uint64_t wait_ns;
};

// Bounded wait of one thread: false once the CTA's abort flag is up, or when the phase is still
// incomplete limit_ns after the wait began (which raises the flag).  The first check is a
// non-blocking test.
__device__ __forceinline__ bool bw_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t limit_ns)
{
    const uint64_t t0 = tc::globaltimer();
    if (tc::mbar_test(bar, parity)) return true;
    while (true) {
        if (*abort) return false;
        if (tc::globaltimer() - t0 >= limit_ns) {
            *abort = 1;
            return false;
        }
        if (tc::mbar_try(bar, parity)) return true;
    }
}

// The same for a whole warp: every lane takes the same decision.
__device__ __forceinline__ bool bw_wait_warp(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t limit_ns)
{
    return __all_sync(0xffffffffu, bw_wait(bar, parity, abort, limit_ns));
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Four floats split into BF16 high parts and BF16 low parts (x - hi rounded), as 8-byte quads.
__device__ __forceinline__ void split4(const float4& v, uint2& hi, uint2& lo)
{
    const float hx = bf16_round(v.x), hy = bf16_round(v.y), hz = bf16_round(v.z), hw = bf16_round(v.w);
    hi = make_uint2(tc::pack_bf16(hx, hy), tc::pack_bf16(hz, hw));
    lo = make_uint2(tc::pack_bf16(v.x - hx, v.y - hy), tc::pack_bf16(v.z - hz, v.w - hw));
}

// BF16 bits of sign(r) (sign(0) = 0)
__device__ __forceinline__ uint32_t sign_bf16(float r) { return r > 0.0f ? 0x3F80u : (r < 0.0f ? 0xBF80u : 0u); }

// sum_l W_l S_ld - t from the FP32 inputs, accumulated as if in twice FP32 precision (Dot2)
// and rounded: its sign is the sign of the exact residual unless that is within about 1e-13 of
// sum_l |W_l| |S_ld|.
__device__ float exact_residual(const float* w_row, const float* S, int D, int d, float t)
{
    float hi = -t, lo = 0.0f;
#pragma unroll 8
    for (int l = 0; l < kL; ++l) dot2_step(__ldg(w_row + l), __ldg(S + (size_t)l * D + d), hi, lo);
    return __fadd_rn(hi, lo);
}

template <int N>
__device__ __forceinline__ void tie_regs(uint32_t (&v)[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) asm volatile("" : "+r"(v[i]));
}

// W rows of the tile starting at pixel p0 into registers, coalesced: thread et (0..255) holds the
// 16-byte pieces c = et + 256 j (row c / 16, columns 4 (c % 16) ..); rows past P read as zero.
__device__ __forceinline__ void load_w_tile(float4 (&wpre)[8], const float* Wl, int64_t p0, int64_t P, int et)
{
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = et + 256 * j, r = c >> 4, c4 = c & 15;
        wpre[j] = p0 + r < P ? __ldcs(reinterpret_cast<const float4*>(Wl + (p0 + r) * kL + c4 * 4))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// The held W rows -> W_hi and W_lo (swizzled K-major tiles) and each row's sum |W| (the 16 lanes
// of a half-warp hold one row), then this warp's arrival on w_full.
__device__ __forceinline__ void store_w_tile(const float4 (&wpre)[8], uint8_t* smem, float* wsum, int et, int lane,
                                             uint64_t* w_full)
{
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = et + 256 * j, r = c >> 4, c4 = c & 15;
        uint2 hi, lo;
        split4(wpre[j], hi, lo);
        const uint32_t off = tc::sw128(r, c4 * 4);
        *reinterpret_cast<uint2*>(smem + kWHi + off) = hi;
        *reinterpret_cast<uint2*>(smem + kWLo + off) = lo;
        float sa = fabsf(wpre[j].x) + fabsf(wpre[j].y) + fabsf(wpre[j].z) + fabsf(wpre[j].w);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) sa += __shfl_xor_sync(0xffffffffu, sa, o);
        if ((lane & 15) == 0) wsum[r] = sa;
    }
    tc::fence_proxy_async();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(tc::smem_u32(w_full));
}

__global__ void __launch_bounds__(kThreads, 1)
    l1_decode_backward_tc_kernel(const __grid_constant__ CUtensorMap tmT, L1TcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kMisc);
    uint64_t* ring_full = bar;            // [kStages] a target stage landed (TMA bytes)
    uint64_t* ring_empty = bar + 2;       // [kStages] the epilogue read it (8 warps)
    uint64_t* w_full = bar + 4;           // the tile's W_hi / W_lo are written (8 warps)
    uint64_t* w_free = bar + 5;           // every MMA reading the tile's W completed (commit)
    uint64_t* f_full = bar + 6;           // the chunk's F is in TMEM (commit)
    uint64_t* f_free = bar + 7;           // the epilogue loaded F (8 warps)
    uint64_t* g_full = bar + 8;           // the chunk's G is written (8 warps)
    uint64_t* g_free = bar + 9;           // dW and dS^T of the chunk completed (commit)
    uint64_t* dw_full = bar + 10;         // the tile's dW is in TMEM (commit)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 11);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
    unsigned* smax_bits = reinterpret_cast<unsigned*>(tslot + 2);
    unsigned* fix_count = reinterpret_cast<unsigned*>(tslot + 3);
    float* wsum = reinterpret_cast<float*>(smem + kMisc + kWsumOff);        // [kM] sum_l |W| of the tile's pixels
    uint64_t* fix = reinterpret_cast<uint64_t*>(smem + kMisc + kFixOff);   // [kFixCap] listed near ties
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lev = blockIdx.y;
    const int D = a.D, nc = D / kDC;
    const int64_t P = a.P;
    const int64_t ntiles = (P + kM - 1) / kM;
    const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const float* Wl = a.W + (size_t)lev * P * kL;
    const float* Sl = a.S + (size_t)lev * kL * D;
    auto tile_p0 = [&](int i) -> int64_t { return ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kM; };

    if (warp == 1) tc::tmem_alloc(tc::smem_u32(tslot), kTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(tc::smem_u32(ring_full + s), 1);
            tc::mbar_init(tc::smem_u32(ring_empty + s), kEpiWarps);
        }
        tc::mbar_init(tc::smem_u32(w_full), kEpiWarps);
        tc::mbar_init(tc::smem_u32(w_free), 1);
        tc::mbar_init(tc::smem_u32(f_full), 1);
        tc::mbar_init(tc::smem_u32(f_free), kEpiWarps);
        tc::mbar_init(tc::smem_u32(g_full), kEpiWarps);
        tc::mbar_init(tc::smem_u32(g_free), 1);
        tc::mbar_init(tc::smem_u32(dw_full), 1);
        *abort = 0;
        *smax_bits = 0u;
        *fix_count = 0u;
    }
    __syncthreads();
    // S of the level -> S_hi, S_lo: element (l, d) of feature block d / 64 at byte sw128(l, d % 64)
    // of its S_hi (S_lo 8 KB further); and max |S|
    float smax_local = 0.0f;
    const int d4n = D / 4;
    for (int i = tid; i < kL * d4n; i += kThreads) {
        const int l = i / d4n, d = (i - l * d4n) * 4;
        const float4 v = __ldg(reinterpret_cast<const float4*>(Sl + (size_t)l * D + d));
        uint2 hi, lo;
        split4(v, hi, lo);
        const uint32_t off = (uint32_t)(d >> 6) * kSStride + tc::sw128(l, d & 63);
        *reinterpret_cast<uint2*>(smem + kS + off) = hi;
        *reinterpret_cast<uint2*>(smem + kS + kSBlock + off) = lo;
        smax_local = fmaxf(smax_local, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int o = 16; o > 0; o >>= 1) smax_local = fmaxf(smax_local, __shfl_xor_sync(0xffffffffu, smax_local, o));
    if (lane == 0) atomicMax(smax_bits, __float_as_uint(smax_local));   // non-negative floats order as their bits
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const float smax = __uint_as_float(*smax_bits);

    if (warp == 0) {
        // ---- TMA producer: the target boxes of every tile and chunk, in the epilogue's order
        if (lane == 0 && my_tiles > 0) {
            const int per_tile = nc * kStagesPerChunk;
            const int total = my_tiles * per_tile;
            auto box = [&](int k, int& x, int& y) {
                const int i = k / per_tile;
                x = (k - i * per_tile) * kSD;
                y = (int)tile_p0(i);
            };
            int x, y;
            for (int k = 0; k < kPrefetch && k < total; ++k) {
                box(k, x, y);
                tc::tma_prefetch_3d(&tmT, x, y, lev);
            }
            int issued = 0;
            for (int k = 0; k < total; ++k) {
                const int s = k % kStages;
                if (k >= kStages &&
                    !bw_wait(tc::smem_u32(ring_empty + s), (uint32_t)((k / kStages - 1) & 1), abort, a.wait_ns))
                    break;
                box(k, x, y);
                tc::bulk_load_arm(tc::smem_u32(ring_full + s), kStageBytes);
                tc::tma_load_3d(tc::smem_u32(smem + kRing + s * kStageBytes), &tmT, x, y, lev,
                                tc::smem_u32(ring_full + s));
                issued = k + 1;
                if (k + kPrefetch < total) {
                    box(k + kPrefetch, x, y);
                    tc::tma_prefetch_3d(&tmT, x, y, lev);
                }
            }
            // no load may still be landing when the CTA retires
            for (int k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
                (void)tc::mbar_wait(tc::smem_u32(ring_full + k % kStages), (uint32_t)((k / kStages) & 1), kDrainNs);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0 && my_tiles > 0) {
            const uint32_t idF = tc::idesc_bf16_major(kM, kDC, false, true);
            const uint32_t idW = tc::idesc_bf16_major(kM, 2 * kL, false, false);
            const uint32_t idS = tc::idesc_bf16_major(kM, kL, true, true);
            const uint32_t sb = tc::smem_u32(smem);
            const uint32_t sHi = sb + kS, sLo = sb + kS + kSBlock, wHi = sb + kWHi, wLo = sb + kWLo, gB = sb + kG;
            uint32_t last_bar = 0, last_par = 0;   // the latest commit (it covers every earlier MMA)
            auto commit = [&](uint64_t* b, uint32_t par) {
                tc::mma_commit(tc::smem_u32(b));
                last_bar = tc::smem_u32(b);
                last_par = par;
            };
            // dS^T and dW of chunk cc (global chunk g) of local tile i, once its G is written; at the
            // tile's last chunk W is released (w_free) as soon as dS^T, its last reader, is issued
            auto grads = [&](int g, int cc, int i, bool last) -> bool {
                if (!bw_wait(tc::smem_u32(g_full), (uint32_t)(g & 1), abort, a.wait_ns)) return false;
                tc::fence_after();
                for (int t = 0; t < 2; ++t) {
                    const uint32_t wB = t ? wLo : wHi;
#pragma unroll
                    for (int j = 0; j < kM / 16; ++j)
                        tc::mma_bf16(tmem + kColDS + (uint32_t)cc * 64, tc::desc_sw128_mn(gB + (uint32_t)j * 2048, kGAtom),
                                     tc::desc_sw128_mn(wB + (uint32_t)j * 2048, kGAtom), idS,
                                     (i > 0 || t > 0 || j > 0) ? 1u : 0u);
                }
                if (last) commit(w_free, (uint32_t)(i & 1));
                // dW += G [S_hi | S_lo]^T: N = 128 rows, the feature block's S_hi rows then its S_lo rows
#pragma unroll
                for (int j = 0; j < kDC / 16; ++j) {
                    const int d0 = cc * kDC + 16 * j;
                    tc::mma_bf16(tmem + kColDW, tc::desc_sw128(gB + (uint32_t)(j >> 2) * kGAtom + (uint32_t)(j & 3) * 32),
                                 tc::desc_sw128(sHi + (uint32_t)(d0 >> 6) * kSStride + (uint32_t)(j & 3) * 32), idW,
                                 (cc > 0 || j > 0) ? 1u : 0u);
                }
                commit(g_free, (uint32_t)(g & 1));
                if (last) commit(dw_full, (uint32_t)(i & 1));
                return true;
            };
            bool ok = true;
            int gc = 0;
            for (int i = 0; i < my_tiles && ok; ++i) {
                for (int c = 0; c < nc; ++c, ++gc) {
                    if (c == 0 && !bw_wait(tc::smem_u32(w_full), (uint32_t)(i & 1), abort, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (gc > 0 && !bw_wait(tc::smem_u32(f_free), (uint32_t)((gc - 1) & 1), abort, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    for (int t = 0; t < 3; ++t) {
                        const uint32_t aB = t == 2 ? wLo : wHi, bB = t == 1 ? sLo : sHi;
#pragma unroll
                        for (int k = 0; k < kL / 16; ++k)
                            tc::mma_bf16(tmem + kColF, tc::desc_sw128(aB + (uint32_t)k * 32),
                                         tc::desc_sw128_mn(bB + (uint32_t)(2 * c) * kSStride + (uint32_t)k * 2048, kSStride),
                                         idF, (t > 0 || k > 0) ? 1u : 0u);
                    }
                    commit(f_full, (uint32_t)(gc & 1));
                    if (c > 0 && !grads(gc - 1, c - 1, i, false)) {
                        ok = false;
                        break;
                    }
                }
                if (!ok) break;
                if (!grads(gc - 1, nc - 1, i, true)) {
                    ok = false;
                    break;
                }
            }
            if (!ok) report(a.status, LSV2_ERR_TIMEOUT);
            if (last_bar) (void)tc::mbar_wait(last_bar, last_par, kDrainNs);
        }
        __syncwarp();
    } else {
        // ---- epilogue
        const int e = warp - 2;                  // 0..7
        const int q = warp & 3;                  // TMEM lane quarter (pixels 32 q ..)
        const int h = e >> 2;                    // features 16 h .. 16 h + 15 of every ring stage
        const int row = q * 32 + lane;           // pixel row of the tile
        const int et = e * 32 + lane;            // 0..255: share of the W tile load
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        float4 wpre[8];
        double lacc = 0.0;
        bool ok = my_tiles > 0;
        if (ok) {
            load_w_tile(wpre, Wl, tile_p0(0), P, et);
            store_w_tile(wpre, smem, wsum, et, lane, w_full);
            if (my_tiles > 1) load_w_tile(wpre, Wl, tile_p0(1), P, et);
        }
        int gc = 0, k = 0;
        for (int i = 0; i < my_tiles && ok; ++i) {
            const int64_t p = tile_p0(i) + row;
            const bool valid = p < P;
            if (!bw_wait_warp(tc::smem_u32(w_full), (uint32_t)(i & 1), abort, a.wait_ns)) {
                ok = false;
                break;
            }
            const float tau = kTieRel * wsum[row] * smax;
            for (int c = 0; c < nc; ++c, ++gc) {
                if (!bw_wait_warp(tc::smem_u32(f_full), (uint32_t)(gc & 1), abort, a.wait_ns)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                uint32_t f[kStagesPerChunk][16];
#pragma unroll
                for (int s = 0; s < kStagesPerChunk; ++s) tc::tmem_ld16(tq + kColF + (uint32_t)(kSD * s + 16 * h), f[s]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int s = 0; s < kStagesPerChunk; ++s) tie_regs(f[s]);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_u32(f_free));
                float lsum = 0.0f;
                uint32_t gb[kStagesPerChunk][8];   // the chunk's signs (BF16 pairs) until G is free
                uint64_t ties = 0;
#pragma unroll
                for (int s = 0; s < kStagesPerChunk; ++s, ++k) {
                    const int slot = k % kStages;
                    if (!bw_wait_warp(tc::smem_u32(ring_full + slot), (uint32_t)((k / kStages) & 1), abort, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    // this thread's 16 target values: row `row`, 16-byte chunks 4 h .. 4 h + 3 (swizzled)
                    const uint8_t* st = smem + kRing + slot * kStageBytes + row * 128;
                    float t[16];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float4 x = *reinterpret_cast<const float4*>(st + (((4 * h + v) ^ (row & 7)) << 4));
                        t[4 * v] = x.x, t[4 * v + 1] = x.y, t[4 * v + 2] = x.z, t[4 * v + 3] = x.w;
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(tc::smem_u32(ring_empty + slot));
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        const float r0 = __uint_as_float(f[s][j]) - t[j], r1 = __uint_as_float(f[s][j + 1]) - t[j + 1];
                        const bool n0 = fabsf(r0) < tau, n1 = fabsf(r1) < tau;   // near ties: settled later
                        lsum += (n0 ? 0.0f : fabsf(r0)) + (n1 ? 0.0f : fabsf(r1));
                        ties |= (uint64_t)n0 << (16 * s + j);
                        ties |= (uint64_t)n1 << (16 * s + j + 1);
                        gb[s][j / 2] = sign_bf16(r0) | (sign_bf16(r1) << 16);
                    }
                }
                if (!ok) break;
                // G of this chunk once the previous chunk's MMAs have read the buffer: row `row`,
                // features fo .. fo + 15 of the chunk (atom fo / 64) per ring stage
                if (gc > 0 && !bw_wait_warp(tc::smem_u32(g_free), (uint32_t)((gc - 1) & 1), abort, a.wait_ns)) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int s = 0; s < kStagesPerChunk; ++s) {
                    const int fo = kSD * s + 16 * h;
                    uint8_t* gA = smem + kG + (fo >> 6) * kGAtom;
                    *reinterpret_cast<uint4*>(gA + tc::sw128(row, fo & 63)) = make_uint4(gb[s][0], gb[s][1], gb[s][2], gb[s][3]);
                    *reinterpret_cast<uint4*>(gA + tc::sw128(row, (fo & 63) + 8)) =
                        make_uint4(gb[s][4], gb[s][5], gb[s][6], gb[s][7]);
                }
                // near ties: listed with their provisional sign for the pass at the end; if the list is
                // full, settled here from the accurate residual (then G takes its sign)
                if (__any_sync(0xffffffffu, ties != 0) && valid) {
                    while (ties) {
                        const int b = __ffsll((long long)ties) - 1;
                        ties &= ties - 1;
                        const int fo = kSD * (b >> 4) + 16 * h + (b & 15);   // feature within the chunk
                        const int d = c * kDC + fo;
                        uint16_t* gp = reinterpret_cast<uint16_t*>(smem + kG + (fo >> 6) * kGAtom + tc::sw128(row, fo & 63));
                        const unsigned slot = atomicAdd(fix_count, 1u);
                        if (slot < (unsigned)kFixCap) {
                            const uint64_t sg = *gp == 0x3F80u ? 1u : (*gp == 0xBF80u ? 2u : 0u);
                            fix[slot] = (uint64_t)(uint32_t)p | ((uint64_t)d << 32) | (sg << 48);
                        } else {
                            const float r = exact_residual(Wl + p * kL, Sl, D, d, __ldg(a.target + ((size_t)lev * P + p) * D + d));
                            lacc += (double)fabsf(r);
                            *gp = (uint16_t)sign_bf16(r);
                        }
                    }
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_u32(g_full));
                lacc += (double)lsum;
            }
            if (!ok) break;
            // the next tile's W once every MMA of this tile has read W, then this tile's dW
            if (i + 1 < my_tiles) {
                if (!bw_wait_warp(tc::smem_u32(w_free), (uint32_t)(i & 1), abort, a.wait_ns)) {
                    ok = false;
                    break;
                }
                store_w_tile(wpre, smem, wsum, et, lane, w_full);
                if (i + 2 < my_tiles) load_w_tile(wpre, Wl, tile_p0(i + 2), P, et);
            }
            if (!bw_wait_warp(tc::smem_u32(dw_full), (uint32_t)(i & 1), abort, a.wait_ns)) {
                ok = false;
                break;
            }
            tc::fence_after();
            uint32_t dwh[32], dwl[32];   // G S_hi^T and G S_lo^T, codebook rows 32 h .. 32 h + 31
            tc::tmem_ld32(tq + kColDW + (uint32_t)(32 * h), dwh);
            tc::tmem_ld32(tq + kColDW + (uint32_t)(kL + 32 * h), dwl);
            tc::tmem_wait_ld_regs(dwh);
            tc::tmem_wait_ld_regs(dwl);
            tc::fence_before();
            if (valid) {
                float4* out = reinterpret_cast<float4*>(a.dW + ((size_t)lev * P + p) * kL + 32 * h);
                auto v4 = [&](int j) { return (__uint_as_float(dwh[j]) + __uint_as_float(dwl[j])) * a.inv_n; };
#pragma unroll
                for (int v = 0; v < 8; ++v) out[v] = make_float4(v4(4 * v), v4(4 * v + 1), v4(4 * v + 2), v4(4 * v + 3));
            }
        }
        // the listed near ties, after every epilogue warp has stored its dW rows (named barrier of
        // the 8 epilogue warps): the accurate residual's sign; where it differs from the
        // provisional one, dW and dS get (sign - provisional) / n times S and W
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
        const unsigned nfix = min(*reinterpret_cast<volatile unsigned*>(fix_count), (unsigned)kFixCap);
        if (ok && !*abort) {
            for (unsigned fi = (unsigned)et; fi < nfix; fi += 32u * kEpiWarps) {
                const uint64_t ent = fix[fi];
                const int64_t pp = (int64_t)(uint32_t)ent;
                const int d = (int)((ent >> 32) & 0xFFFFu);
                const int sg = (int)(ent >> 48);
                const float* wrow = Wl + pp * kL;
                const float r = exact_residual(wrow, Sl, D, d, __ldg(a.target + ((size_t)lev * P + pp) * D + d));
                lacc += (double)fabsf(r);
                const int ge = r > 0.0f ? 1 : (r < 0.0f ? -1 : 0), gp = sg == 1 ? 1 : (sg == 2 ? -1 : 0);
                if (ge != gp) {
                    const float delta = (float)(ge - gp) * a.inv_n;
                    for (int l = 0; l < kL; ++l) {
                        atomicAdd(a.dW + ((size_t)lev * P + pp) * kL + l, delta * __ldg(Sl + (size_t)l * D + d));
                        atomicAdd(a.dS + ((size_t)lev * kL + l) * D + d, delta * __ldg(wrow + l));
                    }
                }
            }
        }
        if (ok && my_tiles > 0) {
            // dS^T of this CTA (every MMA completed before the last dw_full): lane = feature within
            // a 128-feature block, column = codebook row; one atomic add per entry
            float* dSl = a.dS + (size_t)lev * kL * D;
            for (int cc = 0; cc < nc; ++cc) {
                uint32_t v[32];
                tc::tmem_ld32(tq + kColDS + (uint32_t)(cc * 64 + 32 * h), v);
                tc::tmem_wait_ld_regs(v);
                const int d = cc * kDC + row;
#pragma unroll
                for (int j = 0; j < 32; ++j) atomicAdd(dSl + (size_t)(32 * h + j) * D + d, __uint_as_float(v[j]) * a.inv_n);
            }
            tc::fence_before();
            for (int o = 16; o > 0; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
            if (lane == 0) atomicAdd(a.loss, (float)(lacc * (double)a.inv_n));
        }
        if (!ok && lane == 0) report(a.status, LSV2_ERR_TIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

bool l1_decode_backward_tc_supported(int D) { return D % kDC == 0 && D >= kDC && D <= kMaxD; }

cudaError_t launch_l1_decode_backward_tc(int levels, int64_t P, int D, const float* W, const float* S,
                                         const float* target, float* loss, float* dW, float* dS, int num_sms,
                                         int32_t* status, cudaStream_t stream)
{
    if (P == 0) return cudaSuccess;
    if (!l1_decode_backward_tc_supported(D) || P > (int64_t)INT32_MAX - kM) return cudaErrorInvalidValue;
    CUtensorMap tmT;
    // target [levels][P][D] FP32 in boxes of 32 features x 128 pixels (128-byte swizzle)
    if (!encode_tmap_3d(&tmT, target, false, (uint64_t)D, (uint64_t)P, (uint64_t)levels, (uint32_t)kSD, (uint32_t)kM,
                        true))
        return cudaErrorInvalidValue;
    L1TcArgs a{P, D, (float)(1.0 / ((double)levels * (double)P * (double)D)), W, S, target, loss, dW, dS, status,
               wait_limit_ns()};
    cudaError_t e = cudaFuncSetAttribute(l1_decode_backward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (P + kM - 1) / kM;
    int per_level = num_sms / levels;
    if (per_level < 1) per_level = 1;
    if (per_level > ntiles) per_level = (int)ntiles;
    l1_decode_backward_tc_kernel<<<dim3(per_level, levels), kThreads, kSmemBytes, stream>>>(tmT, a);
    return cudaGetLastError();
}

}  // namespace lsv2
