// decode_tc.cu -- Eq. 7 decode F_lev = W_lev S_lev on the tensor cores (tcgen05, BF16 operands,
// FP32 accumulation in TMEM), written for HBM: the (P x 64)(64 x D) product has 64 FMA per
// output element, so the kernel's job is to stream W in and F out at copy bandwidth.
//
// Persistent: one CTA (8 warps) per SM, CTAs split across levels.  Per CTA:
//  * S_lev^T (D x 64 BF16) is written once to shared memory in the 128-byte-swizzled K-major
//    layout the MMA reads (converted from FP32 if needed).
//  * The 128-pixel W tile reaches the same layout either by one TMA tensor load (BF16 W: the
//    map's 128-byte swizzle is the MMA's) or through registers with conversion (FP32 W).  It
//    is fetched for the next tile while the current tile's epilogue runs.
//  * One thread issues D/128 x 4 tcgen05.mma (M=128, N=128, K=16) into TMEM columns [0, D)
//    and commits to an mbarrier.
//  * Epilogue: warp w reads TMEM lane quarter w % 4 and half w / 4 of the columns, one 128-byte
//    wide box (32 rows) at a time, converts it into a 4 KB slot of its own ring in shared
//    memory (128-byte swizzle: conflict-free), and sends the box to HBM with one TMA tensor
//    store.  A slot is rewritten once the store issued kSlots boxes earlier has read it, so
//    the stores of consecutive tiles stream back to back; a tile's last box releases TMEM to
//    the next tile's MMA through an mbarrier, without a block-wide barrier.
// Every wait is time-bounded: on expiry the CTA records LSV2_ERR_TIMEOUT, lets its W load,
// MMA and bulk stores in flight complete, frees TMEM and returns.
#include "decode_tc.cuh"
#include "tc.cuh"
#include "tmap.cuh"

#include <cstring>

namespace lsv2 {
namespace {

constexpr int kM = 128;
constexpr int kK = 64;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSlots = 4;                  // output boxes in flight per warp
constexpr int kBoxBytes = 32 * 128;        // 32 rows x 128 bytes

struct DecodeTcArgs {
    int64_t P;
    int D;
    const void* W;
    int w_bf16;
    const void* S;
    int s_bf16;
    int out_bf16;
    int32_t* status;
    uint64_t wait_ns;     // bound of a wait on another warp's progress
};

__host__ __device__ constexpr size_t smem_bytes(int D)
{
    return 1024 + (size_t)D * 128 + (size_t)kM * 128 + (size_t)kWarps * kSlots * kBoxBytes + 64;
}

__device__ __forceinline__ void fetch_w(const DecodeTcArgs& a, int lev, int64_t p0, uint4 (&pre)[8])
{
    const int tid = threadIdx.x;
    if (a.w_bf16) {
        const __nv_bfloat16* Wl = static_cast<const __nv_bfloat16*>(a.W) + (size_t)lev * a.P * kK;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tid + kThreads * j, row = c >> 3, kc = c & 7;
            pre[j] = (p0 + row < a.P) ? __ldcs(reinterpret_cast<const uint4*>(Wl + (p0 + row) * kK + kc * 8))
                                      : make_uint4(0, 0, 0, 0);
        }
    } else {
        const float* Wl = static_cast<const float*>(a.W) + (size_t)lev * a.P * kK;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = tid + kThreads * j, row = c >> 4, c4 = c & 15;
            float4 v = (p0 + row < a.P) ? __ldcs(reinterpret_cast<const float4*>(Wl + (p0 + row) * kK + c4 * 4))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            pre[j] = make_uint4(__float_as_uint(v.x), __float_as_uint(v.y), __float_as_uint(v.z), __float_as_uint(v.w));
        }
    }
}

__device__ __forceinline__ void store_w(const DecodeTcArgs& a, uint8_t* sA, const uint4 (&pre)[8])
{
    const int tid = threadIdx.x;
    if (a.w_bf16) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tid + kThreads * j, row = c >> 3, kc = c & 7;
            *reinterpret_cast<uint4*>(sA + tc::sw128(row, kc * 8)) = pre[j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = tid + kThreads * j, row = c >> 4, c4 = c & 15;
            const uint2 v = make_uint2(tc::pack_bf16(__uint_as_float(pre[j].x), __uint_as_float(pre[j].y)),
                                       tc::pack_bf16(__uint_as_float(pre[j].z), __uint_as_float(pre[j].w)));
            *reinterpret_cast<uint2*>(sA + tc::sw128(row, c4 * 4)) = v;
        }
    }
}

__device__ __forceinline__ void issue_mma(uint32_t tmem, const uint8_t* sA, const uint8_t* sB, int D)
{
    const uint32_t idesc = tc::idesc_bf16(kM, 128);
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
    for (int nc = 0; nc < D / 128; ++nc)
#pragma unroll
        for (int k = 0; k < kK / 16; ++k)
            tc::mma_bf16(tmem + (uint32_t)(nc * 128), tc::desc_sw128(a0 + k * 32),
                         tc::desc_sw128(b0 + nc * 128 * 128 + k * 32), idesc, k > 0 ? 1u : 0u);
}

// kWTma: W is BF16 and arrives by TMA through tmW; otherwise through registers.
template <bool kWTma>
__global__ void __launch_bounds__(kThreads, 1)
    decode_tc_kernel(const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmW, DecodeTcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int D = a.D;
    uint8_t* sB = smem;
    uint8_t* sA = sB + (size_t)D * 128;
    uint8_t* sOut = sA + kM * 128;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sOut + kWarps * kSlots * kBoxBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const uint32_t mma_bar = tc::smem_u32(bar), free_bar = tc::smem_u32(bar + 1), w_bar = tc::smem_u32(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lev = blockIdx.y;
    const uint32_t ncols = D <= 128 ? 128u : (D <= 256 ? 256u : 512u);

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), ncols);
    if (tid == 0) {
        tc::mbar_init(mma_bar, 1);
        tc::mbar_init(free_bar, kWarps);
        tc::mbar_init(w_bar, 1);
    }
    // S_lev^T into the swizzled K-major layout: element (n, k) = S[lev][k][n]
    for (int i = tid; i < kK * D; i += kThreads) {
        const int k = i / D, n = i - k * D;
        const size_t src = (size_t)lev * kK * D + i;
        const __nv_bfloat16 v = a.s_bf16 ? static_cast<const __nv_bfloat16*>(a.S)[src]
                                         : __float2bfloat16_rn(static_cast<const float*>(a.S)[src]);
        *reinterpret_cast<__nv_bfloat16*>(sB + tc::sw128(n, k)) = v;
    }
    const int64_t ntiles = (a.P + kM - 1) / kM;
    int64_t tile = blockIdx.x;
    uint4 pre[8];
    if (!kWTma && tile < ntiles) {
        fetch_w(a, lev, tile * kM, pre);
        store_w(a, sA, pre);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    bool failed = false;
    uint32_t w_loads = 0, commits = 0;   // thread 0: TMA loads of W and MMA commits it issued
    if (tid == 0 && tile < ntiles) {
        if (kWTma) {
            tc::bulk_load_arm(w_bar, kM * 128);
            tc::tma_load_3d(tc::smem_u32(sA), &tmW, 0, (int)(tile * kM), lev, w_bar);
            ++w_loads;
            failed = !tc::mbar_wait(w_bar, 0, a.wait_ns);
        }
        if (!failed) {
            issue_mma(tmem, sA, sB, D);
            tc::mma_commit(mma_bar);
            ++commits;
        }
    }
    __syncwarp();

    const int q = warp & 3, half = warp >> 2;
    const int esz = a.out_bf16 ? 2 : 4;
    const int box_cols = 128 / esz;
    const int nbox = (D / 2) / box_cols;         // boxes per warp per tile
    uint8_t* ring = sOut + warp * (kSlots * kBoxBytes);
    const uint32_t tlane = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t g = 0;                              // boxes this warp has stored
    for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
        const int64_t next = tile + gridDim.x;
        if (!__all_sync(0xffffffffu, tc::mbar_wait(mma_bar, (uint32_t)it & 1u, a.wait_ns))) {
            failed = true;
            break;
        }
        tc::fence_after();
        // the next tile's W: sA is free now that this tile's MMA has completed
        if (next < ntiles) {
            if (kWTma) {
                if (tid == 0) {
                    tc::bulk_load_arm(w_bar, kM * 128);
                    tc::tma_load_3d(tc::smem_u32(sA), &tmW, 0, (int)(next * kM), lev, w_bar);
                    ++w_loads;
                }
            } else {
                fetch_w(a, lev, next * kM, pre);
            }
        }
        const int y = (int)(tile * kM) + q * 32;
        for (int b = 0; b < nbox; ++b, ++g) {
            const int col = half * (D / 2) + b * box_cols;
            uint8_t* slot = ring + (g % kSlots) * kBoxBytes;
            if (g >= (uint32_t)kSlots) {
                if (lane == 0) tc::bulk_wait_read<kSlots - 1>();
                __syncwarp();
            }
            uint32_t r[32];
            uint4 chunk[8];
            tc::tmem_ld32(tlane + (uint32_t)col, r);
            if (a.out_bf16) {
                uint32_t r2[32];
                tc::tmem_ld32(tlane + (uint32_t)(col + 32), r2);
                tc::tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    chunk[c] = make_uint4(tc::pack_bf16(__uint_as_float(r[8 * c]), __uint_as_float(r[8 * c + 1])),
                                          tc::pack_bf16(__uint_as_float(r[8 * c + 2]), __uint_as_float(r[8 * c + 3])),
                                          tc::pack_bf16(__uint_as_float(r[8 * c + 4]), __uint_as_float(r[8 * c + 5])),
                                          tc::pack_bf16(__uint_as_float(r[8 * c + 6]), __uint_as_float(r[8 * c + 7])));
                    chunk[c + 4] =
                        make_uint4(tc::pack_bf16(__uint_as_float(r2[8 * c]), __uint_as_float(r2[8 * c + 1])),
                                   tc::pack_bf16(__uint_as_float(r2[8 * c + 2]), __uint_as_float(r2[8 * c + 3])),
                                   tc::pack_bf16(__uint_as_float(r2[8 * c + 4]), __uint_as_float(r2[8 * c + 5])),
                                   tc::pack_bf16(__uint_as_float(r2[8 * c + 6]), __uint_as_float(r2[8 * c + 7])));
                }
            } else {
                tc::tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c) chunk[c] = make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
            }
            // row `lane` of the box: 16-byte chunk c at chunk position c ^ (lane % 8)
#pragma unroll
            for (int c = 0; c < 8; ++c)
                *reinterpret_cast<uint4*>(slot + lane * 128 + ((c ^ (lane & 7)) << 4)) = chunk[c];
            tc::fence_proxy_async();
            __syncwarp();
            // a box wholly past the level's last pixel is not stored (a ring slot is reused once at
            // most kSlots - 1 newer groups are pending, which holds with or without its group)
            if (lane == 0 && y < a.P) {
                tc::tma_store_3d(&tmF, col, y, lev, tc::smem_u32(slot));
                tc::bulk_commit();
            }
        }
        if (!kWTma && next < ntiles) store_w(a, sA, pre);
        // this warp is done with TMEM (and, FP32 W, has written its part of the next W tile)
        tc::fence_proxy_async();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(free_bar);
        if (tid == 0 && next < ntiles) {
            bool ok = tc::mbar_wait(free_bar, (uint32_t)it & 1u, a.wait_ns);
            if (kWTma && ok) ok = tc::mbar_wait(w_bar, (uint32_t)(it + 1) & 1u, a.wait_ns);
            if (ok) {
                tc::fence_after();
                issue_mma(tmem, sA, sB, D);
                tc::mma_commit(mma_bar);
                ++commits;
            } else {
                failed = true;
            }
        }
        __syncwarp();
    }
    if (failed) report(a.status, LSV2_ERR_TIMEOUT);
    // Thread 0 drains what it issued before TMEM is freed and the CTA retires: the latest W load
    // (load k completes phase k of w_bar) and the latest MMA commit (commit k completes phase k of
    // mma_bar; it covers every earlier MMA).  On the normal path both completed already.
    if (tid == 0) {
        if (w_loads > 0) (void)tc::mbar_wait(w_bar, (w_loads - 1) & 1u, kDrainNs);
        if (commits > 0) (void)tc::mbar_wait(mma_bar, (commits - 1) & 1u, kDrainNs);
    }
    if (lane == 0) tc::bulk_wait_all();
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ncols);
    }
}

}  // namespace

cudaError_t launch_decode_tc(int levels, int64_t P, int D, const void* W, bool w_bf16, const void* S, bool s_bf16,
                             void* F, bool out_bf16, int num_sms, int32_t* status, cudaStream_t stream)
{
    if (P == 0) return cudaSuccess;
    if (P > (int64_t)INT32_MAX - kM) return cudaErrorInvalidValue;   // TMA coordinates are 32-bit
    CUtensorMap tmF, tmW;
    // F [levels][P][D] in boxes of 128 bytes x 32 rows; W [levels][P][64] BF16 in 128-row tiles
    if (!encode_tmap_3d(&tmF, F, out_bf16, (uint64_t)D, (uint64_t)P, (uint64_t)levels, 128u / (out_bf16 ? 2u : 4u),
                        32u, false))
        return cudaErrorInvalidValue;
    if (w_bf16) {
        if (!encode_tmap_3d(&tmW, W, true, (uint64_t)kK, (uint64_t)P, (uint64_t)levels, (uint32_t)kK, (uint32_t)kM,
                            true))
            return cudaErrorInvalidValue;
    } else {
        std::memset(&tmW, 0, sizeof(tmW));
    }
    DecodeTcArgs a{P, D, W, w_bf16 ? 1 : 0, S, s_bf16 ? 1 : 0, out_bf16 ? 1 : 0, status, wait_limit_ns()};
    const size_t smem = smem_bytes(D);
    auto kernel = w_bf16 ? decode_tc_kernel<true> : decode_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (P + kM - 1) / kM;
    int per_level = num_sms / levels;
    if (per_level < 1) per_level = 1;
    if (per_level > ntiles) per_level = (int)ntiles;
    kernel<<<dim3(per_level, levels), kThreads, smem, stream>>>(tmF, tmW, a);
    return cudaGetLastError();
}

bool decode_tc_supported(int D) { return D % 128 == 0 && D <= 512 && smem_bytes(D) <= 232448; }

}  // namespace lsv2
