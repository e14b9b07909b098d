// decode_tc.cu -- Eq. 7 decode F_lev = W_lev S_lev on the tensor cores (tcgen05, BF16 operands,
// FP32 accumulation in TMEM), written for HBM: the (P x 64)(64 x D) product has 64 FMA per
// output element, so the kernel's job is to stream W in and F out at copy bandwidth.
//
// Persistent: one CTA (8 warps) per SM, CTAs split across levels.  Per CTA:
//  * S_lev^T (D x 64 BF16) is written once to shared memory in the 128-byte-swizzled K-major
//    layout the MMA reads (converted from FP32 if needed).
//  * Per 128-pixel tile: the W tile is converted to BF16 into the same layout; one thread
//    issues D/128 x 4 tcgen05.mma (M=128, N=128, K=16) into TMEM columns [0, D) and commits to
//    an mbarrier; the next tile's W is fetched into registers while the MMA runs.
//  * Epilogue: all 8 warps read TMEM (tcgen05.ld 32x32b; warps w and w+4 share lane quarter
//    w % 4 and split the columns), convert, write their row segment into a padded shared
//    staging row (16-byte skew between rows: conflict-free), and send each 512-byte segment
//    to HBM with one cp.async.bulk store.
// Every wait is time-bounded: on expiry the CTA records LSV2_ERR_TIMEOUT, drains its bulk
// stores, frees TMEM and returns.
#include "decode_tc.cuh"
#include "tc.cuh"

namespace lsv2 {
namespace {

constexpr int kM = 128;
constexpr int kK = 64;
constexpr int kThreads = 256;
constexpr int kRowBytes = 1024;            // staged bytes per row per pass
constexpr int kRowStride = kRowBytes + 16;

struct DecodeTcArgs {
    int64_t P;
    int D;
    const void* W;
    int w_bf16;
    const void* S;
    int s_bf16;
    void* F;
    int out_bf16;
    int32_t* status;
};

__host__ __device__ constexpr size_t smem_bytes(int D)
{
    return 1024 + (size_t)D * 128 + (size_t)kM * 128 + (size_t)kM * kRowStride + 64;
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

__global__ void __launch_bounds__(kThreads, 1) decode_tc_kernel(DecodeTcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int D = a.D;
    uint8_t* sB = smem;
    uint8_t* sA = sB + (size_t)D * 128;
    uint8_t* sOut = sA + kM * 128;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sOut + kM * kRowStride);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lev = blockIdx.y;
    const uint32_t ncols = D <= 128 ? 128u : (D <= 256 ? 256u : 512u);

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), ncols);
    if (tid == 0) tc::mbar_init(tc::smem_u32(bar), 1);
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
    if (tile < ntiles) {
        fetch_w(a, lev, tile * kM, pre);
        store_w(a, sA, pre);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(kM, 128);
    const int q = warp & 3, half = warp >> 2;
    const int row = q * 32 + lane;
    const int esz = a.out_bf16 ? 2 : 4;
    const int cols_pass = kRowBytes / esz < D ? kRowBytes / esz : D;   // columns staged per pass
    const int npass = D / cols_pass;
    const int seg_cols = cols_pass / 2;                                 // per thread per pass
    uint32_t phase = 0;
    bool failed = false;

    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t p0 = tile * kM;
        if (tid == 0) {
            tc::fence_after();
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
            for (int nc = 0; nc < D / 128; ++nc)
#pragma unroll
                for (int k = 0; k < kK / 16; ++k)
                    tc::mma_bf16(tmem + (uint32_t)(nc * 128), tc::desc_sw128(a0 + k * 32),
                                 tc::desc_sw128(b0 + nc * 128 * 128 + k * 32), idesc, k > 0 ? 1u : 0u);
            tc::mma_commit(tc::smem_u32(bar));
        }
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) fetch_w(a, lev, next * kM, pre);
        const bool ok = tc::mbar_wait(tc::smem_u32(bar), phase);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after();
        const int64_t p = p0 + row;
        uint8_t* srow = sOut + row * kRowStride + half * (seg_cols * esz);
        for (int pass = 0; pass < npass; ++pass) {
            tc::bulk_wait_read_all();
            for (int c = 0; c < seg_cols; c += 32) {
                uint32_t r[32];
                const int col = pass * cols_pass + half * seg_cols + c;
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, r);
                tc::tmem_wait_ld();
                if (a.out_bf16) {
                    uint4* dst = reinterpret_cast<uint4*>(srow + c * 2);
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        dst[v] = make_uint4(tc::pack_bf16(__uint_as_float(r[8 * v]), __uint_as_float(r[8 * v + 1])),
                                            tc::pack_bf16(__uint_as_float(r[8 * v + 2]), __uint_as_float(r[8 * v + 3])),
                                            tc::pack_bf16(__uint_as_float(r[8 * v + 4]), __uint_as_float(r[8 * v + 5])),
                                            tc::pack_bf16(__uint_as_float(r[8 * v + 6]), __uint_as_float(r[8 * v + 7])));
                } else {
                    uint4* dst = reinterpret_cast<uint4*>(srow + c * 4);
#pragma unroll
                    for (int v = 0; v < 8; ++v) dst[v] = make_uint4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
                }
            }
            if (p < a.P) {
                tc::fence_proxy_async();
                char* g = static_cast<char*>(a.F) +
                          (((size_t)lev * a.P + p) * D + pass * cols_pass + half * seg_cols) * esz;
                tc::bulk_store(g, tc::smem_u32(srow), (uint32_t)(seg_cols * esz));
                tc::bulk_commit();
            }
        }
        if (next < ntiles) store_w(a, sA, pre);
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
    }
    if (failed && tid == 0) report(a.status, LSV2_ERR_TIMEOUT);
    tc::bulk_wait_all();
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
    DecodeTcArgs a{P, D, W, w_bf16 ? 1 : 0, S, s_bf16 ? 1 : 0, F, out_bf16 ? 1 : 0, status};
    const size_t smem = smem_bytes(D);
    cudaError_t e = cudaFuncSetAttribute(decode_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (P + kM - 1) / kM;
    int per_level = num_sms / levels;
    if (per_level < 1) per_level = 1;
    if (per_level > ntiles) per_level = (int)ntiles;
    decode_tc_kernel<<<dim3(per_level, levels), kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

bool decode_tc_supported(int D) { return D % 128 == 0 && D <= 512 && smem_bytes(D) <= 232448; }

}  // namespace lsv2
