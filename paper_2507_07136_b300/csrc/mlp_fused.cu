// mlp_fused.cu -- the decoder MLP of the decoder-based comparison path (LangSplat*, Sec. 3.1,
// Table 1) as one persistent tensor-core kernel.  Every layer's product runs on tcgen05 (BF16
// operands, FP32 accumulation in TMEM); bias and ReLU are applied in the epilogue, which rounds
// to BF16 and writes the result straight back into shared memory as the next layer's operand.
// Only the input rows are read and the output rows written: the hidden activations, which the
// layer-by-layer library GEMMs move through HBM (18 GB for a 1440x1080 frame at three levels),
// never leave the SM.
//
// One CTA per SM walks its 128-row tiles one at a time.  The tile's activations live in one
// buffer (128 rows x up to 256 BF16 columns, K-major with the 128-byte swizzle: the A operand,
// four 64-column K blocks); the accumulators alternate between two TMEM buffers of 256 columns,
// so the MMAs of product g + 1 run while the epilogue still reads product g.  The epilogue hands
// its output over one 64-column block at a time (act_ready[block]): the next product's MMAs
// start on block 0 while blocks 1..3 are still being written, which hides most of the tensor
// work behind the epilogue.  The weights stream through a ring of three 32 KB stages from a
// pre-swizzled image of W^T (a chunk = one product's outputs x 64 inputs, the K-major B operand)
// in the order the MMA warp takes them.  A last layer wider than 256 outputs runs as parts of
// 256 that read the same operand; its rows go out through a per-warp staging tile in shared
// memory, so that each store instruction writes 64-byte runs of 8 rows instead of 16 bytes of
// 32 rows.  Warps: 0 the weight producer, 1 the MMA issuer, 2-17 the epilogue (warp w reads TMEM
// lane quarter w % 4 and one 32-column piece of every 128 columns).  Every wait is bounded by the
// caller's limit; a CTA that gives up records LSV2_ERR_TIMEOUT, lets its copies and MMAs complete
// and frees TMEM.
//
// Measured on B300 at the decoder's widths (8-16-32-64-128-256-256-512, 2^20 rows): 0.96 ms,
// against 0.69 ms for the library GEMMs that stream every activation through HBM.  With one
// 128-row tile in flight per SM, each layer is a round trip MMA -> commit -> epilogue -> operand
// hand-over -> MMA whose latency the tensor pipe cannot hide (0.65 ms with the epilogue's
// arithmetic removed), and the epilogue's 16 warps are bound by their instruction issue; two
// tiles in flight (one TMEM accumulator each, MMAs alternating between them) measured 0.92 ms.
// TMEM (512 columns) and shared memory (one 64 KB operand per tile) allow no more tiles per SM
// while the weights stream.  So the library path is the default, and this kernel is the choice
// where memory is short: its workspace is the packed weights (under 2 MB) instead of two
// activation buffers of a row block (about 1 GB).
#include <cuda_bf16.h>

#include "device.cuh"
#include "mlp_fused.cuh"
#include "tc.cuh"

namespace lsv2 {
namespace {

constexpr int kM = 128;                           // rows per tile (TMEM lanes)
constexpr int kMaxK = 256;                        // widest operand held on chip
constexpr int kKBlock = kM * 128;                 // one 64-column K block of the tile (16 KB)
constexpr int kActBytes = kM * kMaxK * 2;         // 64 KB
constexpr int kStageBytes = 256 * 128;            // one weight chunk: <= 256 outputs x 64 inputs
constexpr int kStages = 3;
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kBufCols = 256;                // TMEM columns per accumulator buffer (two)
constexpr int kOutStage = 32 * 64;                // per epilogue warp: 32 rows x 32 BF16 columns
constexpr int kInStage = kM * 4 * 32;             // a tile's input: 128 rows x 4 chunks of 8 F32
constexpr int kRingOff = kActBytes;
constexpr int kOutOff = kRingOff + kStages * kStageBytes;
constexpr int kInOff = kOutOff + kEpiWarps * kOutStage;
constexpr int kBarOff = kInOff + kInStage;
constexpr int kBiasOff = kBarOff + 256;
constexpr int kSmemLimit = 232448;                // the opt-in maximum per CTA
constexpr int kMaxBias = (kSmemLimit - kBiasOff) / 16 * 4;   // biases held in shared memory as FP32
constexpr int kMaxInW = 32;                       // input width: one 16-byte chunk per epilogue group
static_assert(kMaxBias >= 1024, "room for the biases");

struct MlpArgs {
    MlpPlan plan;
    int64_t rows;
    const void* x;
    int x_f32;
    const uint8_t* image;
    const __nv_bfloat16* bias;
    __nv_bfloat16* y;
    int32_t* status;
    uint64_t wait_ns;
};

// Bounded wait of one thread: false once another thread gave up (abort flag) or after limit_ns
// (then it raises the flag).  The first check is a non-blocking test.
__device__ __forceinline__ bool mw(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t limit_ns)
{
    if (tc::mbar_test(bar, parity)) return true;
    const uint64_t t0 = tc::globaltimer();
    while (true) {
        if (*abort) return false;
        if (tc::globaltimer() - t0 >= limit_ns) {
            *abort = 1;
            return false;
        }
        if (tc::mbar_sleep(bar, parity, 20000u)) return true;
    }
}

// tcgen05.wait::ld with the loaded registers tied to it, so that no use of them moves above it.
template <int N>
__device__ __forceinline__ void wait_ld(uint32_t (&v)[N])
{
    if constexpr (N == 32) {
        tc::tmem_wait_ld_regs(v);
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 6)
            tc::tmem_wait_ld_tie6(v[i], v[i + 1 < N ? i + 1 : N - 1], v[i + 2 < N ? i + 2 : N - 1],
                                  v[i + 3 < N ? i + 3 : N - 1], v[i + 4 < N ? i + 4 : N - 1], v[i + 5 < N ? i + 5 : N - 1]);
    }
}

// Where the epilogue of one product sends its rows.
struct EpiOut {
    uint8_t* act;              // hidden product: the activation buffer (next layer's operand)
    uint8_t* stage;            // last layer: this warp's staging tile
    __nv_bfloat16* y;          // last layer: output, row-major [rows][out_w]
    int64_t row0;              // global row of this warp's lane 0
    int64_t rows;
    int out_w, out_col;
};

// NC accumulator columns of this thread's row (already loaded from TMEM): + bias (FP32, shared
// memory; `bias` points at column col), rounded to BF16, then for hidden products the ReLU on the
// rounded pairs (exact: rounding is monotonic and keeps the sign) and a store into the activation
// buffer (row r, columns col ..).  The last layer's parts go through the warp's staging tile
// (row = lane, 16-byte chunks XOR-swizzled by (row / 2) % 4 so that both the row-wise writes and
// the run-wise reads below are free of bank conflicts) and then out as 8 (NC = 32) or 16
// (NC = 16) row runs of NC * 2 bytes per store instruction.
template <int NC>
__device__ __forceinline__ void epi_finish(const uint32_t (&v)[NC], const float* bias, bool relu, const EpiOut& o,
                                           int r, int lane, int col)
{
    static_assert(NC == 32 || NC == 16, "32- or 16-column pieces");
    constexpr int kChunks = NC / 8;   // 16-byte chunks per row
    // the activation row's 128-byte line in this piece's K block, and its swizzle
    uint8_t* arow = o.act + (col >> 6) * kKBlock + r * 128;
    const int c0 = (col >> 3) & 7, rx = r & 7;
#pragma unroll
    for (int g = 0; g < kChunks; ++g) {
        const float4 b0 = *reinterpret_cast<const float4*>(bias + 8 * g);
        const float4 b1 = *reinterpret_cast<const float4*>(bias + 8 * g + 4);
        uint32_t pk[4];
        pk[0] = tc::pack_bf16(__uint_as_float(v[8 * g + 0]) + b0.x, __uint_as_float(v[8 * g + 1]) + b0.y);
        pk[1] = tc::pack_bf16(__uint_as_float(v[8 * g + 2]) + b0.z, __uint_as_float(v[8 * g + 3]) + b0.w);
        pk[2] = tc::pack_bf16(__uint_as_float(v[8 * g + 4]) + b1.x, __uint_as_float(v[8 * g + 5]) + b1.y);
        pk[3] = tc::pack_bf16(__uint_as_float(v[8 * g + 6]) + b1.z, __uint_as_float(v[8 * g + 7]) + b1.w);
        if (relu) {
            const __nv_bfloat162 zero = __float2bfloat162_rn(0.0f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const __nv_bfloat162 h = __hmax2(*reinterpret_cast<const __nv_bfloat162*>(&pk[j]), zero);
                pk[j] = *reinterpret_cast<const uint32_t*>(&h);
            }
            *reinterpret_cast<uint4*>(arow + (((c0 + g) ^ rx) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        } else {
            *reinterpret_cast<uint4*>(o.stage + lane * 64 + ((g ^ ((lane >> 1) & 3)) << 4)) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
    if (!relu) {
        __syncwarp();
        constexpr int kRowsPerStore = 32 / kChunks;
#pragma unroll
        for (int i = 0; i < kChunks; ++i) {
            const int rr = i * kRowsPerStore + lane / kChunks, ch = lane % kChunks;
            const uint4 w = *reinterpret_cast<const uint4*>(o.stage + rr * 64 + ((ch ^ ((rr >> 1) & 3)) << 4));
            const int64_t grow = o.row0 + rr;
            if (grow < o.rows)
                *reinterpret_cast<uint4*>(o.y + grow * o.out_w + o.out_col + col + 8 * ch) = w;
        }
        __syncwarp();   // the staging tile is free for the next piece
    }
}

// Arrival of this warp on the operand blocks next_blk .. blk (a hidden product's output written
// through block blk), after making its shared-memory writes visible to the tensor cores.
__device__ __forceinline__ void arrive_through(int& next_blk, int blk, int lane, uint64_t* act_ready)
{
    if (next_blk > blk) return;
    tc::fence_proxy_async();
    __syncwarp();
    if (lane == 0)
        for (int b = next_blk; b <= blk; ++b) tc::mbar_arrive(tc::smem_u32(act_ready + b));
    next_blk = blk + 1;
}

// One product's epilogue for this warp: its pieces are the 32-column pieces at
// c = 64 (2k + grp / 2) + 32 (grp % 2), k = 0, 1, .. below N (the 64-column blocks of parity
// grp / 2); a width of 16 mod 32 ends in a 16-column piece.  The TMEM load of the next piece is
// in flight while one is processed (each tcgen05.wait::ld covers exactly one outstanding load).
// A hidden product signals each 64-column block of its output as soon as this warp's share of
// it is written (every warp arrives on every block, in order).
__device__ __forceinline__ void epi_product(uint32_t tacc, int grp, int N, const float* bias, bool relu,
                                            const EpiOut& o, int r, int lane, uint64_t* act_ready)
{
    int next_blk = relu ? 0 : 4;   // first block this warp has not arrived on (none for the last layer)
    const int half = grp >> 1, sub = grp & 1;
    uint32_t va[32], vb[32];
    int k = 0;
    int c = 64 * half + 32 * sub;
    if (c + 32 <= N) {
        tc::tmem_ld32(tacc + (uint32_t)c, va);
        wait_ld(va);
        while (true) {
            // va holds the piece at c
            const int cn = c + 128;
            const bool more = cn + 32 <= N;
            if (more) tc::tmem_ld32(tacc + (uint32_t)cn, vb);
            epi_finish<32>(va, bias + c, relu, o, r, lane, c);
            arrive_through(next_blk, 2 * k + half, lane, act_ready);
            ++k;
            c = cn;
            if (!more) break;
            wait_ld(vb);
            const int cm = cn + 128;
            const bool more2 = cm + 32 <= N;
            if (more2) tc::tmem_ld32(tacc + (uint32_t)cm, va);
            epi_finish<32>(vb, bias + cn, relu, o, r, lane, cn);
            arrive_through(next_blk, 2 * k + half, lane, act_ready);
            ++k;
            c = cm;
            if (!more2) break;
            wait_ld(va);
        }
    }
    if (c < N) {   // the 16-column piece of a width of 16 mod 32
        uint32_t vs[16];
        tc::tmem_ld16(tacc + (uint32_t)c, vs);
        wait_ld(vs);
        epi_finish<16>(vs, bias + c, relu, o, r, lane, c);
        arrive_through(next_blk, c >> 6, lane, act_ready);
    }
    arrive_through(next_blk, (N + 63) / 64 - 1, lane, act_ready);
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(sdst)), "l"(gsrc) : "memory");
}

// Fetch of this thread's input chunk (row grow, columns 8 grp .. 8 grp + 7) of a tile into its
// slot of the input staging area (32 bytes per row and chunk) by cp.async, so that the load is
// in flight while the epilogue works and holds no registers.  Rows past the end and columns past
// the input width are not fetched.
__device__ __forceinline__ void fetch_input(const MlpArgs& a, uint8_t* istage, int r, int grp, int64_t grow)
{
    const int in_w = a.plan.in_w, c8 = grp * 8;
    if (grow < a.rows && c8 < in_w) {
        uint8_t* dst = istage + (r * 4 + grp) * 32;
        if (a.x_f32) {
            const float* src = static_cast<const float*>(a.x) + grow * in_w + c8;
            cp_async16(dst, src);
            cp_async16(dst + 16, src + 4);
        } else {
            cp_async16(dst, static_cast<const __nv_bfloat16*>(a.x) + grow * in_w + c8);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The fetched chunk as the first layer's operand (BF16, an F32 input rounded to nearest even;
// zero past the input width and past the last row), then this warp's arrival on K block 0.
__device__ __forceinline__ void store_input(const MlpArgs& a, const uint8_t* istage, uint8_t* act, int r, int grp,
                                            int lane, int64_t grow, uint64_t* act_ready)
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    const int c8 = grp * 8;
    if (c8 < a.plan.in_kp) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (grow < a.rows && c8 < a.plan.in_w) {
            const uint8_t* src = istage + (r * 4 + grp) * 32;
            if (a.x_f32) {
                const float4 lo = *reinterpret_cast<const float4*>(src), hi = *reinterpret_cast<const float4*>(src + 16);
                v = make_uint4(tc::pack_bf16(lo.x, lo.y), tc::pack_bf16(lo.z, lo.w), tc::pack_bf16(hi.x, hi.y),
                               tc::pack_bf16(hi.z, hi.w));
            } else {
                v = *reinterpret_cast<const uint4*>(src);
            }
        }
        *reinterpret_cast<uint4*>(act + tc::sw128(r, c8)) = v;
    }
    tc::fence_proxy_async();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(tc::smem_u32(act_ready));
}

__global__ void __launch_bounds__(kThreads, 1) mlp_fused_kernel(const __grid_constant__ MlpArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    // the 128-byte swizzle needs 1024-byte aligned operand tiles: a base that is not is reported,
    // never used
    if ((tc::smem_u32(smem) & 1023u) != 0) {
        if (threadIdx.x == 0) report(a.status, LSV2_ERR_UNSUPPORTED);
        return;
    }
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBarOff);
    uint64_t* w_full = bar;                     // [kStages] a weight chunk landed (transaction bytes)
    uint64_t* w_empty = bar + kStages;          // [kStages] the MMAs that read it completed (commit)
    uint64_t* acc_full = bar + 2 * kStages;     // [2] a product is complete in TMEM buffer b (commit)
    uint64_t* tfree = acc_full + 2;             // [2] the epilogue has read TMEM buffer b (16 warps)
    uint64_t* act_ready = tfree + 2;            // [4] a 64-column block of the operand is written (16 warps)
    uint64_t* drain = act_ready + 4;            // the MMA warp's last commit
    volatile int* abort = reinterpret_cast<volatile int*>(drain + 1);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1) + 1;
    float* sbias = reinterpret_cast<float*>(smem + kBiasOff);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const MlpPlan& P = a.plan;
    const int nsub = P.nsub;
    const int64_t ntiles = (a.rows + kM - 1) / kM;
    const int my_tiles = (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1);   // grid <= ntiles

    if (warp == 1) tc::tmem_alloc(tc::smem_u32(tslot), 2 * kBufCols);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(tc::smem_u32(w_full + s), 1);
            tc::mbar_init(tc::smem_u32(w_empty + s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(tc::smem_u32(acc_full + b), 1);
            tc::mbar_init(tc::smem_u32(tfree + b), kEpiWarps);
        }
        for (int j = 0; j < 4; ++j) tc::mbar_init(tc::smem_u32(act_ready + j), kEpiWarps);
        tc::mbar_init(tc::smem_u32(drain), 1);
        *abort = 0;
    }
    for (int i = tid; i < P.n_bias; i += kThreads) sbias[i] = __bfloat162float(a.bias[i]);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        // ---- producer: the weight chunks in the order the MMA warp takes them
        if (lane == 0) {
            const uint32_t ring = tc::smem_u32(smem + kRingOff);
            int k = 0;
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i)
                for (int l = 0; l < nsub && ok; ++l) {
                    const MlpSub& S = P.L[l];
                    const uint32_t bytes = (uint32_t)S.N * 128u;
                    for (int kb = 0; kb < S.nkb; ++kb, ++k) {
                        const int s = k % kStages;
                        if (k >= kStages &&
                            !mw(tc::smem_u32(w_empty + s), (uint32_t)((k / kStages - 1) & 1), abort, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc::bulk_load_arm(tc::smem_u32(w_full + s), bytes);
                        tc::bulk_load(ring + (uint32_t)(s * kStageBytes), a.image + S.w_off + (size_t)kb * bytes, bytes,
                                      tc::smem_u32(w_full + s));
                    }
                }
            // no copy may still be landing when the CTA retires
            for (int j = k > kStages ? k - kStages : 0; j < k; ++j)
                (void)tc::mbar_wait(tc::smem_u32(w_full + j % kStages), (uint32_t)((j / kStages) & 1), kDrainNs);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t ring = tc::smem_u32(smem + kRingOff);
            const uint32_t act = tc::smem_u32(smem);
            uint32_t ready_ph = 0;   // bit j: parity of the next act_ready[j] phase to wait for
            int k = 0;
            bool ok = true, issued = false;
            for (int i = 0; i < my_tiles && ok; ++i)
                for (int l = 0; l < nsub && ok; ++l) {
                    const int g = i * nsub + l, b = g & 1;
                    // the epilogue of product g - 2 has read this TMEM buffer
                    if (g >= 2 && !mw(tc::smem_u32(tfree + b), (uint32_t)(((g >> 1) - 1) & 1), abort, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const MlpSub& S = P.L[l];
                    // a product reads a fresh operand unless it is a further part of the last layer
                    const bool fresh = l == 0 || P.L[l - 1].relu;
                    const uint32_t d = tmem + (uint32_t)b * kBufCols;
                    const uint32_t idesc = tc::idesc_bf16(kM, S.N);
                    for (int kb = 0; kb < S.nkb; ++kb, ++k) {
                        if (fresh) {
                            if (!mw(tc::smem_u32(act_ready + kb), (ready_ph >> kb) & 1u, abort, a.wait_ns)) {
                                ok = false;
                                break;
                            }
                            ready_ph ^= 1u << kb;
                        }
                        const int s = k % kStages;
                        if (!mw(tc::smem_u32(w_full + s), (uint32_t)((k / kStages) & 1), abort, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint32_t wb = ring + (uint32_t)(s * kStageBytes);
                        const int left = (S.Kp - 64 * kb) / 16;
                        const int steps = left < 4 ? left : 4;
                        for (int kk = 0; kk < steps; ++kk)
                            tc::mma_bf16(d, tc::desc_sw128(act + (uint32_t)(kb * kKBlock + kk * 32)),
                                         tc::desc_sw128(wb + (uint32_t)(kk * 32)), idesc, (kb | kk) ? 1u : 0u);
                        tc::mma_commit(tc::smem_u32(w_empty + s));
                        issued = true;
                    }
                    if (!ok) break;
                    tc::mma_commit(tc::smem_u32(acc_full + b));
                }
            // no MMA may still read shared memory or write TMEM when the CTA retires
            if (issued) {
                tc::mma_commit(tc::smem_u32(drain));
                (void)tc::mbar_wait(tc::smem_u32(drain), 0u, kDrainNs);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp (q, grp) owns TMEM lane quarter q (rows 32 q ..) of every product
        const int e = warp - 2;
        const int q = warp & 3, grp = e >> 2;
        const int r = q * 32 + lane;
        uint8_t* act = smem;
        uint8_t* istage = smem + kInOff;
        EpiOut o;
        o.act = act;
        o.stage = smem + kOutOff + e * kOutStage;
        o.y = a.y;
        o.rows = a.rows;
        o.out_w = P.out_w;
        fetch_input(a, istage, r, grp, (int64_t)blockIdx.x * kM + r);
        store_input(a, istage, act, r, grp, lane, (int64_t)blockIdx.x * kM + r, act_ready);
        bool ok = true;
        for (int i = 0; i < my_tiles && ok; ++i) {
            const int64_t tile = (int64_t)blockIdx.x + (int64_t)i * gridDim.x;
            o.row0 = tile * kM + q * 32;
            const bool has_next = i + 1 < my_tiles;
            const int64_t next_row = (tile + gridDim.x) * kM + r;
            for (int l = 0; l < nsub; ++l) {
                const int g = i * nsub + l, b = g & 1;
                const bool last = l == nsub - 1;
                // the next tile's input starts loading two products before the end
                if (has_next && l == (nsub >= 2 ? nsub - 2 : 0)) fetch_input(a, istage, r, grp, next_row);
                if (!__all_sync(0xffffffffu, mw(tc::smem_u32(acc_full + b), (uint32_t)((g >> 1) & 1), abort, a.wait_ns))) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                // every MMA of this tile has completed: the operand buffer takes the next tile's
                // input, so that its first product runs while this epilogue writes the output
                if (last && has_next) store_input(a, istage, act, r, grp, lane, next_row, act_ready);
                const MlpSub& S = P.L[l];
                o.out_col = S.out_col;
                epi_product(tmem + (uint32_t)b * kBufCols + ((uint32_t)(q * 32) << 16), grp, S.N, sbias + S.b_off,
                            S.relu != 0, o, r, lane, act_ready);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_u32(tfree + b));
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (tid == 0 && *abort) report(a.status, LSV2_ERR_TIMEOUT);
    if (warp == 1) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 2 * kBufCols);
    }
}

// The weight image: for each part, its K blocks of 64 inputs one after another, each block N
// rows (outputs) x 128 bytes, 128-byte swizzle (K-major, 8-row groups 1024 bytes apart); inputs
// past the layer's width are zero.
__global__ void mlp_pack_kernel(const __grid_constant__ MlpPlan P, const __nv_bfloat16* __restrict__ W,
                                uint8_t* __restrict__ img)
{
    const MlpSub& S = P.L[blockIdx.y];
    const int total = S.nkb * 64 * S.N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int k = i / S.N, n = i % S.N;   // input, output within the part
        __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
        if (k < S.K) v = W[S.w_src + (int64_t)k * S.n_full + S.out_col + n];
        *reinterpret_cast<__nv_bfloat16*>(img + S.w_off + (size_t)(k >> 6) * (size_t)(S.N * 128) + tc::sw128(n, k & 63)) = v;
    }
}

int num_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 148;
    return n > 0 ? n : 148;
}

}  // namespace

bool mlp_fused_plan(int n_layers, const int32_t* widths, MlpPlan* plan, size_t* image_bytes)
{
    if (n_layers < 1 || widths[0] < 8 || widths[0] > kMaxInW || widths[0] % 8 != 0) return false;
    MlpPlan P{};
    P.in_w = widths[0];
    P.in_kp = (widths[0] + 15) / 16 * 16;
    P.out_w = widths[n_layers];
    int ns = 0, b_src = 0;
    int64_t w_src = 0;
    size_t off = 0;
    for (int l = 0; l < n_layers; ++l) {
        const int K = widths[l], N = widths[l + 1];
        const bool last = l == n_layers - 1;
        if (N < 16 || N % 16 != 0 || (!last && N > kMaxK)) return false;
        for (int o = 0; o < N; o += 256) {
            if (ns == kMlpMaxSub) return false;
            MlpSub& S = P.L[ns++];
            S.K = K;
            S.Kp = (K + 15) / 16 * 16;
            S.N = N - o < 256 ? N - o : 256;
            S.nkb = (S.Kp + 63) / 64;
            S.w_off = (int)off;
            S.b_off = b_src + o;
            S.out_col = o;
            S.relu = last ? 0 : 1;
            S.n_full = N;
            S.w_src = w_src;
            off += (size_t)S.nkb * (size_t)S.N * 128;
        }
        w_src += (int64_t)K * N;
        b_src += N;
    }
    if (b_src > kMaxBias) return false;
    P.nsub = ns;
    P.n_bias = b_src;
    *plan = P;
    *image_bytes = off;
    return true;
}

cudaError_t launch_mlp_fused(const MlpPlan& plan, int64_t rows, const void* x, bool x_f32, const void* weights,
                             const void* biases, void* y, void* image, int32_t* status, cudaStream_t stream)
{
    mlp_pack_kernel<<<dim3(32, plan.nsub), 256, 0, stream>>>(plan, static_cast<const __nv_bfloat16*>(weights),
                                                             static_cast<uint8_t*>(image));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    MlpArgs a{};
    a.plan = plan;
    a.rows = rows;
    a.x = x;
    a.x_f32 = x_f32 ? 1 : 0;
    a.image = static_cast<const uint8_t*>(image);
    a.bias = static_cast<const __nv_bfloat16*>(biases);
    a.y = static_cast<__nv_bfloat16*>(y);
    a.status = status;
    a.wait_ns = wait_limit_ns();
    const int64_t ntiles = (rows + kM - 1) / kM;
    const int sms = num_sms();
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    const int smem_bytes = kBiasOff + plan.n_bias * 4;
    mlp_fused_kernel<<<grid, kThreads, smem_bytes, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace lsv2
