// query_tc.cu -- relevancy (Sec. 3.2) through the linearity of Eq. 7 on the tensor cores.
//
// Per level, Y = W B with B = [C | S t ...] (64 x N), S S^T = C C^T (C lower triangular, factored
// once per call), is one (128 x 64)(64 x N) tcgen05 product per 128-pixel tile (BF16 operands, FP32
// accumulation in TMEM).  The text columns are staged text-major: column 64 + t Qp + q holds text
// t (0 = positive, 1.. = negatives) of query q, Qp = Q rounded up to 8, so a thread reads 8
// queries' positives and each negative with one 8-column TMEM load apiece.  The epilogue thread
// that owns a pixel (one TMEM lane) forms
//     |F|^2 = W^T C C^T W = sum_j Y_j^2 (j < 64),
//     rel_q = sigmoid(tau (cos_pos - max_i cos_neg_i)),  cos_t = Y_t / (|F| |t|) (0 if |F| < 1e-12)
// as sigmoid(tau / |F| (Y_pos / |t_pos| - max_i Y_neg_i / |t_neg_i|)) (|F| > 0 commutes with the
// max), and writes rel[q][lev][p] (coalesced over the warp's 32 consecutive pixels).  F is never
// formed.  Persistent CTAs split over levels, B^T swizzled once per CTA.  Each 128-pixel W tile
// is 32 KB contiguous in HBM: one thread keeps a ring of two cp.async.bulk copies in flight
// (mbarrier transaction counts), all threads convert the landed tile to the swizzled BF16
// operand, one thread issues the MMA.  All waits are bounded.
#include "query_tc.cuh"
#include "tc.cuh"
#include "tmap.cuh"
#include "gram.cuh"

namespace lsv2 {
namespace {

constexpr int kM = 128;
constexpr int kK = 64;

struct QueryTcArgs {
    int Q, n_neg, Qp, npad;        // Qp = Q rounded up to 8; npad = 64 + (1 + n_neg) Qp rounded up to 16
    int q_off, Q_all;              // this launch's queries are q_off .. q_off + Q - 1 of Q_all
    float tau;
    const void* W;                 // per view v: [levels][P_v][64] at W + seg[v].w_off elements
    int w_bf16;                    // W in BF16 (else FP32)
    const float* Bt;               // [levels][64 + Q (1 + n_neg)][64] f32 (rows of B^T, query-major texts)
    const float* tnorm;            // [Q (1 + n_neg)] (query-major)
    void* rel;                     // per view v: [Q][levels][P_v] at rel + seg[v].rel_off
    int rel_bf16;
    int levels;
    int nseg;                      // views
    int64_t total_tiles;           // 128-pixel tiles over all views (per level)
    QuerySeg seg[kMaxQueryViews + 1];
    int32_t* status;
    uint64_t wait_ns;              // bound of a wait on another warp's progress
};

constexpr int kStages = 2;                      // W tiles in flight per CTA (bulk copies)
constexpr int kTileBytes = kM * kK * 4;         // one W tile (FP32: 32 KB; BF16: 16 KB), contiguous in HBM

__host__ __device__ constexpr int pad8(int q) { return (q + 7) / 8 * 8; }
__host__ __device__ constexpr int npad_of(int Q, int n_neg) { return (64 + (1 + n_neg) * pad8(Q) + 15) / 16 * 16; }

// ntp = (1 + n_neg) Qp reciprocal text norms, text-major
__host__ __device__ constexpr size_t smem_bytes(int npad, int ntp)
{
    return 1024 + (size_t)kStages * kTileBytes + (size_t)npad * 128 + (size_t)kM * 128 + (size_t)ntp * 4 + 128;
}

__host__ __device__ constexpr uint32_t tmem_cols(int npad)
{
    return npad <= 32 ? 32u : npad <= 64 ? 64u : npad <= 128 ? 128u : npad <= 256 ? 256u : 512u;
}

// BF16 tile (row-major, 128 bytes per row, in the ring) -> the swizzled K-major operand.
template <int NT>
__device__ __forceinline__ void copy_w_bf16(const uint8_t* src, int valid_rows, uint8_t* sA)
{
#pragma unroll
    for (int j = 0; j < 1024 / NT; ++j) {
        const int c = threadIdx.x + NT * j, row = c >> 3, kc = c & 7;
        const uint4 v = row < valid_rows ? *reinterpret_cast<const uint4*>(src + row * 128 + kc * 16)
                                         : make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(sA + tc::sw128(row, kc * 8)) = v;
    }
}

// FP32 tile (row-major, 64 floats per row, in the ring) -> BF16 swizzled K-major operand.
template <int NT>
__device__ __forceinline__ void convert_w(const float* src, int valid_rows, uint8_t* sA)
{
#pragma unroll
    for (int j = 0; j < 2048 / NT; ++j) {
        const int c = threadIdx.x + NT * j, row = c >> 4, c4 = c & 15;
        const float4 v = row < valid_rows ? *reinterpret_cast<const float4*>(src + row * kK + c4 * 4)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<uint2*>(sA + tc::sw128(row, c4 * 4)) =
            make_uint2(tc::pack_bf16(v.x, v.y), tc::pack_bf16(v.z, v.w));
    }
}

// BF16 relevancy from hk = tau / (2 |F|) and d = cos_pos - max cos_neg (in units of |F|): the
// sigmoid through the hardware tanh, 1/2 + tanh(hk d) / 2
__device__ __forceinline__ __nv_bfloat16 rel_bf16_of(float hk, float d)
{
    float th;
    asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(hk * d));
    return __float2bfloat16_rn(fmaf(0.5f, th, 0.5f));
}

// NT threads: 256 when two CTAs share an SM (TMEM allows), else 512, so that the epilogue of the
// one resident CTA has 16 warps (four per TMEM lane quarter).
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) query_tc_kernel(QueryTcArgs a)
{
    constexpr int kThreads = NT;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* ring = reinterpret_cast<float*>(smem);
    uint8_t* sB = smem + (size_t)kStages * kTileBytes;
    uint8_t* sA = sB + (size_t)a.npad * 128;
    float* sTn = reinterpret_cast<float*>(sA + kM * 128);
    const int per = 1 + a.n_neg;
    const int ntp = per * a.Qp;
    uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(sTn) + (((size_t)ntp * 4 + 15) & ~size_t(15)));
    uint64_t* full = bar + 1;                 // kStages barriers: W tile landed in the ring
    uint32_t* tslot = reinterpret_cast<uint32_t*>(full + kStages);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lev = blockIdx.y;
    const uint32_t ncols_alloc = tmem_cols(a.npad);
    const int64_t ntiles = a.total_tiles;
    // global tile -> (view, first pixel); tiles of view v are [seg[v].tile_base, seg[v + 1].tile_base)
    auto locate = [&](int64_t tile, int& v, int64_t& p0) {
        v = 0;
        while (v + 1 < a.nseg && tile >= a.seg[v + 1].tile_base) ++v;
        p0 = (tile - a.seg[v].tile_base) * kM;
    };
    // tiles of this CTA: blockIdx.x + i * gridDim.x, i = 0, 1, ...
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    int64_t last_issued = -1;       // thread 0: index of the last tile whose copy was issued
    auto issue = [&](int64_t i) {   // thread 0: bulk-copy the i-th tile of this CTA into its stage
        last_issued = i;
        int v;
        int64_t p0;
        locate(blockIdx.x + i * gridDim.x, v, p0);
        const int64_t Pv = a.seg[v].P;
        const int64_t rows = Pv - p0 < kM ? Pv - p0 : kM;
        const int esz = a.w_bf16 ? 2 : 4;
        const uint32_t bytes = (uint32_t)(rows * kK * esz);
        const int s = (int)(i % kStages);
        const uint8_t* src = static_cast<const uint8_t*>(a.W) + (a.seg[v].w_off + ((size_t)lev * Pv + p0) * kK) * esz;
        tc::bulk_load_arm(tc::smem_u32(full + s), bytes);
        tc::bulk_load(tc::smem_u32(ring + (size_t)s * kM * kK), src, bytes, tc::smem_u32(full + s));
    };

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), ncols_alloc);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(bar), 1);
        for (int s = 0; s < kStages; ++s) tc::mbar_init(tc::smem_u32(full + s), 1);
    }
    // B^T rows (N x 64 K-major, swizzled): the 64 rows of C^T (S S^T = C C^T), then the text rows S t / |t|
    // (the text norm folded in before the BF16 rounding, as in query_pipe_kernel) permuted from
    // query-major (64 + q per + t) to text-major (64 + t Qp + q); zero padding rows
    const float* Bl = a.Bt + (size_t)lev * (64 + a.Q * per) * kK;
    for (int i = tid; i < a.npad * kK; i += kThreads) {
        const int n = i >> 6, k = i & 63;
        int src = n < 64 ? n : -1;
        float scale = 1.0f;
        if (n >= 64 && n < 64 + ntp) {
            const int t = (n - 64) / a.Qp, q = (n - 64) % a.Qp;
            src = q < a.Q ? 64 + q * per + t : -1;
            if (q < a.Q) scale = 1.0f / a.tnorm[q * per + t];
        }
        const float v = src >= 0 ? Bl[(size_t)src * kK + k] * scale : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(sB + tc::sw128(n, k)) = __float2bfloat16_rn(v);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0)
        for (int64_t i = 0; i < kStages && i < my_tiles; ++i) issue(i);
    const uint32_t tmem = *tslot;
    const int q4 = warp & 3, part = warp >> 2;   // TMEM lane quarter; share of the query chunks
    const int row = q4 * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16);
    // 8-query chunks handled by this warp: contiguous shares of the NT / 128 warps of a quarter
    constexpr int kParts = NT / 128;
    const int nch = a.Qp / 8, ch = (nch + kParts - 1) / kParts;
    const int cb = part * ch < nch ? part * ch : nch, ce = (part + 1) * ch < nch ? (part + 1) * ch : nch;
    uint32_t phase = 0;
    bool failed = false;
    bool mma_pending = false;   // thread 0: an MMA was committed and not yet seen complete

    for (int64_t i = 0; i < my_tiles; ++i) {
        int vw;
        int64_t p0;
        locate(blockIdx.x + i * gridDim.x, vw, p0);
        const int64_t Pv = a.seg[vw].P;
        const int s = (int)(i % kStages);
        const bool landed = tc::mbar_wait(tc::smem_u32(full + s), (uint32_t)((i / kStages) & 1), a.wait_ns);
        if (__syncthreads_or(!landed)) {
            failed = true;
            break;
        }
        const int valid = Pv - p0 < kM ? (int)(Pv - p0) : kM;
        if (a.w_bf16) copy_w_bf16<NT>(reinterpret_cast<const uint8_t*>(ring + (size_t)s * kM * kK), valid, sA);
        else convert_w<NT>(ring + (size_t)s * kM * kK, valid, sA);
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();          // stage s is consumed; sA holds this tile; TMEM drained
        if (tid == 0) {
            if (i + kStages < my_tiles) issue(i + kStages);
            tc::fence_after();
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
            for (int n0 = 0; n0 < a.npad; n0 += 256) {
                const int nn = a.npad - n0 < 256 ? a.npad - n0 : 256;
                const uint32_t idesc = tc::idesc_bf16(kM, nn);
#pragma unroll
                for (int k = 0; k < kK / 16; ++k)
                    tc::mma_bf16(tmem + (uint32_t)n0, tc::desc_sw128(a0 + k * 32), tc::desc_sw128(b0 + n0 * 128 + k * 32),
                                 idesc, k > 0 ? 1u : 0u);
            }
            tc::mma_commit(tc::smem_u32(bar));
            mma_pending = true;
        }
        const bool ok = tc::mbar_wait(tc::smem_u32(bar), phase, a.wait_ns);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        mma_pending = false;
        phase ^= 1u;
        tc::fence_after();
        const int64_t p = p0 + row;
        // |F|^2 = |W C|^2: columns 0..63 of Y
        float n2;
        {
            uint32_t y0[32], y1[32];
            tc::tmem_ld32(trow, y0);
            tc::tmem_ld32(trow + 32u, y1);
            tc::tmem_wait_ld();
            n2 = chol_norm2(y0, y1);
        }
        const float nf = sqrtf(fmaxf(n2, 0.0f));
        const float kneg = nf < 1e-12f ? 0.0f : -a.tau / nf;   // exp(-tau (cos_p - max cos_n)) = exp(kneg d)
        for (int c = cb; c < ce; ++c) {
            const int q0 = c * 8;
            uint32_t rp[8], rn[8];
            tc::tmem_ld8(trow + (uint32_t)(64 + q0), rp);
            // the products are <F, t> / |t| (B's text rows carry 1/|t|): the same arithmetic as
            // query_pipe_kernel, so both give the same relevancy from the same W
            float best[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) best[j] = per > 1 ? -INFINITY : 0.0f;
            for (int t = 1; t < per; ++t) {
                tc::tmem_ld8(trow + (uint32_t)(64 + t * a.Qp + q0), rn);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; ++j) best[j] = fmaxf(best[j], __uint_as_float(rn[j]));
            }
            tc::tmem_wait_ld();
            if (p < Pv) {
                // rel = sigmoid(-kneg d); the element of query q is o0 + q stride
                const size_t stride = (size_t)a.levels * Pv;
                const size_t o0 = a.seg[vw].rel_off + (size_t)lev * Pv + p + (size_t)q0 * stride;
                const int nq = a.Q - q0 < 8 ? a.Q - q0 : 8;
                if (a.rel_bf16) {
                    // BF16 output: sigmoid(x) = 1/2 + tanh(x/2)/2 with the hardware tanh (its
                    // error, below 2.5e-4, is a tenth of the BF16 rounding of the result)
                    __nv_bfloat16* out = static_cast<__nv_bfloat16*>(a.rel) + o0;
                    const float hk = -0.5f * kneg;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (j >= nq) break;
                        out[(size_t)j * stride] = rel_bf16_of(hk, __uint_as_float(rp[j]) - best[j]);
                    }
                } else {
                    float* out = static_cast<float*>(a.rel) + o0;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (j >= nq) break;
                        const float d = __uint_as_float(rp[j]) - best[j];
                        out[(size_t)j * stride] = __fdividef(1.0f, 1.0f + __expf(kneg * d));
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();   // TMEM and the W tile are free
    }
    if (failed && tid == 0) report(a.status, LSV2_ERR_TIMEOUT);
    // an MMA whose completion the CTA gave up waiting for must finish before TMEM is freed
    if (tid == 0 && mma_pending) (void)tc::mbar_wait(tc::smem_u32(bar), phase, kDrainNs);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ncols_alloc);
    }
    // A CTA that gave up may still have bulk copies in flight into its shared memory: wait for
    // them (bounded) before the CTA retires.
    if (failed && tid == 0)
        for (int64_t i = last_issued; i >= 0 && i > last_issued - kStages; --i)
            (void)tc::mbar_wait(tc::smem_u32(full + (int)(i % kStages)), (uint32_t)((i / kStages) & 1), kDrainNs);
}

// ---- Pipelined form for a BF16 coefficient map and N <= 256 columns --------------------------
// Warp 0 streams W tiles into a ring of shared-memory stages with TMA tensor loads (the map's
// 128-byte swizzle is the MMA operand layout, so no copy or conversion); warp 1 issues each
// tile's MMA into one of ng TMEM accumulators; the remaining warps form ng epilogue warpgroups
// (ng = 3 for accumulators of up to 128 columns, else 2), tile i going to accumulator i % ng and
// warpgroup i % ng, so each accumulator's phases are consumed in order by one warpgroup.  The
// W stage is released by the completion of the MMA that read it (tcgen05.commit), the accumulator
// by its epilogue once the TMEM loads are done, through mbarriers, so tiles overlap: no
// block-wide barrier per tile.  W is addressed as rows of 64
// BF16 (row = view offset + level * P_v + pixel); a level's ragged last tile loads rows of the
// next level (or zeros past the end), whose results are not stored.

constexpr int kPStages = 8;
// epilogue warpgroups (= TMEM accumulators) for accumulators of `bufcols` columns
__host__ __device__ constexpr int pipe_groups(uint32_t bufcols) { return bufcols <= 128 ? 3 : 2; }

// per accumulator two warpgroups (splitting the query chunks) when there are at least two 8-query
// chunks and two accumulators, else one
__host__ __device__ constexpr int pipe_split(int ng, int nch) { return ng == 2 && nch >= 2 ? 2 : 1; }

__host__ __device__ constexpr size_t pipe_smem_bytes(int npad, int ntp)
{
    return 1024 + (size_t)kPStages * kM * 128 + (size_t)npad * 128 + (((size_t)ntp * 4 + 15) & ~size_t(15)) + 256;
}

// Bounded wait on a barrier phase: false once the CTA's abort flag is up, or when the phase is
// still incomplete limit_ns after the wait began (which raises the flag).  The first check is a
// non-blocking test, so with limit 0 the wait gives up unless the phase is complete at once.
__device__ __forceinline__ bool pipe_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t limit_ns)
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

// NB: TMEM accumulators; WPA: epilogue warpgroups per accumulator (template parameters, so that
// the per-tile ring and phase arithmetic divides by constants).  With WPA = 2 both warpgroups of
// an accumulator form |F|^2 from all 64 factor columns themselves (the same two 32-term sums in the
// same order, so the same value) and take alternate 8-query chunks: no exchange between them and
// no barrier per tile (sharing the halves through shared memory behind a named barrier measured
// 0.251 against 0.212 ms at 32 queries).

template <int NB, int WPA>
__global__ void __launch_bounds__(64 + 128 * NB * WPA, 1)
    query_pipe_kernel(const __grid_constant__ CUtensorMap tmW, QueryTcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ring = smem;                                        // kPStages x (128 x 128 bytes)
    uint8_t* sB = ring + (size_t)kPStages * kM * 128;
    float* sTn = reinterpret_cast<float*>(sB + (size_t)a.npad * 128);
    const int per = 1 + a.n_neg;
    const int ntp = per * a.Qp;
    uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(sTn) + (((size_t)ntp * 4 + 15) & ~size_t(15)));
    uint64_t* w_full = bar;                  // [kPStages] W tile landed (transaction bytes)
    uint64_t* w_empty = bar + kPStages;      // [kPStages] the MMA that read the tile has completed
    uint64_t* m_full = bar + 2 * kPStages;   // [4] accumulator b holds its tile (MMA commit)
    uint64_t* t_empty = m_full + 4;          // [4] accumulator b has been read (4 WPA warps)
    volatile int* abort = reinterpret_cast<volatile int*>(t_empty + 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(t_empty + 5);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lev = blockIdx.y;
    const uint32_t bufcols = tmem_cols(a.npad);
    constexpr int nb = NB;
    const uint32_t ncols_alloc = nb * bufcols <= 256u ? (nb * bufcols <= 128u ? 128u : 256u) : 512u;
    const int64_t ntiles = a.total_tiles;
    auto locate = [&](int64_t tile, int& v, int64_t& p0) {
        v = 0;
        while (v + 1 < a.nseg && tile >= a.seg[v + 1].tile_base) ++v;
        p0 = (tile - a.seg[v].tile_base) * kM;
    };
    // local tile counts fit 32 bits (at most 2^31 / 128 tiles per view and level)
    const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), ncols_alloc);
    if (tid == 0) {
        for (int s = 0; s < kPStages; ++s) {
            tc::mbar_init(tc::smem_u32(w_full + s), 1);
            tc::mbar_init(tc::smem_u32(w_empty + s), 1);
        }
        for (int b = 0; b < 4; ++b) {
            tc::mbar_init(tc::smem_u32(m_full + b), 1);
            tc::mbar_init(tc::smem_u32(t_empty + b), 4 * WPA);
        }
        *abort = 0;
    }
    // B^T rows: C^T (S S^T = C C^T), then the text rows S t / |t| text-major (the cosine's text
    // norm folded in before the BF16 rounding, so the products are <F, t> / |t|), zero padding
    const float* Bl = a.Bt + (size_t)lev * (64 + a.Q_all * per) * kK;
    for (int i = tid; i < a.npad * kK; i += (int)blockDim.x) {
        const int n = i >> 6, k = i & 63;
        int src = n < 64 ? n : -1;
        float scale = 1.0f;
        if (n >= 64 && n < 64 + ntp) {
            const int t = (n - 64) / a.Qp, q = (n - 64) % a.Qp;
            src = q < a.Q ? 64 + (a.q_off + q) * per + t : -1;
            if (q < a.Q) scale = 1.0f / a.tnorm[(a.q_off + q) * per + t];
        }
        const float v = src >= 0 ? Bl[(size_t)src * kK + k] * scale : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(sB + tc::sw128(n, k)) = __float2bfloat16_rn(v);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        // TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < my_tiles; ++i) {
                const int s = i % kPStages;
                if (i >= kPStages && !pipe_wait(tc::smem_u32(w_empty + s), (uint32_t)((i / kPStages - 1) & 1), abort, a.wait_ns))
                    break;
                int v;
                int64_t p0;
                locate((int64_t)blockIdx.x + (int64_t)i * gridDim.x, v, p0);
                const int64_t row = (int64_t)(a.seg[v].w_off / kK) + (int64_t)lev * a.seg[v].P + p0;
                tc::bulk_load_arm(tc::smem_u32(w_full + s), kM * 128);
                tc::tma_load_3d(tc::smem_u32(ring + (size_t)s * kM * 128), &tmW, 0, (int)row, 0, tc::smem_u32(w_full + s));
                issued = i + 1;
            }
            // no copy may still be landing when the CTA retires
            for (int i = issued > kPStages ? issued - kPStages : 0; i < issued; ++i)
                (void)tc::mbar_wait(tc::smem_u32(w_full + i % kPStages), (uint32_t)((i / kPStages) & 1), kDrainNs);
        }
        __syncwarp();
    } else if (warp == 1) {
        // MMA issuer: the W stage is released by the MMA's own completion (the epilogue does not
        // read W), the accumulator by its epilogue warps
        if (lane == 0) {
            int done = 0;
            for (int i = 0; i < my_tiles; ++i) {
                const int s = i % kPStages, b = i % nb;
                if (!pipe_wait(tc::smem_u32(w_full + s), (uint32_t)((i / kPStages) & 1), abort, a.wait_ns)) break;
                if (i >= nb && !pipe_wait(tc::smem_u32(t_empty + b), (uint32_t)((i / nb - 1) & 1), abort, a.wait_ns)) break;
                tc::fence_after();
                const uint32_t a0 = tc::smem_u32(ring + (size_t)s * kM * 128), b0 = tc::smem_u32(sB);
                const uint32_t idesc = tc::idesc_bf16(kM, a.npad);
#pragma unroll
                for (int k = 0; k < kK / 16; ++k)
                    tc::mma_bf16(tmem + (uint32_t)b * bufcols, tc::desc_sw128(a0 + k * 32), tc::desc_sw128(b0 + k * 32),
                                 idesc, k > 0 ? 1u : 0u);
                tc::mma_commit(tc::smem_u32(m_full + b));
                tc::mma_commit(tc::smem_u32(w_empty + s));
                done = i + 1;
            }
            // no MMA may still be writing TMEM when it is freed
            if (done > 0) {
                const int i = done - 1;
                (void)tc::mbar_wait(tc::smem_u32(m_full + i % nb), (uint32_t)((i / nb) & 1), kDrainNs);
            }
        }
        __syncwarp();
    } else {
        // epilogue: accumulator g's warpgroups (member m) take local tiles g, g + nb, ...; this
        // warp owns TMEM lane quarter q4
        const int e = warp - 2;
        const int g = e / (4 * WPA), m = (e >> 2) % WPA, q4 = warp & 3;
        const int row = q4 * 32 + lane;
        const int nch = a.Qp / 8;
        for (int i = g; i < my_tiles; i += nb) {
            const int b = i % nb;
            const uint32_t trow = tmem + (uint32_t)b * bufcols + ((uint32_t)(q4 * 32) << 16);
            const bool ok = __all_sync(0xffffffffu, pipe_wait(tc::smem_u32(m_full + b), (uint32_t)((i / nb) & 1), abort, a.wait_ns));
            if (!ok) break;
            tc::fence_after();
            float n2;
            {
                uint32_t y0[32], y1[32];
                tc::tmem_ld32(trow, y0);
                tc::tmem_ld32(trow + 32u, y1);
                tc::tmem_wait_ld();
                n2 = chol_norm2(y0, y1);
            }
            const float nf = sqrtf(fmaxf(n2, 0.0f));
            const float kneg = nf < 1e-12f ? 0.0f : -a.tau / nf;
            int vw;
            int64_t p0;
            locate((int64_t)blockIdx.x + (int64_t)i * gridDim.x, vw, p0);
            const int64_t Pv = a.seg[vw].P;
            const int64_t p = p0 + row;
            // this member's chunks m, m + WPA, ...; the accumulator is released after its last TMEM load
            const int c_last = m + ((nch - 1 - m) / WPA) * WPA;   // (WPA = 2 only with nch >= 2)
            if (m >= nch) {   // no chunk for this member: its last TMEM load was the norm's
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_u32(t_empty + b));
            }
            for (int c = m; c < nch; c += WPA) {
                const int q0 = c * 8;
                uint32_t rp[8], rn[8];
                tc::tmem_ld8(trow + (uint32_t)(64 + q0), rp);
                // best[j] = max over the negatives of <F, t_neg> / |t_neg| (0 with none)
                float best[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) best[j] = per > 1 ? -INFINITY : 0.0f;
                if (per == 5) {
                    // four negatives: their loads behind one wait
                    uint32_t r4[4][8];
#pragma unroll
                    for (int t = 0; t < 4; ++t) tc::tmem_ld8(trow + (uint32_t)(64 + (t + 1) * a.Qp + q0), r4[t]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 4; ++t)
#pragma unroll
                        for (int j = 0; j < 8; ++j) best[j] = fmaxf(best[j], __uint_as_float(r4[t][j]));
                } else {
                    for (int t = 1; t < per; ++t) {
                        tc::tmem_ld8(trow + (uint32_t)(64 + t * a.Qp + q0), rn);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 8; ++j) best[j] = fmaxf(best[j], __uint_as_float(rn[j]));
                    }
                    tc::tmem_wait_ld();
                }
                if (c == c_last) {
                    // this warp's last TMEM load of the tile is done: release the accumulator
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(tc::smem_u32(t_empty + b));
                }
                if (p < Pv) {
                    const size_t stride = (size_t)a.levels * Pv;
                    const size_t o0 = a.seg[vw].rel_off + (size_t)lev * Pv + p + (size_t)(a.q_off + q0) * stride;
                    const int nq = a.Q - q0 < 8 ? a.Q - q0 : 8;
                    float d[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) d[j] = __uint_as_float(rp[j]) - best[j];
                    if (a.rel_bf16) {
                        __nv_bfloat16* out = static_cast<__nv_bfloat16*>(a.rel) + o0;
                        const float hk = -0.5f * kneg;
                        if (nq == 8) {
#pragma unroll
                            for (int j = 0; j < 8; ++j, out += stride) *out = rel_bf16_of(hk, d[j]);
                        } else {
                            for (int j = 0; j < nq; ++j, out += stride) *out = rel_bf16_of(hk, d[j]);
                        }
                    } else {
                        float* out = static_cast<float*>(a.rel) + o0;
                        if (nq == 8) {
#pragma unroll
                            for (int j = 0; j < 8; ++j, out += stride) *out = __fdividef(1.0f, 1.0f + __expf(kneg * d[j]));
                        } else {
                            for (int j = 0; j < nq; ++j, out += stride) *out = __fdividef(1.0f, 1.0f + __expf(kneg * d[j]));
                        }
                    }
                }
            }
        }
    }
    if (tid == 0 && *abort) report(a.status, LSV2_ERR_TIMEOUT);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ncols_alloc);
    }
}

}  // namespace

bool query_tc_supported(int Q, int n_neg)
{
    if (Q < 1 || n_neg < 1) return false;
    const int npad = npad_of(Q, n_neg), ntp = (1 + n_neg) * pad8(Q);
    return npad <= 512 && smem_bytes(npad, ntp) <= 232448 &&
           (512u / tmem_cols(npad) >= 2 || smem_bytes(npad, ntp) >= 117760);
}

cudaError_t launch_query_tc_views(int levels, int V, const int64_t* P, int Q, int n_neg, float tau, const void* W,
                                  bool w_bf16,
                                  const float* Bt, const float* tnorm, void* rel, bool rel_bf16, int num_sms,
                                  int32_t* status, cudaStream_t stream)
{
    if (V < 1 || V > kMaxQueryViews) return cudaErrorInvalidValue;
    const int npad = npad_of(Q, n_neg), ntp = (1 + n_neg) * pad8(Q);
    if (npad > 512) return cudaErrorInvalidValue;
    QueryTcArgs a{};
    a.Q = Q;
    a.q_off = 0;
    a.Q_all = Q;
    a.n_neg = n_neg;
    a.Qp = pad8(Q);
    a.npad = npad;
    a.tau = tau;
    a.W = W;
    a.w_bf16 = w_bf16 ? 1 : 0;
    a.Bt = Bt;
    a.tnorm = tnorm;
    a.rel = rel;
    a.rel_bf16 = rel_bf16 ? 1 : 0;
    a.levels = levels;
    a.nseg = V;
    a.status = status;
    a.wait_ns = wait_limit_ns();
    int64_t tiles = 0;
    size_t w_off = 0, rel_off = 0;
    for (int v = 0; v < V; ++v) {
        a.seg[v] = QuerySeg{P[v], tiles, w_off, rel_off};
        tiles += (P[v] + kM - 1) / kM;
        w_off += (size_t)levels * P[v] * kK;
        rel_off += (size_t)Q * levels * P[v];
    }
    a.seg[V] = QuerySeg{0, tiles, w_off, rel_off};
    a.total_tiles = tiles;
    if (tiles == 0) return cudaSuccess;
    // pipelined form (BF16 W): queries in groups whose columns fit a 256-column accumulator
    int Qg = Q;
    while (Qg > 8 && tmem_cols(npad_of(Qg, n_neg)) > 256) Qg = (Qg - 1) / 8 * 8;
    if (w_bf16 && tmem_cols(npad_of(Qg, n_neg)) <= 256) {
        // W as rows of 64 BF16 over all views and levels
        CUtensorMap tmW;
        if (!encode_tmap_3d(&tmW, W, true, (uint64_t)kK, (uint64_t)(w_off / kK), 1u, (uint32_t)kK, (uint32_t)kM, true))
            return cudaErrorInvalidValue;
        int per_level = num_sms / levels;
        if (per_level < 1) per_level = 1;
        if (per_level > tiles) per_level = (int)tiles;
        for (int q0 = 0; q0 < Q; q0 += Qg) {
            QueryTcArgs g = a;
            g.q_off = q0;
            g.Q = Q - q0 < Qg ? Q - q0 : Qg;
            g.Qp = pad8(g.Q);
            g.npad = npad_of(g.Q, n_neg);
            size_t smem = pipe_smem_bytes(g.npad, (1 + n_neg) * g.Qp);
            if (smem < 117760) smem = 117760;   // one CTA per SM: its TMEM allocation never waits
            if (smem > 232448) return cudaErrorInvalidValue;
            const int ng = pipe_groups(tmem_cols(g.npad)), split = pipe_split(ng, g.Qp / 8);
            auto kern = ng == 3 ? query_pipe_kernel<3, 1> : split == 2 ? query_pipe_kernel<2, 2> : query_pipe_kernel<2, 1>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            kern<<<dim3(per_level, levels), 64 + 128 * ng * split, smem, stream>>>(tmW, g);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // Two CTAs per SM when their TMEM allocations fit (one CTA's MMA and W conversion overlap the
    // other's epilogue); the shared-memory request keeps one more CTA from being resident, so
    // tcgen05.alloc never waits on another CTA.
    const int resident = 512u / tmem_cols(npad) >= 2 ? 2 : 1;
    size_t smem = smem_bytes(npad, ntp);
    const size_t floor_bytes = 233472 / (size_t)(resident + 1) + 1024;
    if (smem < floor_bytes) smem = floor_bytes;
    if (smem > 232448) return cudaErrorInvalidValue;
    auto kern = resident == 2 ? query_tc_kernel<256> : query_tc_kernel<512>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_level = num_sms * resident / levels;
    if (per_level < 1) per_level = 1;
    if (per_level > tiles) per_level = (int)tiles;
    kern<<<dim3(per_level, levels), resident == 2 ? 256 : 512, smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_query_tc(int levels, int64_t P, int Q, int n_neg, float tau, const void* W, bool w_bf16,
                            const float* Bt,
                            const float* tnorm, void* rel, bool rel_bf16, int num_sms, int32_t* status,
                            cudaStream_t stream)
{
    if (P == 0) return cudaSuccess;
    return launch_query_tc_views(levels, 1, &P, Q, n_neg, tau, W, w_bf16, Bt, tnorm, rel, rel_bf16, num_sms, status,
                                 stream);
}

}  // namespace lsv2
