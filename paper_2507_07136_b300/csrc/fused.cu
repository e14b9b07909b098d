// fused.cu -- one frame's sparse-coefficient splat (Sec. 3.4, Algorithm 1), decode F = W S
// (Eq. 7) and relevancy (Sec. 3.2 through Eq. 7) in one kernel: the coefficient map W never
// leaves the SM.
//
// One CTA per 16x8 half of a 16x16 bin tile, two CTAs per SM, so that one CTA's decode (bound by
// the HBM write stream) overlaps the other's splat (bound by shared memory and latency).  A CTA
// is 4 consumer warps (8x4 pixels each) and one producer warp, as in the plain splat
// (splat_core.cuh).  After the splat each consumer warp holds the FP32 coefficients of its 32
// pixels in shared-memory columns.  Then:
//  1. Transit: every thread stores its pixel's 3 x 64 coefficients, rounded to BF16, into its
//     TMEM lane (tcgen05.st), which frees the accumulator memory; after a barrier it reads them
//     back (tcgen05.ld) and writes the 128-byte-swizzled K-major A tile of each level (128 rows =
//     the block's pixels in row-major order) into that memory.
//  2. The producer warp streams the codebook S_lev^T in 8 KB chunks of 64 rows (the pre-swizzled
//     BF16 copy) through a 2-slot ring with bulk async copies, and each level's query matrix
//     [C | S t / |t| ...] (S S^T = C C^T; text-major rows, as in query_tc.cu); its lane 0 issues the
//     tcgen05.mma: per level Y = W [C | S t / |t|] (M = 128, N = npadq <= 128) into TMEM columns
//     [128, 256), then
//     F chunks of 64 features (M = 128, N = 64, K = 64) into two TMEM buffers [0, 64) and
//     [64, 128) that alternate, each committed to an mbarrier.
//  3. The consumer warps run the epilogues in the same order (warp q reads TMEM lanes 32q ..,
//     i.e. image rows 2q and 2q + 1 of the block): relevancy as in query_tc.cu (|F|^2 = |W C|^2,
//     sigmoid of the scaled cosine gap), and F chunks converted to BF16 into two
//     16-pixel x 128-byte staging boxes per warp, each sent by one TMA tensor store through a
//     {D, W, H, levels} map (columns past the image edge are clipped by the map).
// The operands and the MMA sequence (K = 64 in four steps of 16) are those of decode_tc.cu and
// query_tc.cu, so F and the relevancy equal those kernels' results on the splat's W.  Every wait
// is time-bounded: on expiry the CTA records LSV2_ERR_TIMEOUT, skips the rest, lets the copies
// and MMAs it issued complete, and frees TMEM.
#include <cuda_bf16.h>

#include <cstring>

#include "query.cuh"
#include "splat_core.cuh"
#include "gram.cuh"
#include "tmap.cuh"

namespace lsv2 {
namespace {

constexpr int kLev = 3, kKp = 4, kTW = 16, kTH = 16, kHH = 8;   // bin tile 16x16, CTA block 16x8
using FC = SplatCfg<kLev, kKp, kTW, kHH, 0>;                     // 4 consumer warps + the producer
constexpr int kM = 128;                                          // pixels of a CTA block = MMA rows
constexpr int kATile = kM * 128;                                 // one A tile: 128 rows x 64 BF16
constexpr int kBChunk = 64 * 128;                                // 64 codebook rows x 64 BF16
constexpr int kBSlots = 2;
constexpr int kQMaxRows = 128;
constexpr int kAOff = 0;                                         // A [level] (3 x 16 KB)
constexpr int kBOff = kAOff + kLev * kATile;                     // B ring (2 x 8 KB)
constexpr int kQOff = kBOff + kBSlots * kBChunk;                 // one level's query matrix (<= 16 KB)
constexpr int kBoxBytes = 16 * 128;                              // F staging box: 16 pixels x 128 bytes
constexpr int kStgOff = kQOff + kQMaxRows * 128;                 // 4 warps x 2 boxes
constexpr int kBarOff = FC::kAccBytes + 256;                     // fused-phase barriers (after the splat's)
constexpr uint32_t kTmemCols = 256;                              // F buffers [0, 128), Y [128, 256)
static_assert(kStgOff + FC::kWarps * 2 * kBoxBytes <= FC::kAccBytes, "fused operands fit in the accumulator memory");
static_assert(kStgOff % 1024 == 0 && kQOff % 1024 == 0 && kBOff % 1024 == 0, "swizzled tiles are 1024-byte aligned");
static_assert(FC::kWarps == 4, "one consumer warp per TMEM lane quarter");

struct FusedArgs {
    int width, height, GX;
    const uint32_t* tile_ranges;
    const uint32_t* gauss_ids;
    const float* recs;
    float* final_T;
    uint32_t* n_last;
    int D;                       // features (multiple of 128, <= 512)
    const uint8_t* Bdec;         // [levels][D / 64][64 rows x 128 B] swizzled BF16 S^T
    int do_dec;                  // write F (through the tensor map)
    int Q, n_neg, Qp, npadq;     // Q = 0: no query
    float tau;
    const uint8_t* Bq;           // [levels][npadq rows x 128 B] swizzled BF16 [C | S t / |t|] (text-major)
    void* rel;                   // [Q][levels][P]
    int rel_bf16;
    int32_t* status;
    uint64_t wait_ns;            // bound of a wait on another warp's progress
};

struct FusedBars {
    uint64_t bfull[kBSlots], bempty[kBSlots], dfull[2], dempty[2], qfull, qempty, qload, qfree;
    uint32_t tslot;
};
static_assert(kBarOff + sizeof(FusedBars) <= FC::kFixedBytes, "fused barriers fit in the fixed area");

__global__ void __launch_bounds__(FC::kThreads, 2) fused_kernel(const __grid_constant__ CUtensorMap tmF, FusedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the swizzled operand tiles need 1024-byte alignment (1 KB of slack is requested)
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const SplatSmem<FC> sm(smem);
    FusedBars* fb = reinterpret_cast<FusedBars*>(smem + kBarOff);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x >> 1, sub = blockIdx.x & 1;
    const int x0 = (tile % a.GX) * kTW, y0 = (tile / a.GX) * kTH + sub * kHH;
    const size_t P = (size_t)a.width * a.height;
    const bool do_query = a.Q > 0, do_dec = a.do_dec != 0;
    const int nfc = a.D / 64;    // F chunks per level

    if (tid == 0) {
        sm.init();
        *sm.skip = a.status && *reinterpret_cast<volatile int32_t*>(a.status) == LSV2_ERR_TIMEOUT;
        for (int s = 0; s < kBSlots; ++s) {
            tc::mbar_init(tc::smem_u32(&fb->bfull[s]), 1);
            tc::mbar_init(tc::smem_u32(&fb->bempty[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(tc::smem_u32(&fb->dfull[s]), 1);
            tc::mbar_init(tc::smem_u32(&fb->dempty[s]), FC::kWarps);
        }
        tc::mbar_init(tc::smem_u32(&fb->qfull), 1);
        tc::mbar_init(tc::smem_u32(&fb->qempty), FC::kWarps);
        tc::mbar_init(tc::smem_u32(&fb->qload), 1);
        tc::mbar_init(tc::smem_u32(&fb->qfree), 1);
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&fb->tslot), kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = fb->tslot;
    const bool skip = *sm.skip;

    if (!skip) {
        // ---- splat: W stays in the consumer warps' shared-memory columns
        TileJob j{a.width, a.height, x0, y0, a.tile_ranges[2 * tile], a.tile_ranges[2 * tile + 1], a.gauss_ids,
                  a.recs, nullptr, a.final_T, a.n_last, a.status};
        j.wait_ns = a.wait_ns;
        (void)splat_tile<kLev, kKp, kTW, kHH, 0, false>(j, sm, 0u);
    }
    bool ok = !skip && !*reinterpret_cast<volatile int*>(sm.abort);
    // ---- transit: coefficients -> BF16 in this thread's TMEM lane, columns [32 l, 32 l + 32)
    const uint32_t lrow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    if (ok && warp < FC::kWarps) {
        const float* acc = sm.acc + warp * FC::kAccFloats;
#pragma unroll 1
        for (int l = 0; l < kLev; ++l) {
            uint32_t r[32];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                r[i] = tc::pack_bf16(acc[(l * 64 + 2 * i) * 33 + lane], acc[(l * 64 + 2 * i + 1) * 33 + lane]);
            tc::tmem_st32(lrow + (uint32_t)(l * 32), r);
        }
        tc::tmem_wait_st();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    // ---- TMEM -> swizzled A tiles in the freed accumulator memory, row = the pixel's row-major
    //      index in the 16x8 block; the producer starts the operand copies into the same memory
    if (ok && warp < FC::kWarps) {
        const int row = FC::lane_y(warp, lane) * kTW + FC::lane_x(warp, lane);
#pragma unroll 1
        for (int l = 0; l < kLev; ++l) {
            uint32_t r[32];
            tc::tmem_ld32(lrow + (uint32_t)(l * 32), r);
            tc::tmem_wait_ld();
            uint8_t* A = smem + kAOff + l * kATile;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                *reinterpret_cast<uint4*>(A + tc::sw128(row, 8 * c)) = make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
        }
    }
    const int nb = do_dec ? kLev * nfc : 0;   // B chunks per block
    if (ok && warp == FC::kWarps && lane == 0) {
        for (int g = 0; g < kBSlots && g < nb; ++g) {
            tc::bulk_load_arm(tc::smem_u32(&fb->bfull[g]), kBChunk);
            tc::bulk_load(tc::smem_u32(smem + kBOff + g * kBChunk), a.Bdec + (size_t)g * kBChunk, kBChunk,
                          tc::smem_u32(&fb->bfull[g]));
        }
        if (do_query) {
            const uint32_t qb = (uint32_t)a.npadq * 128;
            tc::bulk_load_arm(tc::smem_u32(&fb->qload), qb);
            tc::bulk_load(tc::smem_u32(smem + kQOff), a.Bq, qb, tc::smem_u32(&fb->qload));
        }
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    volatile int* abort_flag = sm.abort;
    if (ok && warp == FC::kWarps) {
        // ---- MMA issue (lane 0) and operand copies, in the epilogue's order
        const uint32_t idd = tc::idesc_bf16(kM, 64);
        int g = 0;            // F MMA groups issued
        int bc = 0;           // B chunks consumed
        int b_loaded = nb < kBSlots ? nb : kBSlots;   // B chunks whose copies were issued
        int q_loaded = do_query ? 1 : 0;              // query-matrix copies issued
        uint32_t last_bar = 0, last_par = 0;          // the latest MMA commit (it covers all earlier MMAs)
        const uint32_t qb = (uint32_t)a.npadq * 128;
        for (int l = 0; l < kLev && ok; ++l) {
            if (do_query) {
                if (warp_wait(&fb->qload, (uint32_t)(l & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone ||
                    (l > 0 && warp_wait(&fb->qempty, (uint32_t)((l - 1) & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    tc::fence_after();
                    const uint32_t a0 = tc::smem_u32(smem + kAOff + l * kATile), b0 = tc::smem_u32(smem + kQOff);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tc::mma_bf16(tmem + 128u, tc::desc_sw128(a0 + k * 32), tc::desc_sw128(b0 + k * 32),
                                     tc::idesc_bf16(kM, a.npadq), k > 0 ? 1u : 0u);
                    tc::mma_commit(tc::smem_u32(&fb->qfull));
                    tc::mma_commit(tc::smem_u32(&fb->qfree));
                }
                __syncwarp();
                last_bar = tc::smem_u32(&fb->qfree);   // level l's commit: phase l
                last_par = (uint32_t)(l & 1);
                if (l + 1 < kLev) {
                    // the next level's query matrix replaces this one once the MMA has read it
                    if (warp_wait(&fb->qfree, (uint32_t)(l & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone) { ok = false; break; }
                    if (lane == 0) {
                        tc::bulk_load_arm(tc::smem_u32(&fb->qload), qb);
                        tc::bulk_load(tc::smem_u32(smem + kQOff), a.Bq + (size_t)(l + 1) * qb, qb, tc::smem_u32(&fb->qload));
                    }
                    ++q_loaded;
                }
            }
            if (!do_dec) continue;
            for (int c = 0; c < nfc; ++c, ++bc, ++g) {
                const int s = bc % kBSlots, buf = g & 1;
                if (warp_wait(&fb->bfull[s], (uint32_t)((bc / kBSlots) & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone ||
                    (g >= 2 && warp_wait(&fb->dempty[buf], (uint32_t)(((g - 2) >> 1) & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    tc::fence_after();
                    const uint32_t a0 = tc::smem_u32(smem + kAOff + l * kATile), b0 = tc::smem_u32(smem + kBOff + s * kBChunk);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tc::mma_bf16(tmem + (uint32_t)(buf * 64), tc::desc_sw128(a0 + k * 32), tc::desc_sw128(b0 + k * 32),
                                     idd, k > 0 ? 1u : 0u);
                    tc::mma_commit(tc::smem_u32(&fb->dfull[buf]));
                    tc::mma_commit(tc::smem_u32(&fb->bempty[s]));
                }
                __syncwarp();
                last_bar = tc::smem_u32(&fb->dfull[buf]);   // group g is buffer buf's commit g / 2
                last_par = (uint32_t)((g >> 1) & 1);
                // refill this slot with chunk bc + kBSlots once the MMA has read it
                const int nxt = bc + kBSlots;
                if (nxt < nb) {
                    if (warp_wait(&fb->bempty[s], (uint32_t)((bc / kBSlots) & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        tc::bulk_load_arm(tc::smem_u32(&fb->bfull[s]), kBChunk);
                        tc::bulk_load(tc::smem_u32(smem + kBOff + s * kBChunk), a.Bdec + (size_t)nxt * kBChunk, kBChunk,
                                      tc::smem_u32(&fb->bfull[s]));
                    }
                    ++b_loaded;
                }
            }
        }
        if (!ok) {
            if (lane == 0) report(a.status, LSV2_ERR_TIMEOUT);
            *abort_flag = 1;
        }
        // Before the CTA frees TMEM and retires, the copies this warp issued must have landed and
        // its last MMA (hence every earlier one) completed: also when its own loop finished,
        // since an epilogue warp may have given up on an MMA that is still running.  On the
        // normal path these phases completed already.  Each wait is bounded by kDrainNs.
        for (int c = b_loaded > kBSlots ? b_loaded - kBSlots : 0; c < b_loaded; ++c)
            (void)tc::mbar_wait(tc::smem_u32(&fb->bfull[c % kBSlots]), (uint32_t)((c / kBSlots) & 1), kDrainNs);
        if (q_loaded > 0) (void)tc::mbar_wait(tc::smem_u32(&fb->qload), (uint32_t)((q_loaded - 1) & 1), kDrainNs);
        if (last_bar) (void)tc::mbar_wait(last_bar, last_par, kDrainNs);
    } else if (ok && warp < FC::kWarps) {
        // ---- epilogues: this warp owns MMA rows 32 q4 .. 32 q4 + 31 = image rows 2 q4, 2 q4 + 1
        const int q4 = warp, row = 32 * q4 + lane;
        const int gx = x0 + (row & 15), gy = y0 + (row >> 4);
        const bool in = gx < a.width && gy < a.height;
        const size_t pix = (size_t)gy * a.width + gx;
        const int per = 1 + a.n_neg;
        uint8_t* box = smem + kStgOff + (size_t)(q4 * 2 + (lane >> 4)) * kBoxBytes;   // this lane's image row
        const int br = lane & 15;                                                       // its row in the box
        int g = 0;
        for (int l = 0; l < kLev && ok; ++l) {
            if (do_query) {
                if (warp_wait(&fb->qfull, (uint32_t)(l & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone) { ok = false; break; }
                tc::fence_after();
                // |F|^2 = |W C|^2 (S S^T = C C^T): columns 0..63 of Y
                float n2;
                {
                    uint32_t ya[32], yb[32];
                    tc::tmem_ld32(lrow + 128u, ya);
                    tc::tmem_ld32(lrow + 128u + 32u, yb);
                    tc::tmem_wait_ld();
                    n2 = chol_norm2(ya, yb);
                }
                const float nf = sqrtf(fmaxf(n2, 0.0f));
                const float kneg = nf < 1e-12f ? 0.0f : -a.tau / nf;
                const int nch = a.Qp / 8;
                for (int c = 0; c < nch; ++c) {
                    const int q0 = c * 8;
                    uint32_t rp[8], rn[8];
                    tc::tmem_ld8(lrow + 128u + (uint32_t)(64 + q0), rp);
                    float best[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) best[e] = per > 1 ? -INFINITY : 0.0f;
                    for (int t = 1; t < per; ++t) {
                        tc::tmem_ld8(lrow + 128u + (uint32_t)(64 + t * a.Qp + q0), rn);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 8; ++e) best[e] = fmaxf(best[e], __uint_as_float(rn[e]));
                    }
                    tc::tmem_wait_ld();
                    if (in) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int q = q0 + e;
                            if (q < a.Q) {
                                const float d = __uint_as_float(rp[e]) - best[e];
                                const size_t o = ((size_t)q * kLev + l) * P + pix;
                                if (a.rel_bf16) {
                                    // as the tensor-core relevancy: sigmoid through the hardware tanh
                                    float th;
                                    asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(-0.5f * kneg * d));
                                    static_cast<__nv_bfloat16*>(a.rel)[o] = __float2bfloat16_rn(fmaf(0.5f, th, 0.5f));
                                } else {
                                    static_cast<float*>(a.rel)[o] = __fdividef(1.0f, 1.0f + __expf(kneg * d));
                                }
                            }
                        }
                    }
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_u32(&fb->qempty));
            }
            if (!do_dec) continue;
            for (int c = 0; c < nfc && ok; ++c, ++g) {
                const int buf = g & 1;
                if (warp_wait(&fb->dfull[buf], (uint32_t)((g >> 1) & 1), nullptr, 0, abort_flag, a.wait_ns) != kWaitDone) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                uint32_t r[32], r2[32];
                tc::tmem_ld32(lrow + (uint32_t)(buf * 64), r);
                tc::tmem_ld32(lrow + (uint32_t)(buf * 64 + 32), r2);
                tc::tmem_wait_ld();
                tc::fence_before();
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(tc::smem_u32(&fb->dempty[buf]));
                    tc::bulk_wait_read<0>();   // the previous chunk's boxes have been read
                }
                __syncwarp();
                // this lane's 64 features of the chunk -> row br of its image row's box (128-byte
                // swizzle: 16-byte chunk v at position v ^ (br % 8))
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    *reinterpret_cast<uint4*>(box + br * 128 + ((v ^ (br & 7)) << 4)) =
                        make_uint4(tc::pack_bf16(__uint_as_float(r[8 * v]), __uint_as_float(r[8 * v + 1])),
                                   tc::pack_bf16(__uint_as_float(r[8 * v + 2]), __uint_as_float(r[8 * v + 3])),
                                   tc::pack_bf16(__uint_as_float(r[8 * v + 4]), __uint_as_float(r[8 * v + 5])),
                                   tc::pack_bf16(__uint_as_float(r[8 * v + 6]), __uint_as_float(r[8 * v + 7])));
                    *reinterpret_cast<uint4*>(box + br * 128 + (((v + 4) ^ (br & 7)) << 4)) =
                        make_uint4(tc::pack_bf16(__uint_as_float(r2[8 * v]), __uint_as_float(r2[8 * v + 1])),
                                   tc::pack_bf16(__uint_as_float(r2[8 * v + 2]), __uint_as_float(r2[8 * v + 3])),
                                   tc::pack_bf16(__uint_as_float(r2[8 * v + 4]), __uint_as_float(r2[8 * v + 5])),
                                   tc::pack_bf16(__uint_as_float(r2[8 * v + 6]), __uint_as_float(r2[8 * v + 7])));
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    for (int hh = 0; hh < 2; ++hh) {
                        const int yy = y0 + 2 * q4 + hh;
                        if (yy < a.height)
                            tc::tma_store_4d(&tmF, c * 64, x0, yy, l, tc::smem_u32(smem + kStgOff + (q4 * 2 + hh) * kBoxBytes));
                    }
                    tc::bulk_commit();
                }
            }
        }
        if (lane == 0) tc::bulk_wait_all();
        if (!ok && lane == 0) report(a.status, LSV2_ERR_TIMEOUT);
    }
    // every MMA was waited on by an epilogue, or the issuer drained what it started
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// Operands of the fused kernel: the codebook S^T of every level as swizzled BF16 chunks of 64
// rows, and (with queries) the text-major [C | S t / |t|] rows (S S^T = C C^T).
__global__ void fused_prep_kernel(int levels, int D, const float* S, int Q, int n_neg, int Qp, int npadq,
                                  const float* Bt, const float* tnorm, uint8_t* Bdec, uint8_t* Bq)
{
    const int l = blockIdx.y;
    const int per = 1 + n_neg;
    const int n_dec = D * 64, n_q = Q > 0 ? npadq * 64 : 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_dec + n_q; i += gridDim.x * blockDim.x) {
        if (i < n_dec) {
            const int n = i >> 6, k = i & 63;      // row n of S^T = column n of S
            const float v = S[((size_t)l * 64 + k) * D + n];
            uint8_t* chunk = Bdec + ((size_t)l * (D / 64) + n / 64) * kBChunk;
            *reinterpret_cast<__nv_bfloat16*>(chunk + tc::sw128(n % 64, k)) = __float2bfloat16_rn(v);
        } else {
            const int i2 = i - n_dec, n = i2 >> 6, k = i2 & 63;
            int src = n < 64 ? n : -1;
            float scale = 1.0f;   // text rows S t / |t|, as the split relevancy
            if (n >= 64 && n < 64 + per * Qp) {
                const int t = (n - 64) / Qp, q = (n - 64) % Qp;
                src = q < Q ? 64 + q * per + t : -1;
                if (q < Q) scale = 1.0f / tnorm[q * per + t];
            }
            const float v = src >= 0 ? Bt[((size_t)l * (64 + Q * per) + src) * 64 + k] * scale : 0.0f;
            *reinterpret_cast<__nv_bfloat16*>(Bq + (size_t)l * npadq * 128 + tc::sw128(n, k)) = __float2bfloat16_rn(v);
        }
    }
}

int pad8(int q) { return (q + 7) / 8 * 8; }
int npadq_of(int Q, int n_neg) { return Q > 0 ? (64 + (1 + n_neg) * pad8(Q) + 15) / 16 * 16 : 0; }
size_t a256(size_t b) { return (b + 255) / 256 * 256; }

struct FusedLayout {
    size_t recs, bdec, qws, bq, bytes;
};

FusedLayout fused_layout(int64_t n, int levels, int K, int D, int Q, int n_neg)
{
    FusedLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o += a256(b);
        return at;
    };
    L.recs = take((size_t)n * splat_record_bytes(levels, K));
    L.bdec = take((size_t)levels * D * 128);
    const int nt = Q * (1 + n_neg);
    L.qws = take(Q > 0 ? query_workspace_bytes(levels, nt) : 0);
    L.bq = take((size_t)levels * npadq_of(Q, n_neg) * 128);
    L.bytes = o;
    return L;
}

}  // namespace

bool fused_supported(int levels, int K, int L, int D, int Q, int n_neg, int tw, int th)
{
    if (levels != kLev || K != kKp || L != 64 || tw != kTW || th != kTH) return false;
    if (D < 128 || D > 512 || D % 128 != 0) return false;
    if (Q < 0 || (Q > 0 && (n_neg < 1 || npadq_of(Q, n_neg) > kQMaxRows))) return false;   // Q <= 8 at n_neg = 4
    return true;
}

size_t fused_workspace_bytes(int64_t n, int levels, int K, int D, int Q, int n_neg)
{
    return fused_layout(n, levels, K, D, Q, n_neg).bytes;
}

cudaError_t launch_fused(const lsv2_camera& cam, int64_t n, const lsv2_proj& proj, const uint32_t* tile_ranges,
                         const uint32_t* gauss_ids, const uint8_t* idx, const float* w, const float* codebook, int D,
                         int Q, int n_neg, const float* text, float tau, void* ws, void* F, void* rel, bool rel_bf16,
                         float* final_T, uint32_t* n_last, int32_t* status, cudaStream_t stream)
{
    const FusedLayout Lo = fused_layout(n, kLev, kKp, D, Q, n_neg);
    char* base = static_cast<char*>(ws);
    PackArgs pa{n, kLev, kKp, splat_record_bytes(kLev, kKp), proj.xy, proj.axes, proj.conic_o, proj.extent, idx, w,
                reinterpret_cast<float*>(base + Lo.recs), status};
    cudaError_t e = launch_pack(pa, stream);
    if (e != cudaSuccess) return e;
    const int nt = Q * (1 + n_neg);
    if (Q > 0) {
        e = launch_query_prepare(kLev, D, nt, codebook, text, base + Lo.qws, stream);
        if (e != cudaSuccess) return e;
        e = launch_query_factor(kLev, nt, base + Lo.qws, stream);
        if (e != cudaSuccess) return e;
    }
    const int Qp = pad8(Q), npadq = npadq_of(Q, n_neg);
    fused_prep_kernel<<<dim3(64, kLev), 256, 0, stream>>>(kLev, D, codebook, Q, n_neg, Qp, npadq,
                                                          Q > 0 ? query_ws_bt(base + Lo.qws) : nullptr,
                                                          Q > 0 ? query_ws_tnorm(base + Lo.qws, kLev, nt) : nullptr,
                                                          reinterpret_cast<uint8_t*>(base + Lo.bdec),
                                                          reinterpret_cast<uint8_t*>(base + Lo.bq));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int GX = (cam.width + kTW - 1) / kTW, GY = (cam.height + kTH - 1) / kTH;
    if (GX * GY == 0) return cudaSuccess;
    // F [levels][H][W][D] BF16 in boxes of 64 features x 16 pixels of one image row
    CUtensorMap tmF;
    if (F) {
        if (!encode_tmap_4d(&tmF, F, true, (uint64_t)D, (uint64_t)cam.width, (uint64_t)cam.height, (uint64_t)kLev, 64u,
                            16u, false))
            return cudaErrorInvalidValue;
    } else {
        std::memset(&tmF, 0, sizeof(tmF));
    }
    FusedArgs a{};
    a.width = cam.width;
    a.height = cam.height;
    a.GX = GX;
    a.tile_ranges = tile_ranges;
    a.gauss_ids = gauss_ids;
    a.recs = reinterpret_cast<const float*>(base + Lo.recs);
    a.final_T = final_T;
    a.n_last = n_last;
    a.D = D;
    a.Bdec = reinterpret_cast<const uint8_t*>(base + Lo.bdec);
    a.do_dec = F != nullptr ? 1 : 0;
    a.Q = Q;
    a.n_neg = n_neg;
    a.Qp = Qp;
    a.npadq = npadq;
    a.tau = tau;
    a.Bq = reinterpret_cast<const uint8_t*>(base + Lo.bq);
    a.rel = rel;
    a.rel_bf16 = rel_bf16 ? 1 : 0;
    a.status = status;
    a.wait_ns = wait_limit_ns();
    constexpr int kSmem = FC::kSmemBytes + 1024;
    static_assert(2 * (kSmem + 1024) <= 233472, "two CTAs per SM");
    e = cudaFuncSetAttribute(fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    fused_kernel<<<GX * GY * 2, FC::kThreads, kSmem, stream>>>(tmF, a);
    return cudaGetLastError();
}

}  // namespace lsv2

using namespace lsv2;

extern "C" size_t lsv2_render_fused_workspace_bytes(int64_t n, int32_t levels, int32_t K, int32_t D, int32_t Q,
                                                   int32_t n_neg)
{
    if (n < 0 || !fused_supported(levels, K, 64, D, Q, n_neg, kTW, kTH)) return 0;
    return fused_workspace_bytes(n, levels, K, D, Q, n_neg);
}

extern "C" lsv2_status lsv2_render_fused(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                                         const uint32_t* tile_ranges, const uint32_t* gauss_ids, int32_t levels,
                                         int32_t K, int32_t L, const uint8_t* idx, const float* w,
                                         const float* codebook, int32_t D, int32_t Q, int32_t n_neg,
                                         const float* text, float tau, void* workspace, size_t workspace_bytes,
                                         void* feat, void* rel, lsv2_dtype rel_dtype, float* final_T,
                                         uint32_t* n_last, int32_t* dev_status, void* stream)
{
    if (!cam || cam->width <= 0 || cam->height <= 0 || n < 0 || !proj || !tile_ranges || !gauss_ids || !final_T ||
        !n_last || !codebook)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (!fused_supported(levels, K, L, D, Q, n_neg, cam->tile_w, cam->tile_h)) return LSV2_ERR_UNSUPPORTED;
    if (n > 0 && (!idx || !w || !proj->xy || !proj->axes || !proj->conic_o || !proj->extent))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (!feat && Q == 0) return LSV2_ERR_INVALID_ARGUMENT;
    if (Q > 0 && (!text || !rel || (rel_dtype != LSV2_F32 && rel_dtype != LSV2_BF16))) return LSV2_ERR_INVALID_ARGUMENT;
    if ((feat && (reinterpret_cast<uintptr_t>(feat) & 15u)) || (reinterpret_cast<uintptr_t>(codebook) & 15u) ||
        (text && (reinterpret_cast<uintptr_t>(text) & 15u)))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) ||
        workspace_bytes < fused_workspace_bytes(n, levels, K, D, Q, n_neg))
        return LSV2_ERR_INVALID_ARGUMENT;
    const cudaError_t e = launch_fused(*cam, n, *proj, tile_ranges, gauss_ids, idx, w, codebook, D, Q, n_neg, text, tau,
                                       workspace, feat, rel, rel_dtype == LSV2_BF16, final_T, n_last, dev_status,
                                       static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LSV2_OK : LSV2_ERR_CUDA;
}
