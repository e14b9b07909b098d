// splat.cuh -- record layout and launch configuration of the sparse-coefficient splat.
#pragma once

#include "device.cuh"

namespace lsv2 {

constexpr int kMaxPairs = 24;  // levels * K

// Per-Gaussian splat record (global memory, 16-byte aligned), P = levels * K pairs:
//   floats [0, 4)     u_hi, v_hi, u_lo, v_lo       2D mean as a float pair
//   floats [4, 8)     c_hi, s_hi, A, B             principal frame (see eval_power2)
//   floats [8, 12)    c_lo, s_lo, kappa, opacity
//   floats [12, 12+P) weights
//   words [12+P, 12+2P) byte offset of each pair's accumulator column in the splat's shared
//                     memory: (lev * L + idx) * 33 * 4 (a column spans 33 floats); the
//                     accumulator column is offset / 132
//   last 16 bytes     culling half-extents (ex, ey, 0, 0)
// Repeated indices of one level are merged into one pair; the emptied repeats and any invalid
// index (weight 0) point at the dummy column levels * L, which is accumulated but never
// written out.  So no two pairs of a record that carry weight share a column, and a record's
// pairs can all be loaded before any is stored, whatever order the stores land in.
__host__ __device__ constexpr int smem_record_bytes(int P) { return ((48 + 8 * P) + 15) / 16 * 16; }
__host__ __device__ constexpr int record_bytes(int P) { return smem_record_bytes(P) + 16; }
// Dense record (the non-sparse baseline: every level's 64 coefficients, zeros included):
//   floats [0, 12) as above, floats [12, 12 + 64 levels) dense coefficients, last 16 bytes extents.
__host__ __device__ constexpr int dense_record_bytes(int levels) { return ((48 + 256 * levels) + 15) / 16 * 16 + 16; }

// One CTA per tile: kWarps consumer warps (one pixel per lane, 32 pixels per warp) and one
// producer warp that gathers the tile's records, BATCH at a time, into a ring of kStages
// shared-memory stages with bulk async copies.  BATCH: 16 or 32 records per stage (0 = 32, or
// 16 for dense records).  DENSE: records carry all 64 coefficients of each level and every
// contributing Gaussian updates all 64 columns of each level (the blend without the sparse
// splatting, kept for comparison).
// TM: the last TM consumer warps keep their accumulators in tensor memory (TMEM) instead of
// shared memory (0 or 4, with 8 consumer warps): shared memory then holds the accumulators of
// only kWarps - TM warps, so a 16 x 16 tile of 8 consumer warps still fits twice per SM.
template <int LEVELS, int K, int TW, int TH, int BATCH = 0, bool DENSE = false, int LW = 64, int TM = 0>
struct SplatCfg {
    static constexpr int kPixels = TW * TH;
    static constexpr int kWarps = kPixels / 32;      // consumer warps
    static constexpr int kThreads = kPixels + 32;    // + the producer warp
    static constexpr int kPairs = LEVELS * K;        // pairs in a record
    static constexpr int kLW = LW;                   // codebook size L: accumulator columns per level
    static constexpr int kCols = LEVELS * LW;
    static constexpr int kAccFloats = ((kCols + 1) * 33 + 3) / 4 * 4;   // + the dummy column
    static constexpr int kTmemWarps = TM;
    static constexpr int kSmemAccWarps = kWarps - TM;
    static constexpr bool kDense = DENSE;
    static constexpr int kRecBytes = DENSE ? dense_record_bytes(LEVELS) : record_bytes(kPairs);
    static constexpr int kRecFloats = kRecBytes / 4;
    static constexpr int kBatch = BATCH != 0 ? BATCH : (DENSE ? 16 : 32);
    static constexpr int kAccBytes = kSmemAccWarps * kAccFloats * 4;
    static constexpr int kStageBytes = kBatch * (kRecBytes + 16);   // records + culling boxes
    static constexpr int kFixedBytes = kAccBytes + 512;             // + barriers and flags
    static constexpr int kStagesFit = (232448 - 64 - kFixedBytes) / kStageBytes;
    // 8 consumer warps: as many stages as fit (one CTA per SM); 4 warps: 2 stages, so two CTAs
    // share an SM; fewer warps: 4 stages
    static constexpr int kStages =
        TM > 0 ? 2 : (kWarps >= 8 ? (kStagesFit < 8 ? kStagesFit : 8) : (kWarps >= 4 ? 2 : 4));
    static constexpr int kSmemBytes = kFixedBytes + kStages * kStageBytes;
    // lane -> pixel: each consumer warp covers an 8 x 4 block of the TW x TH block (warps in
    // row-major order).  A square-ish block keeps more of a warp's lanes inside the footprints
    // that pass its culling test than a 16 x 2 or 32 x 1 strip.
    static constexpr int kWarpW = 8, kWarpH = 4, kWarpsX = TW / kWarpW;
    __host__ __device__ static constexpr int lane_x(int warp, int lane) { return (warp % kWarpsX) * kWarpW + lane % kWarpW; }
    __host__ __device__ static constexpr int lane_y(int warp, int lane) { return (warp / kWarpsX) * kWarpH + lane / kWarpW; }
    static_assert(kPixels % 32 == 0 && TW % 8 == 0 && TH % 4 == 0, "warps cover 8 x 4 blocks of a tile");
    static_assert(kPairs <= kMaxPairs, "pairs per record");
    static_assert(!DENSE || LW == 64, "dense records carry 64 coefficients per level");
    static_assert(LW % 8 == 0 && LW <= 256, "codebook size");
    static_assert(kRecBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
    static_assert(kStages >= 2, "at least two stages");
    // TMEM columns a CTA allocates: 256 (two CTAs per SM) when the accumulators and the dummy
    // column fit, else the SM's 512 (one CTA per SM)
    static constexpr uint32_t kTmemCols = kCols + 1 <= 256 ? 256u : 512u;
    static_assert(TM == 0 || (TM == 4 && kWarps == 8 && !DENSE && kCols + 1 <= 512),
                  "TMEM accumulators: warps 4-7 of 8, one lane quarter each, at most 512 columns");
};

struct PackArgs {
    int64_t n;
    int levels, K, rec_bytes;
    const float* xy;
    const float* axes;
    const float* conic_o;
    const float* extent;
    const uint8_t* idx;
    const float* w;
    float* recs;
    int32_t* status;
    int L = 64;                         // codebook size: column of pair (level, index) = level * L + index
};

struct SplatArgs {
    lsv2_camera cam;
    const uint32_t* tile_ranges;
    const uint32_t* gauss_ids;
    const float* recs;
    float* coeff;                       // [levels][P][64] F32, or BF16 when coeff_bf16
    float* final_T;
    uint32_t* n_last;
    int32_t* status;
    int coeff_bf16 = 0;                 // write the coefficient map rounded to BF16 (nearest even)
    int L = 64;                         // codebook size (columns per level of the map)
    uint64_t wait_ns = kDefaultWaitNs;  // bound of a wait on a stage barrier (set at launch)
};

constexpr int kMaxSplatViews = 64;

struct SplatView {
    int width, height, GX, tile_base;   // tile_base: first global tile id of this view
    size_t rec_off;                     // floats: start of this view's records
    size_t coeff_off;                   // elements: start of this view's coefficient map
    size_t pix_off;                     // start of this view's final_T / n_last
};

struct SplatViewsArgs {
    int V, total_tiles;
    SplatView view[kMaxSplatViews + 1];
    const uint32_t* tile_ranges;        // [total_tiles][2]
    const uint32_t* gauss_ids;
    const float* recs;
    float* coeff;
    float* final_T;
    uint32_t* n_last;
    uint32_t* queue;                    // work-queue counter (zeroed by the launcher)
    int32_t* status;
    int coeff_bf16 = 0;                 // coefficient maps in BF16
    uint64_t wait_ns = kDefaultWaitNs;  // bound of a wait on a stage barrier (set at launch)
};

bool splat_supported(int levels, int K, int L, int tw, int th);
// The dense-coefficient baseline: levels 1 or 3, 16 x 16 tiles.
bool splat_dense_supported(int levels, int L, int tw, int th);
int splat_dense_record_bytes(int levels);
cudaError_t launch_pack_dense(const PackArgs& a, cudaStream_t stream);
cudaError_t launch_splat_dense(int levels, const SplatArgs& a, cudaStream_t stream);
// batch: records staged per warp (16 or 32; 0 = default).
cudaError_t launch_splat_views(int levels, int K, int tw, int th, int batch, const SplatViewsArgs& a, int num_sms,
                               cudaStream_t stream);
int splat_record_bytes(int levels, int K);
// Packs records for V views: projection slot and record of (view v, Gaussian g) = v * n + g.
cudaError_t launch_pack(const PackArgs& a, cudaStream_t stream, int V = 1);
cudaError_t launch_splat(int levels, int K, const SplatArgs& a, cudaStream_t stream);

}  // namespace lsv2
