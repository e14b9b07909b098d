/*
 * lsv2.h -- C ABI of the B300 (sm_103a) sparse-coefficient Gaussian splatting library.
 *
 * The library implements the rendering and query path of LangSplatV2 (arXiv 2507.07136):
 * every 3D Gaussian carries, per semantic level, K (index, weight) pairs over an L-entry
 * codebook S of D-dim language features (Sec. 3.3, Eq. 5).  The path is
 *
 *   lsv2_project       Gaussians -> 2D means, conics, tile rectangles, depth keys
 *                      (Sec. 3.1, Eq. 1-2 and EWA projection)
 *   lsv2_bin_sort      per-tile lists ordered by depth ("ordered Gaussian points within a
 *                      tile", Eq. 3)
 *   lsv2_splat_coeffs  front-to-back alpha blending of only the K nonzero coefficients into
 *                      an L-dim coefficient map per pixel and level (Sec. 3.4, Algorithm 1;
 *                      weights e_i of Eq. 7)
 *   lsv2_decode        F = W S per level (Eq. 7)
 *   lsv2_query         relevancy of each pixel for text queries (Sec. 3.2), computed through
 *                      the linearity of Eq. 7 without materialising F
 *   lsv2_query_views   all of the above for many views and queries in one call
 *   lsv2_render_fused  splat + decode + query of one frame in one kernel (W stays on chip)
 *   lsv2_postprocess   mean filter, level selection, localisation point and segmentation mask
 *                      of relevancy maps (appendix "Evaluation Details")
 *   lsv2_mlp_decode    the MLP decoder of the decoder-based comparison path (LangSplat*,
 *                      Sec. 3.1, Table 1), which Eq. 7 replaces
 *   lsv2_splat_backward, lsv2_l1_decode_backward
 *                      gradients of an L1 feature loss (no counterpart in the paper, which
 *                      trains the field but does not describe its gradient)
 *
 * Conventions shared by every entry point:
 *   - All array pointers are DEVICE pointers owned by the caller, unless a parameter says
 *     otherwise.  The library never allocates device memory; scratch space is passed in as
 *     a workspace sized by the matching *_workspace_bytes query.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *     stream-ordered and asynchronous; no call synchronises the host.
 *   - Errors found on the host (null pointers, sizes, unsupported shapes) are returned
 *     immediately and nothing is launched.  Conditions found on the device are written to
 *     `*dev_status` (an int32 in device memory the caller zeroes): the first nonzero
 *     lsv2_status wins; kernels never trap, and every device-side wait is bounded
 *     (lsv2_set_wait_limit_ns).  LSV2_ERR_CUDA reports a launch error.
 *   - Pixel (i, j) is evaluated at image-plane point (i, j).  Images are row-major.
 *   - Constants of the 3DGS rasteriser the paper builds on: 0.3 px^2 dilation, screen
 *     radius ceil(3 sqrt(lambda_max)), guard band 1.3 tan(fov/2), alpha clamp 0.99,
 *     skip alpha < 1/255, stop before a Gaussian that would take T below 1e-4.  All
 *     thresholds are float32 values.
 */
#ifndef LSV2_H
#define LSV2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LSV2_ABI_VERSION 2

typedef enum {
    LSV2_OK = 0,
    LSV2_ERR_INVALID_ARGUMENT = 1,
    LSV2_ERR_UNSUPPORTED = 2,
    LSV2_ERR_CAPACITY = 3,  /* more Gaussian-tile instances than the caller's capacity */
    LSV2_ERR_CUDA = 4,      /* a CUDA launch or runtime call failed */
    LSV2_ERR_TIMEOUT = 5,   /* a bounded device-side wait ran out */
    LSV2_ERR_NONFINITE = 6
} lsv2_status;

typedef enum { LSV2_F32 = 0, LSV2_BF16 = 1 } lsv2_dtype;

/* Post-processing rule (appendix "Evaluation Details"): LERF, or the blended map and masked-mean
 * level rule of the 3D-OVS and Mip-NeRF360 evaluations. */
typedef enum { LSV2_POST_LERF = 0, LSV2_POST_BLENDED = 1 } lsv2_post_mode;

/* Pinhole camera.  World -> camera: t = R m + t0 (x right, y down, z forward).
 * Supported tiles: 16x16 (default), 8x8, 32x8. */
typedef struct {
    int32_t width, height;
    int32_t tile_w, tile_h;
    float fx, fy, cx, cy;
    float near_z;
    float R[9]; /* row-major */
    float t[3];
} lsv2_camera;

/* Per-Gaussian outputs of lsv2_project (device arrays of n entries each, caller-owned).
 *   xy       float[n][4]  2D mean as an unevaluated float pair: u = u_hi + u_lo,
 *                         v = v_hi + v_lo, stored (u_hi, v_hi, u_lo, v_lo)
 *   conic_o  float[n][4]  (a, b, c, opacity); [[a, b], [b, c]] is the inverse of the
 *                         dilated 2D covariance
 *   extent   float[n][2]  half-widths (px) of the bounding box of the ellipse on which
 *                         alpha >= 1/255; negative when no pixel can reach 1/255
 *   depth    float[n]     depth key (camera-space z)
 *   radius   int32[n]     screen radius, ceil(3 sqrt(lambda_max))
 *   rect     int32[n][4]  tile rectangle x0, y0, x1, y1 (max exclusive)
 *   tiles_touched uint32[n]  (x1 - x0) (y1 - y0), 0 when not visible
 *   flags    uint8[n]     bit0 visible, bit1 near-degenerate (FP64 decisions)
 *   axes     float[n][8]  principal frame of the conic, used to evaluate the Gaussian:
 *                         (c_hi, s_hi, A, B, c_lo, s_lo, kappa, 0) where (c, s) = (c_hi + c_lo,
 *                         s_hi + s_lo) is the unit stiff axis (largest conic eigenvalue q1),
 *                         A = -q1 log2(e) / 2, B = -q2 log2(e) / 2 (q2 the smallest), kappa =
 *                         q1 / q2; power * log2(e) = A (e_stiff . d)^2 + B (e_soft . d)^2
 * All arrays must be 16-byte aligned. */
typedef struct {
    float* xy;
    float* conic_o;
    float* extent;
    float* depth;
    int32_t* radius;
    int32_t* rect;
    uint32_t* tiles_touched;
    uint8_t* flags;
    float* axes;
} lsv2_proj;

int32_t lsv2_abi_version(void);
const char* lsv2_status_string(lsv2_status s);

/* Bound of the device-side waits of the pipelined kernels (the splats, the tensor-core decode and
 * relevancy, the fused render, and the many-view call): a wait on another warp's progress (a
 * pipeline stage, a tensor-core accumulator) that is still unfinished `ns` nanoseconds after it
 * began gives up, the kernel records LSV2_ERR_TIMEOUT in *dev_status, lets the copies and MMAs it
 * issued complete (bounded by 100 ms), frees its tensor memory and returns; later CTAs of the
 * splat see the status and skip their tiles.  0 gives up at the first unsuccessful check (used by
 * tests to drive this path).  Default 1,000,000,000 (1 s).  The value is read when a call
 * launches its kernels (a call captured in a CUDA graph keeps the value of its capture); it is
 * process-wide, not per device or stream.  The paper has no counterpart: this is the library's
 * failure detection (a wait never spins without bound, a kernel never traps). */
void lsv2_set_wait_limit_ns(uint64_t ns);
uint64_t lsv2_wait_limit_ns(void);

/* Project n Gaussians (Sec. 3.1, Eq. 1-2, EWA splatting).
 * means float[n][3], scales float[n][3] (activated, > 0), quats float[n][4] (w, x, y, z;
 * normalised inside; a zero quaternion culls the Gaussian), opacity float[n] (activated).
 * Integer outputs follow a fixed FP32 decision specification (correctly rounded operations
 * in a fixed order); Gaussians whose undilated 2D covariance has condition number above
 * ~1e6 take the covariance and depth-key decisions in FP64.  2D means and conics are
 * evaluated in double-float arithmetic so the FP32 blend downstream is not limited by
 * their rounding. */
lsv2_status lsv2_project(const lsv2_camera* cam, int64_t n, const float* means,
                         const float* scales, const float* quats, const float* opacity,
                         const lsv2_proj* out, int32_t* dev_status, void* stream);

/* Workspace for lsv2_bin_sort: per-block tile histograms, tile counters and two key buffers of
 * `capacity` entries. */
size_t lsv2_bin_sort_workspace_bytes(int64_t n, int64_t capacity, int32_t num_tiles);

/* Bin and depth-sort (Eq. 3's ordered per-tile lists).  One instance per (visible Gaussian,
 * tile in its rect), ordered by (tile id = ty * GX + tx, depth key bits, Gaussian id).
 *   gauss_ids   uint32[capacity]      Gaussian id per instance, tile-major
 *   tile_ranges uint32[num_tiles][2]  [start, end) into gauss_ids
 *   dev_num_instances int64 (device)  total instance count I (may exceed capacity)
 * If I > capacity, *dev_status = LSV2_ERR_CAPACITY and the lists are truncated (all ranges
 * stay inside [0, capacity)).  At most 57,344 tiles per view. */
lsv2_status lsv2_bin_sort(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                          void* workspace, size_t workspace_bytes, uint32_t* gauss_ids,
                          int64_t capacity, uint32_t* tile_ranges, int64_t* dev_num_instances,
                          int32_t* dev_status, void* stream);

/* Workspace for lsv2_splat_coeffs: one packed splat record per Gaussian. */
size_t lsv2_splat_workspace_bytes(int64_t n, int32_t levels, int32_t K);

/* Sparse-coefficient splatting (Sec. 3.4, Algorithm 1): per pixel, front to back over its
 * tile's list, W_lev[idx_k] += w_k alpha_i T_i for the K pairs of every level.
 *   idx   uint8[n][levels][K]  codebook indices (< L; repeats are allowed and add up;
 *                              an index >= L sets LSV2_ERR_INVALID_ARGUMENT and is ignored)
 *   w     float[n][levels][K]
 *   coeff float[levels][H*W][L]  output coefficient map W (pixel-major, L contiguous)
 *   final_T float[H*W], n_last uint32[H*W]: transmittance after the last contributor and
 *   the list position (+1, relative to the tile start) of that contributor (0: none).
 * Blending is FP32.  Supported: L = 64 with levels 1 and K in {2, 4, 6, 8}, levels 2 and K = 4,
 * levels 3 and K = 4 (any tile) or K in {2, 6, 8} (16x16 tiles); tiles 16x16, 8x8, 32x8.  Also
 * L in {32, 128} with levels 3, K = 4 and 16x16 tiles (the codebook-size sweep), and L = 8 with
 * levels 3, K = 4 and 16x16 tiles: a dense low-dimensional feature splat (the latent of the
 * decoder-based comparison path, lsv2_mlp_decode) as pairs with indices 0..3. */
lsv2_status lsv2_splat_coeffs(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                              const uint32_t* tile_ranges, const uint32_t* gauss_ids,
                              int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                              const float* w, void* workspace, size_t workspace_bytes,
                              float* coeff, float* final_T, uint32_t* n_last,
                              int32_t* dev_status, void* stream);

/* lsv2_splat_coeffs with the coefficient map written as BF16 (round to nearest even of the FP32
 * blend; 16-byte aligned).  The tensor-core decode and relevancy round W to BF16 before their
 * products, so feeding them this map gives results bit-equal to feeding them the FP32 map, at
 * half the map's bytes.  Other arguments and outputs as for lsv2_splat_coeffs. */
lsv2_status lsv2_splat_coeffs_bf16(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                                   const uint32_t* tile_ranges, const uint32_t* gauss_ids,
                                   int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                                   const float* w, void* workspace, size_t workspace_bytes,
                                   void* coeff_bf16, float* final_T, uint32_t* n_last,
                                   int32_t* dev_status, void* stream);

/* Size of the fixed device scratch used by lsv2_splat_coeffs_noalloc (held on every device
 * that loads this library, until the process exits). */
#define LSV2_SPLAT_NOALLOC_SCRATCH_BYTES (8u << 20)

/* lsv2_splat_coeffs for callers that cannot allocate device memory.  The paper has no
 * counterpart; it exists because some callers cannot call cudaMalloc or provide a workspace
 * (a render loop with a fixed memory budget, a runtime that owns all device memory and only
 * exposes input and output buffers, a host without an allocator of its own).  Same arguments,
 * layouts and results as lsv2_splat_coeffs, minus the workspace: the per-Gaussian scratch
 * lives in a file-scope device array of LSV2_SPLAT_NOALLOC_SCRATCH_BYTES.
 *   - Limit: lsv2_splat_workspace_bytes(n, levels, K) must not exceed
 *     LSV2_SPLAT_NOALLOC_SCRATCH_BYTES (8 MiB: 52,428 Gaussians at 3 levels, K = 4);
 *     larger calls return LSV2_ERR_CAPACITY and launch nothing.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.  The address
 *     is kept for the life of the process, so do not call this after cudaDeviceReset on that
 *     device (the reset reloads the module and the kept address would be stale).
 *   - Nothing in the scratch must start at zero (every record is rewritten before use).
 *   - All calls share the one array: calls that overlap on the GPU (e.g. on two streams)
 *     race on it and must be serialised by the caller.
 *   - Allocates nothing and calls no allocating routine. */
lsv2_status lsv2_splat_coeffs_noalloc(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                                      const uint32_t* tile_ranges, const uint32_t* gauss_ids,
                                      int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                                      const float* w, float* coeff, float* final_T,
                                      uint32_t* n_last, int32_t* dev_status, void* stream);

/* Decode (Eq. 7): feat[lev][p][:] = coeff[lev][p][:] . codebook[lev].
 *   coeff    [levels][P][L]  dtype coeff_dtype (F32 or BF16)
 *   codebook [levels][L][D]  dtype codebook_dtype (F32 or BF16)
 *   feat     [levels][P][D]  dtype out_dtype (F32 or BF16)
 * All three F32: FP32 FMA on the CUDA cores.  Any BF16 among them: tensor cores (tcgen05),
 * with both operands rounded to BF16 and FP32 accumulation.  L = 64, D % 128 == 0 (tensor
 * cores: D <= 512).  A bounded device wait that expires sets LSV2_ERR_TIMEOUT. */
lsv2_status lsv2_decode(int32_t levels, int64_t P, int32_t L, int32_t D, const void* coeff,
                        lsv2_dtype coeff_dtype, const void* codebook, lsv2_dtype codebook_dtype,
                        void* feat, lsv2_dtype out_dtype, int32_t* dev_status, void* stream);

/* Workspace for lsv2_query.  After a call it holds, from its start, float B^T[levels][64 + Q (1 +
 * n_neg)][64]: per level 64 rows of G = S S^T (compute F32) or of C^T (compute BF16: G = C C^T, C
 * lower triangular), then the rows S t of the texts in query-major order; then the text norms. */
size_t lsv2_query_workspace_bytes(int32_t levels, int32_t L, int32_t Q, int32_t n_neg);

/* Relevancy (Sec. 3.2) through the linearity of Eq. 7: with u_t = S t and G = S S^T,
 *   <F, t> = W . u_t,  |F|^2 = W^T G W,  cos_t = <F, t> / (|F| |t|)  (0 when |F| < 1e-12)
 *   rel[q][lev][p] = min_i softmax(tau [cos_pos, cos_neg_i])_0
 *                  = sigmoid(tau (cos_pos - max_i cos_neg_i))
 *   coeff    [levels][P][L], dtype coeff_dtype: F32, or BF16 with compute_dtype BF16
 *   codebook float[levels][L][D]
 *   text     float[Q][1 + n_neg][D]  (positive first)
 *   rel      [Q][levels][P]  dtype rel_dtype (F32 or BF16)
 * compute_dtype F32: FP32 FMA on CUDA cores (rel_dtype F32).  BF16: tcgen05 tensor cores with
 * W and [C | u] rounded to BF16 and FP32 accumulation, |F|^2 = |W C|^2 where G = C C^T (Cholesky in
 * FP32; a pivot below 1e-5 of its diagonal entry, a codebook row within about 3e-3 of its length
 * of the span of the rows before it, gives a zero column).  S S^T and S t are formed per call in
 * twice-FP32 precision (error-free products and sums) and rounded to FP32.  L = 64, D % 4 == 0,
 * n_neg >= 1; BF16: 64 + (1 + n_neg) * 8 * ceil(Q / 8) <= 512 (Q <= 88 at n_neg = 4);
 * F32: Q (1 + n_neg) <= 512.  All arrays 16-byte aligned.
 * A bounded device wait that expires sets LSV2_ERR_TIMEOUT. */
lsv2_status lsv2_query(int32_t levels, int64_t P, int32_t L, int32_t D, const void* coeff,
                       lsv2_dtype coeff_dtype, const float* codebook, int32_t Q, int32_t n_neg,
                       const float* text, float tau, void* workspace, size_t workspace_bytes,
                       void* rel, lsv2_dtype rel_dtype, lsv2_dtype compute_dtype,
                       int32_t* dev_status, void* stream);

/* The two halves of lsv2_query, for callers that prepare the query operands ahead of the map
 * (e.g. on a second stream while the frame renders): lsv2_query_prepare forms, in the workspace,
 * B^T and the text norms from the codebook and the texts (and, for compute_dtype BF16, the factor
 * C of S S^T); lsv2_query_prepared then computes the relevancy of a coefficient map from that
 * workspace.  lsv2_query_prepare + lsv2_query_prepared on one stream is lsv2_query, bit for bit.
 * The workspace must stay untouched in between, and the prepared call must use the same levels,
 * Q, n_neg and compute_dtype.  Arguments as for lsv2_query. */
lsv2_status lsv2_query_prepare(int32_t levels, int32_t L, int32_t D, const float* codebook,
                               int32_t Q, int32_t n_neg, const float* text,
                               lsv2_dtype compute_dtype, void* workspace, size_t workspace_bytes,
                               void* stream);
lsv2_status lsv2_query_prepared(int32_t levels, int64_t P, int32_t L, const void* coeff,
                                lsv2_dtype coeff_dtype, int32_t Q, int32_t n_neg, float tau,
                                const void* workspace, size_t workspace_bytes, void* rel,
                                lsv2_dtype rel_dtype, lsv2_dtype compute_dtype,
                                int32_t* dev_status, void* stream);

/* Workspace for lsv2_query_views (projections, lists, records and coefficient maps of all
 * views, the query matrices and a work-queue counter). */
size_t lsv2_query_views_workspace_bytes(int32_t V, const lsv2_camera* cams, int64_t n,
                                        int32_t levels, int32_t K, int64_t capacity, int32_t Q,
                                        int32_t n_neg);

/* Relevancy of Q text queries in V views of one scene in one call (Sec. 3.2 through Eq. 7, with
 * the rendering of Sec. 3.4): project all views, bin and depth-sort the tiles of all views
 * together, splat with a persistent kernel that takes (view, tile) work items from an atomic
 * queue, then the tensor-core relevancy over all pixels of all views.  The same results as V
 * separate lsv2_project / lsv2_bin_sort / lsv2_splat_coeffs / lsv2_query (BF16) calls.
 *   cams     HOST array of V cameras (views may differ in resolution; one tile shape for all)
 *   means..w as for lsv2_project / lsv2_splat_coeffs (device); codebook float[levels][64][D]
 *   text     float[Q][1 + n_neg][D]; tau as for lsv2_query
 *   capacity instance capacity over all views (LSV2_ERR_CAPACITY in *dev_status if exceeded)
 *   stage_batch  Gaussian records per stage of the splat's shared-memory ring (gathered by one
 *            producer warp per tile): 16, 32 or 0 (= 32); tuned together with the tile shape
 *   rel      views concatenated, view v: [Q][levels][H_v W_v], dtype rel_dtype (F32 or BF16)
 *   dev_num_instances  int64 (device): total instances over all views
 * Everything is stream-ordered with no host synchronisation (capturable in a CUDA graph).
 * Supported: V <= 64, K = 4, L = 64, 64 + (1 + n_neg) * 8 * ceil(Q / 8) <= 512, workspace 256-byte
 * aligned. */
lsv2_status lsv2_query_views(int32_t V, const lsv2_camera* cams, int64_t n, const float* means,
                             const float* scales, const float* quats, const float* opacity,
                             int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                             const float* w, const float* codebook, int32_t D, int32_t Q,
                             int32_t n_neg, const float* text, float tau, int64_t capacity,
                             int32_t stage_batch, void* workspace, size_t workspace_bytes, void* rel,
                             lsv2_dtype rel_dtype, int64_t* dev_num_instances,
                             int32_t* dev_status, void* stream);

/* Workspace for lsv2_splat_coeffs_dense (one dense record per Gaussian). 0 if unsupported. */
size_t lsv2_splat_dense_workspace_bytes(int64_t n, int32_t levels);

/* The blend of lsv2_splat_coeffs WITHOUT the sparse splatting of Sec. 3.4: every Gaussian
 * carries its full 64-entry coefficient vector per level (the K pairs scattered, zeros
 * elsewhere) and every contributing Gaussian updates all 64 coefficients of every level -- the
 * "Sparse, not Efficient" configuration of the paper's speed ablation (Table 9), kept to measure
 * what the sparse splatting saves.  Blending zeros does not alter the result (Sec. 3.4), so the
 * outputs equal lsv2_splat_coeffs' bit for bit.  Arguments as for lsv2_splat_coeffs;
 * workspace lsv2_splat_dense_workspace_bytes(n, levels).  Supported: levels 1 or 3, L = 64,
 * 16 x 16 tiles. */
lsv2_status lsv2_splat_coeffs_dense(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                                    const uint32_t* tile_ranges, const uint32_t* gauss_ids,
                                    int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                                    const float* w, void* workspace, size_t workspace_bytes,
                                    float* coeff, float* final_T, uint32_t* n_last,
                                    int32_t* dev_status, void* stream);

/* Workspace for lsv2_render_fused (per-Gaussian records, the BF16 codebook and query operands).
 * 0 for an unsupported configuration. */
size_t lsv2_render_fused_workspace_bytes(int64_t n, int32_t levels, int32_t K, int32_t D, int32_t Q,
                                         int32_t n_neg);

/* The splat of lsv2_splat_coeffs (Sec. 3.4, Algorithm 1), the decode of lsv2_decode (Eq. 7,
 * BF16 operands and output, FP32 accumulation) and the relevancy of lsv2_query (Sec. 3.2 through
 * Eq. 7, BF16 compute) in one kernel, one CTA per 16 x 8 half of each tile and two per SM (one's
 * decode overlaps the other's splat): the coefficient map W stays in shared memory and tensor
 * memory and is never written to HBM.  F and rel equal what lsv2_splat_coeffs followed by
 * lsv2_decode (BF16) and lsv2_query (BF16 compute) produce.
 *   cam, n, proj, tile_ranges, gauss_ids, idx, w   as for lsv2_splat_coeffs (tile 16 x 16)
 *   codebook  float[levels][64][D], D a multiple of 128, <= 512
 *   Q, n_neg, text, tau   as for lsv2_query; Q = 0: no relevancy
 *   feat      BF16 [levels][P][D] (16-byte aligned), or NULL to skip the decode
 *   rel       [Q][levels][P], dtype rel_dtype (F32 or BF16); unused when Q = 0
 *   final_T, n_last   as for lsv2_splat_coeffs
 *   workspace lsv2_render_fused_workspace_bytes(...) bytes, 256-byte aligned
 * Supported: levels = 3, K = 4, L = 64, 64 + (1 + n_neg) * 8 * ceil(Q / 8) <= 128 (Q <= 8 at
 * n_neg = 4).  At least one of feat and Q > 0.  A bounded device wait that expires sets
 * LSV2_ERR_TIMEOUT. */
lsv2_status lsv2_render_fused(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                              const uint32_t* tile_ranges, const uint32_t* gauss_ids, int32_t levels,
                              int32_t K, int32_t L, const uint8_t* idx, const float* w,
                              const float* codebook, int32_t D, int32_t Q, int32_t n_neg,
                              const float* text, float tau, void* workspace, size_t workspace_bytes,
                              void* feat, void* rel, lsv2_dtype rel_dtype, float* final_T,
                              uint32_t* n_last, int32_t* dev_status, void* stream);

/* Sparse coefficients (Sec. 3.3): each Gaussian's L-dim parameter of a level is normalised by a
 * softmax, its K largest values are kept as the nonzeros and renormalised by their sum.
 *   rows     number of rows (Gaussians x levels), row-major [rows][L]
 *   logits   float[rows][L]
 *   idx      uint8_t[rows][K] out: the kept entries, those with the K largest logits (the
 *            softmax is monotone), in descending order of value, the lower index first among
 *            equal logits (the idx input of lsv2_splat_coeffs)
 *   w        float[rows][K] out: the renormalised weights (= softmax over the kept logits)
 * Supported: L in {16, 32, 64, 128, 256}, K in {1, 2, 4, 8}, K <= L.  K = 4 needs w 16-byte and
 * idx 4-byte aligned.  No workspace. */
lsv2_status lsv2_sparsify(int64_t rows, int32_t L, int32_t K, const float* logits, uint8_t* idx, float* w,
                          void* stream);

/* Gradient of lsv2_sparsify's weights with respect to the logits, the selection held fixed (it
 * is piecewise constant): dlogits[r][c] = 0 for a dropped entry c, and for kept entry k
 * (c = idx[r][k]) w_k (dw_k - sum_m w_m dw_m).
 *   idx, w   lsv2_sparsify's outputs;  dw  float[rows][K] (dLoss/dw)
 *   dlogits  float[rows][L] out (every entry written) */
lsv2_status lsv2_sparsify_backward(int64_t rows, int32_t L, int32_t K, const uint8_t* idx, const float* w,
                                   const float* dw, float* dlogits, void* stream);

/* Workspace for lsv2_postprocess: per (query, level) statistics (Q * levels * 32 bytes,
 * rounded up to 256).  0 for invalid sizes. */
size_t lsv2_postprocess_workspace_bytes(int32_t Q, int32_t levels);

/* Post-processing of relevancy maps (paper appendix, "Evaluation Details"; Sec. 3.2 on running
 * it on the GPU).  For each query q and level l, with M the map rel[q][l] (H x W, row-major):
 *   Avg(M)  mean over the in-image part of the k x k window centred on each pixel (k odd)
 *   S       mode LSV2_POST_LERF: Avg(M);  mode LSV2_POST_BLENDED: 0.5 (M + Avg(M))
 *   mask_l  (S - min S) / (max S - min S) > threshold (all 0 when max S = min S)
 *   level   LERF: the level whose S has the highest value; BLENDED: the level with the highest
 *           mean of S over mask_l (an empty mask ranks lowest); the lowest level on a tie
 *   point   (x, y) of the first pixel in row-major order where S of the selected level is
 *           maximal; score = that maximum
 * Arguments:
 *   rel        [Q][levels][H*W], dtype rel_dtype (F32 or BF16), e.g. the output of lsv2_query
 *   k          window, odd, 1..63;  threshold in [0, 1]
 *   workspace  lsv2_postprocess_workspace_bytes(Q, levels) bytes, 16-byte aligned
 *   smoothed   float[Q][levels][H*W] (written: S of every level)
 *   point      int32[Q][2], level int32[Q], score float[Q] (written)
 *   mask       uint8[Q][H*W]: mask of the selected level (written), or NULL to skip it
 * Supported: levels <= 8, H * W < 2^32.  dev_status is unused (no device-detected condition).
 * Stream-ordered, no host synchronisation (capturable in a CUDA graph). */
lsv2_status lsv2_postprocess(int32_t Q, int32_t levels, int32_t H, int32_t W, const void* rel,
                             lsv2_dtype rel_dtype, int32_t k, int32_t mode, float threshold,
                             void* workspace, size_t workspace_bytes, float* smoothed,
                             int32_t* point, int32_t* level, float* score, uint8_t* mask,
                             int32_t* dev_status, void* stream);

/* Backward of Loss = mean_{lev,p,d} |F - target| with F = W S (Eq. 7's decode; the L1 loss and its
 * adjoint have no counterpart in the paper, which trains the field without stating a gradient):
 *   G = sign(F - target) / (levels P D)  (sign(0) = 0),  dLoss/dW = G S^T,  dLoss/dS = W^T G.
 *   coeff     float[levels][P][L]   W
 *   codebook  float[levels][L][D]   S
 *   target    float[levels][P][D]
 *   loss      float (device scalar, accumulated: zero it first)
 *   dcoeff    float[levels][P][L]   dLoss/dW  (overwritten)
 *   dcodebook float[levels][L][D]   dLoss/dS  (accumulated: zero it first)
 * F is recomputed, not read or stored.  The three products run on the tensor cores with W and S
 * split into BF16 high and low parts (FP32 accumulation): dW and dS within about 4e-6 of the exact
 * products relative to sum |G| |S| and sum |W| |G|; every sign is the sign of the exact F - target
 * (elements whose tensor-core F lies within its error bound of the target are recomputed in FP64).
 * L = 64, D a multiple of 128 up to 512, P < 2^31 - 256, all arrays 16-byte aligned.  A bounded
 * device wait that expires sets LSV2_ERR_TIMEOUT in *dev_status (may be NULL). */
lsv2_status lsv2_l1_decode_backward(int32_t levels, int64_t P, int32_t L, int32_t D,
                                    const float* coeff, const float* codebook,
                                    const float* target, float* loss, float* dcoeff,
                                    float* dcodebook, int32_t* dev_status, void* stream);

/* Workspace for lsv2_splat_backward: per-Gaussian 2D-mean and conic gradients. */
size_t lsv2_splat_backward_workspace_bytes(int64_t n);

/* Backward of lsv2_splat_coeffs and lsv2_project.  Given dLoss/dW (dcoeff, same layout as
 * coeff), walks each pixel's list back to front from n_last, recomputing the transmittance
 * from final_T (T_i = T_{i+1} / (1 - alpha_i)), and accumulates per Gaussian:
 *   dw float[n][levels][K], dopacity float[n], dmeans float[n][3], dscales float[n][3],
 *   dquats float[n][4] (gradient w.r.t. the raw, unnormalised quaternion).
 * All five outputs are accumulated with atomics: zero them first. */
lsv2_status lsv2_splat_backward(const lsv2_camera* cam, int64_t n, const float* means,
                                const float* scales, const float* quats, const lsv2_proj* proj,
                                const uint32_t* tile_ranges, const uint32_t* gauss_ids,
                                int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                                const float* w, const float* final_T, const uint32_t* n_last,
                                const float* dcoeff, void* workspace, size_t workspace_bytes,
                                float* dw, float* dopacity, float* dmeans, float* dscales,
                                float* dquats, int32_t* dev_status, void* stream);

/* block_rows value of lsv2_mlp_decode that selects the fused tensor-core kernel. */
#define LSV2_MLP_FUSED (-1)

/* Workspace for lsv2_mlp_decode (0 for invalid arguments, or for LSV2_MLP_FUSED with widths the
 * fused kernel does not take).  block_rows >= 0: two activation buffers of one row block at the
 * widest hidden layer, a BF16 copy of an F32 input block, and 32 MiB for the library GEMM's own
 * scratch.  LSV2_MLP_FUSED: the packed weights only (under 2 MiB for any row count). */
size_t lsv2_mlp_decode_workspace_bytes(int64_t rows, int32_t n_layers, const int32_t* widths,
                                       int32_t x_dtype, int64_t block_rows);

/* The decoder of the decoder-based comparison path (LangSplat*, Sec. 3.1: the latent feature
 * rendered by Eq. 4 is decoded to the D-dim CLIP space by the MLP g_d; Table 1 times it as the
 * dominant stage).  Not part of LangSplatV2's own path, which replaces g_d by Eq. 7.
 * For every row r:  h_0 = x[r];  h_{l+1} = relu(h_l W_l + b_l)  (l < n_layers - 1);
 *                   y[r] = h_{n_layers-1} W_{n_layers-1} + b_{n_layers-1}.
 *   widths   int32[n_layers + 1], HOST memory: w_0 (input) .. w_n (output); each a multiple of
 *            8 in [8, 4096] (pad a narrower input with zero columns and zero weight rows)
 *   x        [rows][w_0]  dtype x_dtype (F32, rounded to BF16 as it is read; or BF16)
 *   weights  bf16, the W_l one after another, each row-major [w_l][w_{l+1}]
 *   biases   bf16, the b_l one after another, each [w_{l+1}]
 *   y        bf16 [rows][w_n]
 * BF16 operands, FP32 accumulation, bias (+ ReLU) applied to the FP32 sum, every layer's output
 * rounded to BF16.  Two implementations, chosen by block_rows:
 *   >= 0             each layer a library GEMM (cuBLASLt) with a fused bias (+ ReLU) epilogue,
 *                    rows in blocks of block_rows (a multiple of 128; 0 = 1,048,576), which bounds
 *                    the intermediate activation buffers.  The faster of the two on B300 at the
 *                    workload's widths (it streams every activation through HBM, but at full
 *                    bandwidth).
 *   LSV2_MLP_FUSED   one persistent tcgen05 kernel, the hidden activations kept on chip, the
 *                    weights repacked into the workspace on every call; for w_0 <= 32, hidden
 *                    widths that are multiples of 16 up to 256 and an output width that is a
 *                    multiple of 16 (at most 16 products of <= 256 outputs, at most 4,800 biases),
 *                    else LSV2_ERR_UNSUPPORTED.  A workspace under 2 MiB instead of about 1 GiB.
 * All pointers 16-byte aligned.  Returns LSV2_ERR_UNSUPPORTED for a width outside the rule,
 * LSV2_ERR_CUDA if a launch fails or a GEMM cannot be planned.  A device wait of the fused
 * kernel that runs out (lsv2_set_wait_limit_ns) records LSV2_ERR_TIMEOUT in *dev_status (may
 * be NULL; the library path does not use it).  Allocates nothing; capturable in a CUDA graph
 * (the library path after one uncaptured call of the same shapes: its first call of a shape
 * asks the library's heuristic for an algorithm on the host). */
lsv2_status lsv2_mlp_decode(int64_t rows, int32_t n_layers, const int32_t* widths, const void* x,
                            int32_t x_dtype, const void* weights, const void* biases, void* y,
                            int64_t block_rows, void* workspace, size_t workspace_bytes,
                            int32_t* dev_status, void* stream);

/* Rate probes of the units that bind the splat's blend, for roofline denominators measured on the
 * device at hand (no counterpart in the paper).  lsv2_rate_probe launches `blocks` CTAs of 512
 * threads, each running `iters` steps of eight independent chains of one operation:
 *   kind 0  FP32 FMA         kind 1  ex2 (the MUFU unit)
 *   kind 2  4-byte shared-memory load + store of a thread's own words (conflict-free)
 * lsv2_rate_probe_ops gives the operations one such launch performs (FMAs, ex2, or shared-memory
 * accesses); the caller times the launch on `stream` and divides.  sink: float[blocks] on the
 * device (written only to keep the work live).  Asynchronous like every other call. */
double lsv2_rate_probe_ops(int32_t kind, int64_t iters, int32_t blocks);
lsv2_status lsv2_rate_probe(int32_t kind, int64_t iters, int32_t blocks, float* sink, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LSV2_H */
