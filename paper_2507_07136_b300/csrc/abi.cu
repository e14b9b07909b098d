// abi.cu -- the extern "C" entry points declared in include/lsv2.h: host-side argument
// checks, then stream-ordered launches.  No entry point allocates device memory or
// synchronises the host.
#include <algorithm>
#include <atomic>

#include "backward.cuh"
#include "binsort.cuh"
#include "decode.cuh"
#include "decode_tc.cuh"
#include "device.cuh"
#include "project.cuh"
#include "query.cuh"
#include "query_tc.cuh"
#include "splat.cuh"

using namespace lsv2;

namespace {

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

lsv2_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LSV2_OK : LSV2_ERR_CUDA; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool camera_ok(const lsv2_camera* c)
{
    if (!c) return false;
    if (c->width <= 0 || c->height <= 0 || c->width > 32768 || c->height > 32768) return false;
    const bool tile_ok = (c->tile_w == 16 && c->tile_h == 16) || (c->tile_w == 8 && c->tile_h == 8) ||
                         (c->tile_w == 32 && c->tile_h == 8);
    if (!tile_ok) return false;
    if (!(c->fx > 0.0f) || !(c->fy > 0.0f) || !(c->near_z > 0.0f)) return false;
    return true;
}

bool proj_ok(const lsv2_proj* p)
{
    return p && p->xy && p->conic_o && p->extent && p->depth && p->radius && p->rect && p->tiles_touched &&
           p->flags && p->axes && aligned16(p->xy) && aligned16(p->conic_o) && aligned16(p->rect) && aligned16(p->axes) &&
           (reinterpret_cast<uintptr_t>(p->extent) & 7u) == 0;
}

int num_tiles(const lsv2_camera* c)
{
    return ((c->width + c->tile_w - 1) / c->tile_w) * ((c->height + c->tile_h - 1) / c->tile_h);
}

int sm_count()
{
    int dev = 0, n = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};

}  // namespace

uint64_t lsv2::wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

extern "C" {

int32_t lsv2_abi_version(void) { return LSV2_ABI_VERSION; }

void lsv2_set_wait_limit_ns(uint64_t ns) { g_wait_ns.store(ns, std::memory_order_relaxed); }

uint64_t lsv2_wait_limit_ns(void) { return g_wait_ns.load(std::memory_order_relaxed); }

const char* lsv2_status_string(lsv2_status s)
{
    switch (s) {
        case LSV2_OK: return "ok";
        case LSV2_ERR_INVALID_ARGUMENT: return "invalid argument";
        case LSV2_ERR_UNSUPPORTED: return "unsupported configuration";
        case LSV2_ERR_CAPACITY: return "instance capacity exceeded";
        case LSV2_ERR_CUDA: return "CUDA error";
        case LSV2_ERR_TIMEOUT: return "device wait timed out";
        case LSV2_ERR_NONFINITE: return "non-finite value";
    }
    return "unknown status";
}

lsv2_status lsv2_project(const lsv2_camera* cam, int64_t n, const float* means, const float* scales,
                         const float* quats, const float* opacity, const lsv2_proj* out, int32_t* dev_status,
                         void* stream)
{
    if (!camera_ok(cam) || n < 0 || !proj_ok(out)) return LSV2_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!means || !scales || !quats || !opacity || !aligned16(quats))) return LSV2_ERR_INVALID_ARGUMENT;
    if (n > (int64_t)0xFFFFFFFFll) return LSV2_ERR_UNSUPPORTED;
    return cuda_status(launch_project(cam, 1, n, means, scales, quats, opacity, *out, dev_status, S(stream)));
}

size_t lsv2_bin_sort_workspace_bytes(int64_t n, int64_t capacity, int32_t num_tiles_)
{
    if (n < 0 || capacity < 0 || num_tiles_ < 0) return 0;
    return binsort_workspace_bytes(n, capacity, num_tiles_);
}

lsv2_status lsv2_bin_sort(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj, void* workspace,
                          size_t workspace_bytes, uint32_t* gauss_ids, int64_t capacity, uint32_t* tile_ranges,
                          int64_t* dev_num_instances, int32_t* dev_status, void* stream)
{
    if (!camera_ok(cam) || n < 0 || !proj_ok(proj) || !tile_ranges || !dev_num_instances) return LSV2_ERR_INVALID_ARGUMENT;
    if (capacity < 1 || capacity > 0x7FFFFFFFll || !gauss_ids) return LSV2_ERR_INVALID_ARGUMENT;
    const int T = num_tiles(cam);
    if (T > binsort_max_tiles_per_view()) return LSV2_ERR_UNSUPPORTED;
    if (!workspace || workspace_bytes < binsort_workspace_bytes(n, capacity, T) || !aligned16(workspace))
        return LSV2_ERR_INVALID_ARGUMENT;
    BinSortViews a{};
    a.V = 1;
    a.n = n;
    a.GX[0] = (cam->width + cam->tile_w - 1) / cam->tile_w;
    a.T[0] = T;
    a.rect = proj->rect;
    a.touched = proj->tiles_touched;
    a.depth = proj->depth;
    a.workspace = workspace;
    a.gauss_ids = gauss_ids;
    a.capacity = capacity;
    a.tile_ranges = tile_ranges;
    a.num_instances = dev_num_instances;
    a.status = dev_status;
    return cuda_status(launch_binsort_views(a, S(stream)));
}

size_t lsv2_splat_workspace_bytes(int64_t n, int32_t levels, int32_t K)
{
    if (n < 0 || levels < 1 || K < 1 || levels * K > kMaxPairs) return 0;
    const size_t rec = (size_t)splat_record_bytes(levels, K);
    if ((uint64_t)n > (SIZE_MAX - 255) / rec) return 0;   // the size would not fit in size_t
    return align256((size_t)n * rec);
}

lsv2_status lsv2_splat_coeffs(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj, const uint32_t* tile_ranges,
                              const uint32_t* gauss_ids, int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                              const float* w, void* workspace, size_t workspace_bytes, float* coeff, float* final_T,
                              uint32_t* n_last, int32_t* dev_status, void* stream)
{
    if (!camera_ok(cam) || n < 0 || !proj_ok(proj) || !tile_ranges || !gauss_ids || !coeff || !final_T || !n_last)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!idx || !w)) return LSV2_ERR_INVALID_ARGUMENT;
    if (!splat_supported(levels, K, L, cam->tile_w, cam->tile_h)) return LSV2_ERR_UNSUPPORTED;
    if (!aligned16(coeff) || !workspace || !aligned16(workspace) ||
        workspace_bytes < lsv2_splat_workspace_bytes(n, levels, K))
        return LSV2_ERR_INVALID_ARGUMENT;
    PackArgs pa{n, levels, K, splat_record_bytes(levels, K), proj->xy, proj->axes, proj->conic_o, proj->extent, idx,
                w, static_cast<float*>(workspace), dev_status};
    pa.L = L;
    cudaError_t e = launch_pack(pa, S(stream));
    if (e != cudaSuccess) return LSV2_ERR_CUDA;
    SplatArgs sa{*cam, tile_ranges, gauss_ids, static_cast<const float*>(workspace), coeff, final_T, n_last, dev_status};
    sa.L = L;
    return cuda_status(launch_splat(levels, K, sa, S(stream)));
}

lsv2_status lsv2_splat_coeffs_bf16(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                                   const uint32_t* tile_ranges, const uint32_t* gauss_ids, int32_t levels, int32_t K,
                                   int32_t L, const uint8_t* idx, const float* w, void* workspace,
                                   size_t workspace_bytes, void* coeff_bf16, float* final_T, uint32_t* n_last,
                                   int32_t* dev_status, void* stream)
{
    if (!camera_ok(cam) || n < 0 || !proj_ok(proj) || !tile_ranges || !gauss_ids || !coeff_bf16 || !final_T ||
        !n_last)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!idx || !w)) return LSV2_ERR_INVALID_ARGUMENT;
    if (!splat_supported(levels, K, L, cam->tile_w, cam->tile_h)) return LSV2_ERR_UNSUPPORTED;
    if (!aligned16(coeff_bf16) || !workspace || !aligned16(workspace) ||
        workspace_bytes < lsv2_splat_workspace_bytes(n, levels, K))
        return LSV2_ERR_INVALID_ARGUMENT;
    PackArgs pa{n, levels, K, splat_record_bytes(levels, K), proj->xy, proj->axes, proj->conic_o, proj->extent, idx,
                w, static_cast<float*>(workspace), dev_status};
    pa.L = L;
    cudaError_t e = launch_pack(pa, S(stream));
    if (e != cudaSuccess) return LSV2_ERR_CUDA;
    SplatArgs sa{*cam, tile_ranges, gauss_ids, static_cast<const float*>(workspace), static_cast<float*>(coeff_bf16),
                 final_T, n_last, dev_status, 1};
    sa.L = L;
    return cuda_status(launch_splat(levels, K, sa, S(stream)));
}

size_t lsv2_splat_dense_workspace_bytes(int64_t n, int32_t levels)
{
    if (n < 0 || (levels != 1 && levels != 3)) return 0;
    return align256((size_t)n * (size_t)splat_dense_record_bytes(levels));
}

lsv2_status lsv2_splat_coeffs_dense(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                                    const uint32_t* tile_ranges, const uint32_t* gauss_ids, int32_t levels, int32_t K,
                                    int32_t L, const uint8_t* idx, const float* w, void* workspace,
                                    size_t workspace_bytes, float* coeff, float* final_T, uint32_t* n_last,
                                    int32_t* dev_status, void* stream)
{
    if (!camera_ok(cam) || n < 0 || !proj_ok(proj) || !tile_ranges || !gauss_ids || !coeff || !final_T || !n_last ||
        K < 1)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!idx || !w)) return LSV2_ERR_INVALID_ARGUMENT;
    if (!splat_dense_supported(levels, L, cam->tile_w, cam->tile_h)) return LSV2_ERR_UNSUPPORTED;
    if (!aligned16(coeff) || !workspace || !aligned16(workspace) ||
        workspace_bytes < lsv2_splat_dense_workspace_bytes(n, levels))
        return LSV2_ERR_INVALID_ARGUMENT;
    PackArgs pa{n, levels, K, splat_dense_record_bytes(levels), proj->xy, proj->axes, proj->conic_o, proj->extent,
                idx, w, static_cast<float*>(workspace), dev_status};
    cudaError_t e = launch_pack_dense(pa, S(stream));
    if (e != cudaSuccess) return LSV2_ERR_CUDA;
    SplatArgs sa{*cam, tile_ranges, gauss_ids, static_cast<const float*>(workspace), coeff, final_T, n_last, dev_status};
    return cuda_status(launch_splat_dense(levels, sa, S(stream)));
}

lsv2_status lsv2_decode(int32_t levels, int64_t P, int32_t L, int32_t D, const void* coeff, lsv2_dtype coeff_dtype,
                        const void* codebook, lsv2_dtype codebook_dtype, void* feat, lsv2_dtype out_dtype,
                        int32_t* dev_status, void* stream)
{
    if (levels < 1 || P < 0 || !coeff || !codebook || !feat) return LSV2_ERR_INVALID_ARGUMENT;
    if (L != 64 || D <= 0 || D % 128 != 0) return LSV2_ERR_UNSUPPORTED;
    if (!aligned16(coeff) || !aligned16(codebook) || !aligned16(feat)) return LSV2_ERR_INVALID_ARGUMENT;
    const bool dt_ok = (coeff_dtype == LSV2_F32 || coeff_dtype == LSV2_BF16) &&
                       (codebook_dtype == LSV2_F32 || codebook_dtype == LSV2_BF16) &&
                       (out_dtype == LSV2_F32 || out_dtype == LSV2_BF16);
    if (!dt_ok) return LSV2_ERR_INVALID_ARGUMENT;
    if (coeff_dtype == LSV2_F32 && codebook_dtype == LSV2_F32 && out_dtype == LSV2_F32)
        return cuda_status(launch_decode_f32(levels, P, D, static_cast<const float*>(coeff),
                                             static_cast<const float*>(codebook), static_cast<float*>(feat),
                                             S(stream)));
    if (!decode_tc_supported(D)) return LSV2_ERR_UNSUPPORTED;
    return cuda_status(launch_decode_tc(levels, P, D, coeff, coeff_dtype == LSV2_BF16, codebook,
                                        codebook_dtype == LSV2_BF16, feat, out_dtype == LSV2_BF16, sm_count(),
                                        dev_status, S(stream)));
}

size_t lsv2_query_workspace_bytes(int32_t levels, int32_t L, int32_t Q, int32_t n_neg)
{
    if (levels < 1 || L != 64 || Q < 1 || n_neg < 1) return 0;
    return query_workspace_bytes(levels, Q * (1 + n_neg));
}

lsv2_status lsv2_query_prepare(int32_t levels, int32_t L, int32_t D, const float* codebook, int32_t Q, int32_t n_neg,
                               const float* text, lsv2_dtype compute_dtype, void* workspace, size_t workspace_bytes,
                               void* stream)
{
    if (levels < 1 || !codebook || !text || Q < 1 || n_neg < 1 || D <= 0) return LSV2_ERR_INVALID_ARGUMENT;
    if (L != 64 || Q * (1 + n_neg) > 512 || D % 4 != 0 || D > 12288) return LSV2_ERR_UNSUPPORTED;
    if (!aligned16(codebook) || !aligned16(text)) return LSV2_ERR_INVALID_ARGUMENT;
    const int nt = Q * (1 + n_neg);
    if (!workspace || !aligned16(workspace) || workspace_bytes < query_workspace_bytes(levels, nt))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (compute_dtype != LSV2_F32 && compute_dtype != LSV2_BF16) return LSV2_ERR_INVALID_ARGUMENT;
    if (compute_dtype == LSV2_BF16 && !query_tc_supported(Q, n_neg)) return LSV2_ERR_UNSUPPORTED;
    cudaError_t e = launch_query_prepare(levels, D, nt, codebook, text, workspace, S(stream));
    if (e != cudaSuccess) return LSV2_ERR_CUDA;
    if (compute_dtype == LSV2_BF16) e = launch_query_factor(levels, nt, workspace, S(stream));
    return cuda_status(e);
}

lsv2_status lsv2_query_prepared(int32_t levels, int64_t P, int32_t L, const void* coeff, lsv2_dtype coeff_dtype,
                                int32_t Q, int32_t n_neg, float tau, const void* workspace, size_t workspace_bytes,
                                void* rel, lsv2_dtype rel_dtype, lsv2_dtype compute_dtype, int32_t* dev_status,
                                void* stream)
{
    if (levels < 1 || P < 0 || !coeff || !rel || Q < 1 || n_neg < 1) return LSV2_ERR_INVALID_ARGUMENT;
    if (L != 64 || Q * (1 + n_neg) > 512) return LSV2_ERR_UNSUPPORTED;
    const int nt = Q * (1 + n_neg);
    if (!workspace || !aligned16(workspace) || workspace_bytes < query_workspace_bytes(levels, nt))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (!aligned16(coeff)) return LSV2_ERR_INVALID_ARGUMENT;
    if (coeff_dtype != LSV2_F32 && !(coeff_dtype == LSV2_BF16 && compute_dtype == LSV2_BF16))
        return LSV2_ERR_UNSUPPORTED;
    if (rel_dtype != LSV2_F32 && rel_dtype != LSV2_BF16) return LSV2_ERR_INVALID_ARGUMENT;
    if (compute_dtype == LSV2_F32 && rel_dtype == LSV2_F32)
        return cuda_status(launch_query_f32(levels, P, Q, n_neg, tau, static_cast<const float*>(coeff), workspace,
                                            static_cast<float*>(rel), S(stream)));
    if (compute_dtype == LSV2_BF16) {
        if (!query_tc_supported(Q, n_neg)) return LSV2_ERR_UNSUPPORTED;
        return cuda_status(launch_query_tc(levels, P, Q, n_neg, tau, coeff, coeff_dtype == LSV2_BF16,
                                           query_ws_bt(workspace), query_ws_tnorm(workspace, levels, nt), rel,
                                           rel_dtype == LSV2_BF16, sm_count(), dev_status, S(stream)));
    }
    return LSV2_ERR_UNSUPPORTED;
}

lsv2_status lsv2_query(int32_t levels, int64_t P, int32_t L, int32_t D, const void* coeff, lsv2_dtype coeff_dtype,
                       const float* codebook, int32_t Q, int32_t n_neg, const float* text, float tau, void* workspace,
                       size_t workspace_bytes, void* rel, lsv2_dtype rel_dtype, lsv2_dtype compute_dtype,
                       int32_t* dev_status, void* stream)
{
    // every host check of both halves before anything is launched
    if (levels < 1 || P < 0 || !coeff || !codebook || !text || !rel || Q < 1 || n_neg < 1 || D <= 0)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (L != 64 || Q * (1 + n_neg) > 512 || D % 4 != 0 || D > 12288) return LSV2_ERR_UNSUPPORTED;
    if (!aligned16(codebook) || !aligned16(text)) return LSV2_ERR_INVALID_ARGUMENT;
    const int nt = Q * (1 + n_neg);
    if (!workspace || !aligned16(workspace) || workspace_bytes < query_workspace_bytes(levels, nt))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (!aligned16(coeff)) return LSV2_ERR_INVALID_ARGUMENT;
    if (coeff_dtype != LSV2_F32 && !(coeff_dtype == LSV2_BF16 && compute_dtype == LSV2_BF16))
        return LSV2_ERR_UNSUPPORTED;
    if (rel_dtype != LSV2_F32 && rel_dtype != LSV2_BF16) return LSV2_ERR_INVALID_ARGUMENT;
    if (compute_dtype != LSV2_F32 && compute_dtype != LSV2_BF16) return LSV2_ERR_UNSUPPORTED;
    if (compute_dtype == LSV2_F32 && rel_dtype != LSV2_F32) return LSV2_ERR_UNSUPPORTED;
    if (compute_dtype == LSV2_BF16 && !query_tc_supported(Q, n_neg)) return LSV2_ERR_UNSUPPORTED;
    const lsv2_status st = lsv2_query_prepare(levels, L, D, codebook, Q, n_neg, text, compute_dtype, workspace,
                                              workspace_bytes, stream);
    if (st != LSV2_OK) return st;
    return lsv2_query_prepared(levels, P, L, coeff, coeff_dtype, Q, n_neg, tau, workspace, workspace_bytes, rel,
                               rel_dtype, compute_dtype, dev_status, stream);
}

lsv2_status lsv2_l1_decode_backward(int32_t levels, int64_t P, int32_t L, int32_t D, const float* coeff,
                                    const float* codebook, const float* target, float* loss, float* dcoeff,
                                    float* dcodebook, int32_t* dev_status, void* stream)
{
    if (levels < 1 || P < 0 || !coeff || !codebook || !target || !loss || !dcoeff || !dcodebook)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (L != 64 || D <= 0 || D % 128 != 0 || D > 512) return LSV2_ERR_UNSUPPORTED;
    if (P > (int64_t)0x7FFFFF00ll) return LSV2_ERR_UNSUPPORTED;
    if (!aligned16(coeff) || !aligned16(codebook) || !aligned16(target) || !aligned16(dcoeff))
        return LSV2_ERR_INVALID_ARGUMENT;
    return cuda_status(launch_l1_decode_backward_tc(levels, P, D, coeff, codebook, target, loss, dcoeff, dcodebook,
                                                    sm_count(), dev_status, S(stream)));
}

size_t lsv2_splat_backward_workspace_bytes(int64_t n)
{
    if (n < 0) return 0;
    return splat_backward_workspace_bytes(n, 3, 8);
}

lsv2_status lsv2_splat_backward(const lsv2_camera* cam, int64_t n, const float* means, const float* scales,
                                const float* quats, const lsv2_proj* proj, const uint32_t* tile_ranges,
                                const uint32_t* gauss_ids, int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                                const float* w, const float* final_T, const uint32_t* n_last, const float* dcoeff,
                                void* workspace, size_t workspace_bytes, float* dw, float* dopacity, float* dmeans,
                                float* dscales, float* dquats, int32_t* dev_status, void* stream)
{
    (void)dev_status;
    if (!camera_ok(cam) || n < 0 || !proj_ok(proj) || !tile_ranges || !gauss_ids || !final_T || !n_last || !dcoeff)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!means || !scales || !quats || !idx || !w || !dw || !dopacity || !dmeans || !dscales || !dquats))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (L != 64 || !splat_backward_supported(levels, K)) return LSV2_ERR_UNSUPPORTED;
    if (!workspace || !aligned16(workspace) || workspace_bytes < splat_backward_workspace_bytes(n, levels, K) ||
        !aligned16(dcoeff) || !aligned16(quats))
        return LSV2_ERR_INVALID_ARGUMENT;
    SplatBwdArgs a{};
    a.cam = *cam;
    a.tile_ranges = tile_ranges;
    a.gauss_ids = gauss_ids;
    a.xy = proj->xy;
    a.axes = proj->axes;
    a.conic_o = proj->conic_o;
    a.extent = proj->extent;
    a.final_T = final_T;
    a.n_last = n_last;
    a.dcoeff = dcoeff;
    a.workspace = workspace;
    a.dw = dw;
    a.dopacity = dopacity;
    a.num_sms = sm_count();
    ProjBwdArgs pa{*cam, n, means, scales, quats, proj->flags, nullptr, dmeans, dscales, dquats};
    return cuda_status(launch_splat_backward(levels, K, a, pa, idx, w, S(stream)));
}

}  // extern "C"
