// views.cu -- lsv2_query_views: text-query relevancy for many views of one scene in one call.
//
// Stream-ordered sequence of multi-view kernels, no host synchronisation, so the whole call can
// be captured once in a CUDA graph and replayed:
//   project (grid.y = view) -> bin/sort over the concatenated tiles of all views -> pack records
//   (grid.y = view) -> persistent splat over (view, tile) work items from an atomic queue ->
//   B = [C | S t] per level (S S^T = C C^T) -> tensor-core relevancy over all views' pixels.
#include <vector>

#include "binsort.cuh"
#include "device.cuh"
#include "project.cuh"
#include "query.cuh"
#include "query_tc.cuh"
#include "splat.cuh"

namespace lsv2 {
namespace {

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

struct ViewsLayout {
    size_t xy, conic, axes, extent, depth, radius, rect, touched, flags;   // projection arrays [V][n]
    size_t bin, ids, ranges, recs, coeff, finalT, nlast, query, queue, bytes;
    size_t bin_bytes, query_bytes;
    int64_t P_total;
    int T_total;
};

ViewsLayout views_layout(int V, const lsv2_camera* cams, int64_t n, int levels, int K, int64_t capacity, int Q,
                         int n_neg)
{
    ViewsLayout L{};
    const size_t vn = (size_t)V * (size_t)n;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += a256(bytes);
        return at;
    };
    L.xy = take(vn * 16);
    L.conic = take(vn * 16);
    L.axes = take(vn * 32);
    L.extent = take(vn * 8);
    L.depth = take(vn * 4);
    L.radius = take(vn * 4);
    L.rect = take(vn * 16);
    L.touched = take(vn * 4);
    L.flags = take(vn);
    int32_t T[kMaxViews];
    L.T_total = 0;
    L.P_total = 0;
    for (int v = 0; v < V; ++v) {
        T[v] = ((cams[v].width + cams[v].tile_w - 1) / cams[v].tile_w) * ((cams[v].height + cams[v].tile_h - 1) / cams[v].tile_h);
        L.T_total += T[v];
        L.P_total += (int64_t)cams[v].width * cams[v].height;
    }
    L.bin_bytes = binsort_views_workspace_bytes(n, capacity, T, V);
    L.bin = take(L.bin_bytes);
    L.ids = take((size_t)capacity * 4);
    L.ranges = take((size_t)L.T_total * 8);
    L.recs = take(vn * (size_t)splat_record_bytes(levels, K));
    L.coeff = take((size_t)levels * (size_t)L.P_total * 64 * 2);   // BF16: the relevancy rounds W to BF16
    L.finalT = take((size_t)L.P_total * 4);
    L.nlast = take((size_t)L.P_total * 4);
    L.query_bytes = query_workspace_bytes(levels, Q * (1 + n_neg));
    L.query = take(L.query_bytes);
    L.queue = take(16);
    L.bytes = o;
    return L;
}

bool cams_ok(int V, const lsv2_camera* cams)
{
    if (V < 1 || V > kMaxViews || V > kMaxSplatViews || V > kMaxQueryViews || V > kMaxProjectViews || !cams)
        return false;
    for (int v = 0; v < V; ++v) {
        const lsv2_camera& c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 32768 || c.height > 32768) return false;
        if (c.tile_w != cams[0].tile_w || c.tile_h != cams[0].tile_h) return false;
        if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !(c.near_z > 0.0f)) return false;
    }
    return true;
}

int sm_count()
{
    int dev = 0, n = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

}  // namespace
}  // namespace lsv2

using namespace lsv2;

extern "C" size_t lsv2_query_views_workspace_bytes(int32_t V, const lsv2_camera* cams, int64_t n, int32_t levels,
                                                   int32_t K, int64_t capacity, int32_t Q, int32_t n_neg)
{
    if (!cams_ok(V, cams) || n < 0 || levels < 1 || K < 1 || levels * K > kMaxPairs || capacity < 1 || Q < 1 ||
        n_neg < 1)
        return 0;
    return views_layout(V, cams, n, levels, K, capacity, Q, n_neg).bytes;
}

extern "C" lsv2_status lsv2_query_views(int32_t V, const lsv2_camera* cams, int64_t n, const float* means,
                                        const float* scales, const float* quats, const float* opacity, int32_t levels,
                                        int32_t K, int32_t L, const uint8_t* idx, const float* w,
                                        const float* codebook, int32_t D, int32_t Q, int32_t n_neg, const float* text,
                                        float tau, int64_t capacity, int32_t stage_batch, void* workspace,
                                        size_t workspace_bytes, void* rel, lsv2_dtype rel_dtype,
                                        int64_t* dev_num_instances, int32_t* dev_status, void* stream)
{
    if (stage_batch != 0 && stage_batch != 16 && stage_batch != 32) return LSV2_ERR_UNSUPPORTED;
    if (!cams_ok(V, cams) || n < 0 || !rel || !dev_num_instances || Q < 1 || n_neg < 1 || D <= 0)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!means || !scales || !quats || !opacity || !idx || !w)) return LSV2_ERR_INVALID_ARGUMENT;
    if (!codebook || !text || capacity < 1 || capacity > 0x7FFFFFFFll) return LSV2_ERR_INVALID_ARGUMENT;
    if (L != 64 || !splat_supported(levels, K, L, cams[0].tile_w, cams[0].tile_h) || K != 4 ||
        !query_tc_supported(Q, n_neg) || D % 4 != 0 || D > 12288)
        return LSV2_ERR_UNSUPPORTED;
    if (rel_dtype != LSV2_F32 && rel_dtype != LSV2_BF16) return LSV2_ERR_INVALID_ARGUMENT;
    const ViewsLayout Lo = views_layout(V, cams, n, levels, K, capacity, Q, n_neg);
    if (!workspace || workspace_bytes < Lo.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return LSV2_ERR_INVALID_ARGUMENT;
    for (int v = 0; v < V; ++v) {
        const int T = ((cams[v].width + cams[v].tile_w - 1) / cams[v].tile_w) *
                      ((cams[v].height + cams[v].tile_h - 1) / cams[v].tile_h);
        if (T > binsort_max_tiles_per_view()) return LSV2_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    lsv2_proj pj{reinterpret_cast<float*>(ws + Lo.xy), reinterpret_cast<float*>(ws + Lo.conic),
                 reinterpret_cast<float*>(ws + Lo.extent), reinterpret_cast<float*>(ws + Lo.depth),
                 reinterpret_cast<int32_t*>(ws + Lo.radius), reinterpret_cast<int32_t*>(ws + Lo.rect),
                 reinterpret_cast<uint32_t*>(ws + Lo.touched), reinterpret_cast<uint8_t*>(ws + Lo.flags),
                 reinterpret_cast<float*>(ws + Lo.axes)};
    cudaError_t e = launch_project(cams, V, n, means, scales, quats, opacity, pj, dev_status, st);
    if (e != cudaSuccess) return LSV2_ERR_CUDA;

    BinSortViews b{};
    b.V = V;
    b.n = n;
    for (int v = 0; v < V; ++v) {
        b.GX[v] = (cams[v].width + cams[v].tile_w - 1) / cams[v].tile_w;
        b.T[v] = b.GX[v] * ((cams[v].height + cams[v].tile_h - 1) / cams[v].tile_h);
    }
    b.rect = pj.rect;
    b.touched = pj.tiles_touched;
    b.depth = pj.depth;
    b.workspace = ws + Lo.bin;
    b.gauss_ids = reinterpret_cast<uint32_t*>(ws + Lo.ids);
    b.capacity = capacity;
    b.tile_ranges = reinterpret_cast<uint32_t*>(ws + Lo.ranges);
    b.num_instances = dev_num_instances;
    b.status = dev_status;
    e = launch_binsort_views(b, st);
    if (e != cudaSuccess) return LSV2_ERR_CUDA;

    const int rec_bytes = splat_record_bytes(levels, K);
    PackArgs pa{n, levels, K, rec_bytes, pj.xy, pj.axes, pj.conic_o, pj.extent, idx, w,
                reinterpret_cast<float*>(ws + Lo.recs), dev_status};
    e = launch_pack(pa, st, V);
    if (e != cudaSuccess) return LSV2_ERR_CUDA;

    SplatViewsArgs sa{};
    sa.V = V;
    sa.total_tiles = Lo.T_total;
    int tb = 0;
    size_t coeff_off = 0, pix_off = 0;
    std::vector<int64_t> P(V);
    for (int v = 0; v < V; ++v) {
        const int GX = b.GX[v];
        sa.view[v] = SplatView{cams[v].width, cams[v].height, GX, tb, (size_t)v * (size_t)n * (rec_bytes / 4),
                               coeff_off, pix_off};
        P[v] = (int64_t)cams[v].width * cams[v].height;
        tb += b.T[v];
        coeff_off += (size_t)levels * P[v] * 64;
        pix_off += P[v];
    }
    sa.view[V] = SplatView{0, 0, 0, tb, 0, coeff_off, pix_off};
    sa.tile_ranges = b.tile_ranges;
    sa.gauss_ids = b.gauss_ids;
    sa.recs = reinterpret_cast<const float*>(ws + Lo.recs);
    sa.coeff = reinterpret_cast<float*>(ws + Lo.coeff);
    sa.final_T = reinterpret_cast<float*>(ws + Lo.finalT);
    sa.n_last = reinterpret_cast<uint32_t*>(ws + Lo.nlast);
    sa.queue = reinterpret_cast<uint32_t*>(ws + Lo.queue);
    sa.status = dev_status;
    sa.coeff_bf16 = 1;
    e = launch_splat_views(levels, K, cams[0].tile_w, cams[0].tile_h, stage_batch, sa, sm_count(), st);
    if (e == cudaErrorInvalidValue) return LSV2_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return LSV2_ERR_CUDA;

    const int nt = Q * (1 + n_neg);
    void* qws = ws + Lo.query;
    e = launch_query_prepare(levels, D, nt, codebook, text, qws, st);
    if (e != cudaSuccess) return LSV2_ERR_CUDA;
    e = launch_query_factor(levels, nt, qws, st);
    if (e != cudaSuccess) return LSV2_ERR_CUDA;
    e = launch_query_tc_views(levels, V, P.data(), Q, n_neg, tau, sa.coeff, true, query_ws_bt(qws),
                              query_ws_tnorm(qws, levels, nt), rel, rel_dtype == LSV2_BF16, sm_count(), dev_status,
                              st);
    return e == cudaSuccess ? LSV2_OK : LSV2_ERR_CUDA;
}
