// binsort.cuh -- launch interface of the tile binning / depth sort (one or several views).
#pragma once

#include "device.cuh"

namespace lsv2 {

constexpr int kMaxViews = 64;

struct BinSortViews {
    int V;
    int64_t n;                    // Gaussians per view (projection arrays are [V][n])
    int32_t GX[kMaxViews];        // tile-grid width of each view
    int32_t T[kMaxViews];         // tiles of each view (global tile ids are concatenated)
    const int32_t* rect;          // [V][n][4]
    const uint32_t* touched;      // [V][n]
    const float* depth;           // [V][n]
    void* workspace;
    uint32_t* gauss_ids;          // [capacity]
    int64_t capacity;
    uint32_t* tile_ranges;        // [sum T][2]
    int64_t* num_instances;
    int32_t* status;
};

size_t binsort_workspace_bytes(int64_t n, int64_t capacity, int32_t num_tiles);
size_t binsort_views_workspace_bytes(int64_t n, int64_t capacity, const int32_t* num_tiles, int V);
int binsort_max_tiles_per_view();
cudaError_t launch_binsort_views(const BinSortViews& a, cudaStream_t stream);

}  // namespace lsv2
