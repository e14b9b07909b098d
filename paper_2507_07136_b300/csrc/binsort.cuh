// binsort.cuh -- launch interface of the tile binning / depth sort.
#pragma once

#include "device.cuh"

namespace lsv2 {

struct BinSortArgs {
    int64_t n;
    int GX, num_tiles;
    const int32_t* rect;
    const uint32_t* touched;
    const float* depth;
    void* workspace;
    uint32_t* gauss_ids;
    int64_t capacity;
    uint32_t* tile_ranges;
    int64_t* num_instances;
    int32_t* status;
};

size_t binsort_workspace_bytes(int64_t capacity, int32_t num_tiles);
cudaError_t launch_binsort(const BinSortArgs& a, cudaStream_t stream);

}  // namespace lsv2
