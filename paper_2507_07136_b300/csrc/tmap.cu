// tmap.cu -- tiled TMA tensor maps.  The encoder is a driver-API function; it is reached
// through the runtime's driver entry-point query so the library does not link the driver
// library itself.
#include "tmap.cuh"

#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cstring>

namespace lsv2 {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Packed row-major tensor of `rank` dimensions (innermost first), boxes of {b0, b1, 1, ...}.
bool encode_packed(CUtensorMap* map, const void* base, bool bf16, int rank, const uint64_t* d, uint32_t b0, uint32_t b1,
                   bool promote_l2)
{
    std::memset(map, 0, sizeof(*map));
    const PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn || !base) return false;
    for (int i = 0; i < rank; ++i)
        if (d[i] == 0) return false;
    const uint64_t esz = bf16 ? 2 : 4;
    if (b0 * esz > 128 || (b0 * esz) % 16 != 0 || b1 == 0 || b1 > 256) return false;
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], elem[4];
    uint64_t stride = esz;
    for (int i = 0; i < rank; ++i) {
        dims[i] = d[i];
        box[i] = i == 0 ? b0 : (i == 1 ? b1 : 1u);
        elem[i] = 1;
        stride *= d[i];
        if (i + 1 < rank) strides[i] = stride;
    }
    const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          promote_l2 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool encode_tmap_3d(CUtensorMap* map, const void* base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2,
                    uint32_t b0, uint32_t b1, bool promote_l2)
{
    const uint64_t d[3] = {d0, d1, d2};
    return encode_packed(map, base, bf16, 3, d, b0, b1, promote_l2);
}

bool encode_tmap_4d(CUtensorMap* map, const void* base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3,
                    uint32_t b0, uint32_t b1, bool promote_l2)
{
    const uint64_t d[4] = {d0, d1, d2, d3};
    return encode_packed(map, base, bf16, 4, d, b0, b1, promote_l2);
}

}  // namespace lsv2
