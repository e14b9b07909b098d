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

}  // namespace

bool encode_tmap_3d(CUtensorMap* map, const void* base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2,
                    uint32_t b0, uint32_t b1, bool promote_l2)
{
    std::memset(map, 0, sizeof(*map));
    const PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn || !base || d0 == 0 || d1 == 0 || d2 == 0) return false;
    const uint64_t esz = bf16 ? 2 : 4;
    if (b0 * esz > 128 || (b0 * esz) % 16 != 0 || b1 == 0 || b1 > 256) return false;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * esz, d0 * d1 * esz};
    const cuuint32_t box[3] = {b0, b1, 1};
    const cuuint32_t elem[3] = {1, 1, 1};
    const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                          const_cast<void*>(base), dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B,
                          promote_l2 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace lsv2
