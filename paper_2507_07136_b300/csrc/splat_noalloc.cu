// splat_noalloc.cu -- lsv2_splat_coeffs_noalloc: the sparse-coefficient splat for callers that
// cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc or hand over a workspace buffer: code
// running where the device allocator must not be touched (a real-time render loop with a
// fixed memory budget, an embedding runtime that owns all device memory and exposes only its
// input/output buffers, or a host process that has no allocator of its own to size and free
// a workspace).  For them this entry point keeps the splat's per-Gaussian record scratch in a
// file-scope device array of fixed size instead of a caller-provided workspace.  Every GPU
// that loads the library holds this array until the process exits.
//
// The array's name is only a host-side stand-in in host code, not a device address; the
// device address is obtained with cudaGetSymbolAddress once per device (on the first call
// made on that device, with the device current) and passed to the kernels.  The address is kept
// for the life of the process: after cudaDeviceReset the module is loaded again and the kept
// address is stale, so this entry point must not be used on a device after it was reset.
#include <mutex>

#include "device.cuh"
#include "splat.cuh"

namespace lsv2 {
namespace {

constexpr size_t kScratchBytes = (size_t)LSV2_SPLAT_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_splat_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_splat_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_splat_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace lsv2

using namespace lsv2;

extern "C" lsv2_status lsv2_splat_coeffs_noalloc(const lsv2_camera* cam, int64_t n, const lsv2_proj* proj,
                                                 const uint32_t* tile_ranges, const uint32_t* gauss_ids,
                                                 int32_t levels, int32_t K, int32_t L, const uint8_t* idx,
                                                 const float* w, float* coeff, float* final_T, uint32_t* n_last,
                                                 int32_t* dev_status, void* stream)
{
    if (!cam || n < 0 || !proj || !tile_ranges || !gauss_ids || !coeff || !final_T || !n_last)
        return LSV2_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!idx || !w)) return LSV2_ERR_INVALID_ARGUMENT;
    if (!splat_supported(levels, K, L, cam->tile_w, cam->tile_h)) return LSV2_ERR_UNSUPPORTED;
    // more Gaussians than the fixed scratch holds (checked before any size product is formed)
    if ((uint64_t)n > kScratchBytes / (size_t)splat_record_bytes(levels, K)) return LSV2_ERR_CAPACITY;
    const size_t need = lsv2_splat_workspace_bytes(n, levels, K);
    if (need == 0 && n > 0) return LSV2_ERR_INVALID_ARGUMENT;
    if (need > kScratchBytes) return LSV2_ERR_CAPACITY;
    void* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return LSV2_ERR_CUDA;
    // The scratch needs no clearing: the pack kernel writes the record of every Gaussian
    // g < n before the splat kernel reads any, and the splat reads only records of ids < n.
    return lsv2_splat_coeffs(cam, n, proj, tile_ranges, gauss_ids, levels, K, L, idx, w, scratch, need, coeff,
                             final_T, n_last, dev_status, stream);
}
