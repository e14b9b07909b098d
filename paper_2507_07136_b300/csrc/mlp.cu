// mlp.cu -- the decoder of the decoder-based comparison path (LangSplat*, Sec. 3.1 and Table 1):
// a per-pixel MLP g_d from the rendered low-dimensional latent feature (Eq. 4) to the D-dim
// CLIP space, the stage the paper measures as LangSplat*'s bottleneck.  Each layer is a plain
// GEMM with a bias (+ ReLU) epilogue,
//     H_{l+1} = act(H_l W_l + b_l),   H_l rows x w_l,  W_l w_l x w_{l+1},  act = ReLU except after the last,
// with BF16 operands, biases and activations and FP32 accumulation, run by cuBLASLt (a library
// GEMM: nothing about these layers is specific to the method), or on request (block_rows ==
// LSV2_MLP_FUSED) by the fused tensor-core kernel of mlp_fused.cu.  The library path processes
// rows in blocks that bound the two intermediate activation buffers (smaller blocks keep them in
// L2 but make the GEMMs too small to fill the GPU: measured at 4.67 M rows, 2^20 rows per block
// 3.33 ms, 2^18 3.64, 2^16 4.86); the buffers, the BF16 copy of an FP32 input block and
// cuBLASLt's own workspace all live in the caller's workspace, so a call allocates nothing and
// can be captured in a CUDA graph.
#include <cublasLt.h>
#include <cuda_bf16.h>

#include <map>
#include <mutex>
#include <tuple>

#include "device.cuh"
#include "mlp_fused.cuh"

namespace lsv2 {
namespace {

constexpr int64_t kDefaultBlockRows = 1 << 20;
constexpr size_t kLtWorkspace = 32u << 20;   // cuBLASLt's workspace (inside the caller's)
constexpr int kMaxLayers = 16;

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

int64_t block_of(int64_t rows, int64_t block_rows)
{
    const int64_t b = block_rows > 0 ? block_rows : kDefaultBlockRows;
    return rows < b ? rows : b;
}

int max_hidden(int n_layers, const int32_t* widths)
{
    int m = 8;
    for (int l = 1; l < n_layers; ++l) m = widths[l] > m ? widths[l] : m;
    return m;
}

struct Sizes {
    size_t act, xin;
};

Sizes sizes(int64_t rows, int n_layers, const int32_t* widths, int64_t block_rows, bool x_f32)
{
    const int64_t block = block_of(rows, block_rows);
    return {a256((size_t)block * (size_t)max_hidden(n_layers, widths) * 2),
            x_f32 ? a256((size_t)block * (size_t)widths[0] * 2) : 0};
}

cublasLtHandle_t lt_handle()
{
    static cublasLtHandle_t h = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        if (cublasLtCreate(&h) != CUBLAS_STATUS_SUCCESS) h = nullptr;
    });
    return h;
}

// The algorithm cuBLASLt's heuristic picks for a layer shape, looked up once per shape (the
// heuristic query costs tens of microseconds of host time, more than a small layer's GEMM).
using PlanKey = std::tuple<int64_t, int, int, bool>;
std::mutex g_plan_mu;
std::map<PlanKey, cublasLtMatmulAlgo_t> g_plans;

struct LayerDesc {
    cublasLtMatmulDesc_t op = nullptr;
    cublasLtMatrixLayout_t la = nullptr, lb = nullptr, ly = nullptr;
    ~LayerDesc()
    {
        if (ly) cublasLtMatrixLayoutDestroy(ly);
        if (lb) cublasLtMatrixLayoutDestroy(lb);
        if (la) cublasLtMatrixLayoutDestroy(la);
        if (op) cublasLtMatmulDescDestroy(op);
    }
};

#define LT_OK(x) ((x) == CUBLAS_STATUS_SUCCESS)

// Y (row-major rows x n) = act(X (rows x k) W (k x n, row-major) + b).  In cuBLASLt's column-major
// terms: Y^T (n x rows, ld n) = W^T (n x k, ld n) X^T (k x rows, ld k), bias along the n rows.  The
// bias has the output's type (BF16): the library takes no FP32 bias with a BF16 output.
bool describe(LayerDesc& d, int64_t rows, int k, int n, const void* b, bool relu)
{
    const cublasOperation_t tn = CUBLAS_OP_N;
    const cublasLtEpilogue_t epi = relu ? CUBLASLT_EPILOGUE_RELU_BIAS : CUBLASLT_EPILOGUE_BIAS;
    return LT_OK(cublasLtMatmulDescCreate(&d.op, CUBLAS_COMPUTE_32F, CUDA_R_32F)) &&
           LT_OK(cublasLtMatmulDescSetAttribute(d.op, CUBLASLT_MATMUL_DESC_TRANSA, &tn, sizeof(tn))) &&
           LT_OK(cublasLtMatmulDescSetAttribute(d.op, CUBLASLT_MATMUL_DESC_TRANSB, &tn, sizeof(tn))) &&
           LT_OK(cublasLtMatmulDescSetAttribute(d.op, CUBLASLT_MATMUL_DESC_EPILOGUE, &epi, sizeof(epi))) &&
           LT_OK(cublasLtMatmulDescSetAttribute(d.op, CUBLASLT_MATMUL_DESC_BIAS_POINTER, &b, sizeof(b))) &&
           LT_OK(cublasLtMatrixLayoutCreate(&d.la, CUDA_R_16BF, (uint64_t)n, (uint64_t)k, (int64_t)n)) &&
           LT_OK(cublasLtMatrixLayoutCreate(&d.lb, CUDA_R_16BF, (uint64_t)k, (uint64_t)rows, (int64_t)k)) &&
           LT_OK(cublasLtMatrixLayoutCreate(&d.ly, CUDA_R_16BF, (uint64_t)n, (uint64_t)rows, (int64_t)n));
}

bool plan(cublasLtHandle_t h, const LayerDesc& d, int64_t rows, int k, int n, bool relu, cublasLtMatmulAlgo_t* algo)
{
    const PlanKey key{rows, k, n, relu};
    {
        std::lock_guard<std::mutex> g(g_plan_mu);
        auto it = g_plans.find(key);
        if (it != g_plans.end()) {
            *algo = it->second;
            return true;
        }
    }
    cublasLtMatmulPreference_t pref = nullptr;
    cublasLtMatmulHeuristicResult_t heur{};
    int found = 0;
    const bool ok = LT_OK(cublasLtMatmulPreferenceCreate(&pref)) &&
                    LT_OK(cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES,
                                                               &kLtWorkspace, sizeof(kLtWorkspace))) &&
                    LT_OK(cublasLtMatmulAlgoGetHeuristic(h, d.op, d.la, d.lb, d.ly, d.ly, pref, 1, &heur, &found)) &&
                    found > 0;
    if (pref) cublasLtMatmulPreferenceDestroy(pref);
    if (!ok) return false;
    std::lock_guard<std::mutex> g(g_plan_mu);
    g_plans[key] = heur.algo;
    *algo = heur.algo;
    return true;
}

bool layer(cublasLtHandle_t h, int64_t rows, int k, int n, const void* X, const void* W, const void* b, void* Y,
           bool relu, void* lt_ws, cudaStream_t stream)
{
    LayerDesc d;
    cublasLtMatmulAlgo_t algo;
    if (!describe(d, rows, k, n, b, relu) || !plan(h, d, rows, k, n, relu, &algo)) return false;
    const float alpha = 1.0f, beta = 0.0f;
    return LT_OK(cublasLtMatmul(h, d.op, &alpha, W, d.la, X, d.lb, &beta, Y, d.ly, Y, d.ly, &algo, lt_ws,
                                kLtWorkspace, stream));
}

// FP32 -> BF16 (round to nearest even) of one input block, 4 elements per thread.
__global__ void to_bf16_kernel(const float4* __restrict__ x, uint2* __restrict__ y, int64_t n4)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x[i];
        const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
        y[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
    }
}

// block_rows == LSV2_MLP_FUSED asks for the fused tensor-core kernel.
bool fused_requested(int64_t block_rows) { return block_rows == LSV2_MLP_FUSED; }

}  // namespace
}  // namespace lsv2

using namespace lsv2;

extern "C" size_t lsv2_mlp_decode_workspace_bytes(int64_t rows, int32_t n_layers, const int32_t* widths,
                                                  int32_t x_dtype, int64_t block_rows)
{
    if (rows < 0 || n_layers < 1 || n_layers > kMaxLayers || !widths || (block_rows < 0 && !fused_requested(block_rows)))
        return 0;
    if (x_dtype != LSV2_F32 && x_dtype != LSV2_BF16) return 0;
    if (fused_requested(block_rows)) {
        MlpPlan plan;
        size_t image = 0;
        return mlp_fused_plan(n_layers, widths, &plan, &image) ? a256(image) : 0;
    }
    const Sizes z = sizes(rows, n_layers, widths, block_rows, x_dtype == LSV2_F32);
    return 2 * z.act + z.xin + kLtWorkspace;
}

extern "C" lsv2_status lsv2_mlp_decode(int64_t rows, int32_t n_layers, const int32_t* widths, const void* x,
                                       int32_t x_dtype, const void* weights, const void* biases, void* y,
                                       int64_t block_rows, void* workspace, size_t workspace_bytes,
                                       int32_t* dev_status, void* stream)
{
    if (rows < 0 || n_layers < 1 || n_layers > kMaxLayers || !widths || !x || !weights || !biases || !y ||
        !workspace || (block_rows < 0 && !fused_requested(block_rows)) || (block_rows > 0 && block_rows % 128 != 0))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (x_dtype != LSV2_F32 && x_dtype != LSV2_BF16) return LSV2_ERR_INVALID_ARGUMENT;
    for (int l = 0; l <= n_layers; ++l)
        if (widths[l] < 8 || widths[l] > 4096 || widths[l] % 8 != 0) return LSV2_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(weights) | reinterpret_cast<uintptr_t>(y) |
         reinterpret_cast<uintptr_t>(biases) | reinterpret_cast<uintptr_t>(workspace)) & 15u)
        return LSV2_ERR_INVALID_ARGUMENT;
    const bool x_f32 = x_dtype == LSV2_F32;
    if (fused_requested(block_rows)) {
        MlpPlan plan;
        size_t image = 0;
        if (!mlp_fused_plan(n_layers, widths, &plan, &image)) return LSV2_ERR_UNSUPPORTED;
        if (workspace_bytes < a256(image)) return LSV2_ERR_INVALID_ARGUMENT;
        if (rows == 0) return LSV2_OK;
        return launch_mlp_fused(plan, rows, x, x_f32, weights, biases, y, workspace, dev_status,
                                static_cast<cudaStream_t>(stream)) == cudaSuccess
                   ? LSV2_OK
                   : LSV2_ERR_CUDA;
    }
    if (workspace_bytes < lsv2_mlp_decode_workspace_bytes(rows, n_layers, widths, x_dtype, block_rows))
        return LSV2_ERR_INVALID_ARGUMENT;
    if (rows == 0) return LSV2_OK;
    cublasLtHandle_t h = lt_handle();
    if (!h) return LSV2_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t block = block_of(rows, block_rows);
    const Sizes z = sizes(rows, n_layers, widths, block_rows, x_f32);
    char* ws = static_cast<char*>(workspace);
    void* buf[2] = {ws, ws + z.act};
    void* xin = ws + 2 * z.act;
    void* lt_ws = ws + 2 * z.act + z.xin;
    for (int64_t r0 = 0; r0 < rows; r0 += block) {
        const int64_t nr = rows - r0 < block ? rows - r0 : block;
        const void* in;
        if (x_f32) {
            const int64_t n4 = nr * widths[0] / 4;   // widths[0] % 8 == 0
            const int grid = (int)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096);
            to_bf16_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(static_cast<const float*>(x) +
                                                                                (size_t)r0 * widths[0]),
                                                static_cast<uint2*>(xin), n4);
            if (cudaGetLastError() != cudaSuccess) return LSV2_ERR_CUDA;
            in = xin;
        } else {
            in = static_cast<const __nv_bfloat16*>(x) + (size_t)r0 * widths[0];
        }
        size_t woff = 0, boff = 0;
        for (int l = 0; l < n_layers; ++l) {
            const int k = widths[l], n = widths[l + 1];
            const bool last = l == n_layers - 1;
            void* out = last ? static_cast<void*>(static_cast<__nv_bfloat16*>(y) + (size_t)r0 * n) : buf[l & 1];
            const void* W = static_cast<const __nv_bfloat16*>(weights) + woff;
            const void* b = static_cast<const __nv_bfloat16*>(biases) + boff;
            if (!layer(h, nr, k, n, in, W, b, out, !last, lt_ws, s)) return LSV2_ERR_CUDA;
            woff += (size_t)k * n;
            boff += (size_t)n;
            in = out;
        }
    }
    return LSV2_OK;
}
