// probe.cu -- rate probes of the units the splat's blend is bound by (not part of the method):
// the FP32 FMA pipe, the MUFU ex2 unit and shared-memory loads/stores.  Each launch keeps every
// SM busy with eight independent dependency chains per thread, so the measured rate is the
// unit's throughput, not its latency; the caller times the launch and divides the operation
// count (lsv2_rate_probe_ops) by the time.  The results go to `sink` so no work is removed.
#include "device.cuh"

namespace lsv2 {
namespace {

constexpr int kThreads = 512;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) fma_probe(int64_t iters, float seed, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.999999f, k = 1e-7f * seed;
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], m, k);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;   // practically never: keeps the chains alive
}

__global__ void __launch_bounds__(kThreads) ex2_probe(int64_t iters, float seed, float* sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (seed + (float)c);
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
            x[c] = -y;   // stays in [-1, 0): ex2 of it stays in [0.5, 1]
        }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

// Shared memory: per iteration, kChains 4-byte loads and stores of the thread's own words
// (conflict-free: word = thread + 512 chain), each load feeding the next store (the splat's
// accumulator read-modify-write pattern).
__global__ void __launch_bounds__(kThreads) smem_probe(int64_t iters, float seed, float* sink)
{
    __shared__ float buf[kThreads * kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) buf[threadIdx.x + kThreads * c] = seed;
    __syncthreads();
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            volatile float* p = buf + threadIdx.x + kThreads * c;
            *p = *p + 1.0f;
        }
    __syncthreads();
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += buf[threadIdx.x + kThreads * c];
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace lsv2

using namespace lsv2;

extern "C" double lsv2_rate_probe_ops(int32_t kind, int64_t iters, int32_t blocks)
{
    // operations a launch performs: FMAs (kind 0), ex2 (kind 1), 4-byte shared-memory accesses
    // (kind 2: a load and a store per step)
    const double steps = (double)blocks * kThreads * (double)iters * kChains;
    return kind == 2 ? 2.0 * steps : steps;
}

extern "C" lsv2_status lsv2_rate_probe(int32_t kind, int64_t iters, int32_t blocks, float* sink, void* stream)
{
    if (iters < 1 || blocks < 1 || !sink || kind < 0 || kind > 2) return LSV2_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == 0) fma_probe<<<blocks, kThreads, 0, s>>>(iters, 1.0f, sink);
    else if (kind == 1) ex2_probe<<<blocks, kThreads, 0, s>>>(iters, 1.0f, sink);
    else smem_probe<<<blocks, kThreads, 0, s>>>(iters, 1.0f, sink);
    return cudaGetLastError() == cudaSuccess ? LSV2_OK : LSV2_ERR_CUDA;
}
