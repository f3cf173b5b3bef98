// mc_peaks.cu -- throughput microbenchmarks of the execution units the
// wave-propagation kernels are bound by: FP32 fused multiply-add (scalar and
// packed pairs), FP64 fused multiply-add, the special-function unit
// (reciprocal square root, reciprocal), integer multiply-adds, and the
// warp-instruction issue rate (from a stream of independent FP32
// multiply-adds, which issue at the full rate).  They give the measured denominators of the
// arithmetic rooflines the benchmark reports (the HBM denominator is a copy
// measured elsewhere).  Each kernel runs NCHAIN independent dependency chains
// per thread so that latency is hidden and only throughput limits it; the
// caller times the launch with events on its stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mc_internal.h"

namespace mc {
namespace {

constexpr int NCHAIN = 8;
// steps of every chain per loop iteration, so that the loop's own counter,
// compare and branch are about 2% of the instructions
constexpr int NREP = 16;
constexpr int PEAK_THREADS = 256;

// A value the compiler cannot predict, so that no chain folds away; the
// results reach memory only if they take an impossible value.
__device__ __forceinline__ float seedf(int k) { return 1.0f + 1e-3f * float(threadIdx.x + k); }

__global__ void __launch_bounds__(PEAK_THREADS) peak_ffma(int64_t iters, float* sink)
{
    float a[NCHAIN];
    const float b = 0.999f, c = 1e-4f * float(blockIdx.x & 7);
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) a[k] = seedf(k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < NREP; r++)
#pragma unroll
        for (int k = 0; k < NCHAIN; k++) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) s += a[k];
    if (s == -1.0f) *sink = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_ffma2(int64_t iters, float* sink)
{
    float2 a[NCHAIN];
    const float2 b = make_float2(0.999f, 0.998f), c = make_float2(1e-4f * float(blockIdx.x & 7), 2e-4f);
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) a[k] = make_float2(seedf(k), seedf(k + NCHAIN));
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < NREP; r++)
#pragma unroll
        for (int k = 0; k < NCHAIN; k++) a[k] = __ffma2_rn(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) s += a[k].x + a[k].y;
    if (s == -1.0f) *sink = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_dfma(int64_t iters, float* sink)
{
    double a[NCHAIN];
    const double b = 0.999, c = 1e-4 * double(blockIdx.x & 7);
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) a[k] = double(seedf(k));
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < NREP; r++)
#pragma unroll
        for (int k = 0; k < NCHAIN; k++) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) s += a[k];
    if (s == -1.0) *sink = float(s);
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// x -> 1/sqrt(x) maps [0.5, 2] into itself, so the chains stay finite
__global__ void __launch_bounds__(PEAK_THREADS) peak_rsqrt(int64_t iters, float* sink)
{
    float a[NCHAIN];
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) a[k] = seedf(k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < NREP; r++)
#pragma unroll
        for (int k = 0; k < NCHAIN; k++) a[k] = rsqrt_approx(a[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) s += a[k];
    if (s == -1.0f) *sink = s;
}

// x -> 1/x + 1/2 maps [0.5, 2.5] into itself and never returns to its
// argument, so no pair of steps can be folded away
__global__ void __launch_bounds__(PEAK_THREADS) peak_rcp(int64_t iters, float* sink)
{
    float a[NCHAIN];
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) a[k] = seedf(k);
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < NREP; r++)
#pragma unroll
        for (int k = 0; k < NCHAIN; k++) a[k] = rcp_approx(a[k]) + 0.5f;
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) s += a[k];
    if (s == -1.0f) *sink = s;
}

// integer multiply-add: a -> a a + c (a quadratic map, so no chain of steps
// can be composed into one by the compiler, as affine maps could)
__global__ void __launch_bounds__(PEAK_THREADS) peak_iadd(int64_t iters, float* sink)
{
    uint32_t a[NCHAIN];
    const uint32_t c = threadIdx.x | 1u;
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) a[k] = threadIdx.x * 7u + k + blockIdx.x;
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < NREP; r++)
#pragma unroll
        for (int k = 0; k < NCHAIN; k++) a[k] = a[k] * a[k] + c;
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < NCHAIN; k++) s ^= a[k];
    if (s == 0x12345678u) *sink = float(s);
}

}  // namespace
}  // namespace mc

using namespace mc;

extern "C" mc_status mc_peak_run(int32_t kind, int32_t blocks_per_sm, int64_t iters, float* sink,
                                 double* ops_out, void* stream)
{
    if (kind < 0 || kind >= MC_PEAK_NKINDS) return set_error(MC_EINVAL, "unknown peak kind %d", kind);
    if (blocks_per_sm < 1 || blocks_per_sm > 64) return set_error(MC_EINVAL, "blocks_per_sm out of range");
    if (iters < 1 || iters > (1LL << 40)) return set_error(MC_EINVAL, "iters out of range");
    if (!sink) return set_error(MC_EINVAL, "sink must be a device pointer");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    const int blocks = sms * blocks_per_sm;
    const double threads = double(blocks) * PEAK_THREADS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // operations per launch: flops for the multiply-adds (2 per lane and
    // fma), results for the special functions, thread instructions of the
    // timed loop body for the integer and issue kernels
    double per = 0.0;
    switch (kind) {
    case MC_PEAK_FFMA:
        peak_ffma<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
        per = 2.0 * NCHAIN;
        break;
    case MC_PEAK_FFMA2:
        peak_ffma2<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
        per = 4.0 * NCHAIN;
        break;
    case MC_PEAK_DFMA:
        peak_dfma<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
        per = 2.0 * NCHAIN;
        break;
    case MC_PEAK_RSQRT:
        peak_rsqrt<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
        per = NCHAIN;
        break;
    case MC_PEAK_RCP:
        peak_rcp<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
        per = NCHAIN;
        break;
    case MC_PEAK_IADD:
        peak_iadd<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
        per = NCHAIN;
        break;
    default:
        // independent FP32 multiply-adds issue at the full rate of one warp
        // instruction per scheduler and cycle: thread instructions of that
        // stream are the issue ceiling of the step kernels
        peak_ffma<<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
        per = NCHAIN;
        break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "peak kernel launch");
    if (ops_out) *ops_out = per * NREP * threads * double(iters);
    return MC_OK;
}
