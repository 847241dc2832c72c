// peaks.cu -- throughput of the pipes the evaluation kernels run on, measured on the
// device at hand (a measurement utility of the library; the paper has no counterpart):
// scalar FP32 FMA, packed FP32x2 FMA, the MUFU reciprocal square root and FP64 FMA.
//
// Each thread runs kChains independent dependency chains, so that the pipe, not the
// latency of one chain, limits the rate; the grid holds 8 CTAs of 256 threads per SM.
// Every chain's result is stored, so no work can be dropped.  Rates are operations per
// second, an FMA (scalar, each lane of a packed one, or FP64) counting as one operation,
// as the roofline bookkeeping of the evaluation counts them.
#include <cuda_runtime.h>

#include <algorithm>

#include "context.h"

namespace nb {

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float* out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(float* out, int iters, float b, float c) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float mufu_rsqrt(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_mufu(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = mufu_rsqrt(a[k]);  // x -> x^(-1/2) tends to 1
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(double* out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace nb

using namespace nb;

extern "C" int nebem_peak_rates(nebem_ctx* ctx, double* rates) {
    if (!ctx || !rates) return fail(NEBEM_INVALID_ARG, "NULL argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const int blocks = 8 * c->props.multiProcessorCount;
    const double threads = (double)blocks * kPeakThreads;
    DevBuf out;
    if ((e = out.ensure(sizeof(double) * blocks * kPeakThreads)) != cudaSuccess) return cuda_fail(e, "peak buffer");
    cudaStream_t s = c->stream;
    // iterations per thread: about 1e10 operations per FP32 launch, 5e8 per FP64 launch
    const int it32 = 4096, itmufu = 1024, it64 = 256;
    const double ops[4] = {threads * it32 * kChains, threads * it32 * kChains * 2.0, threads * itmufu * kChains,
                           threads * it64 * kChains};
    double best[4] = {0.0, 0.0, 0.0, 0.0};
    for (int rep = 0; rep < 4; ++rep) {  // the first round warms up; the best of the rest counts
        for (int k = 0; k < 4; ++k) {
            if ((e = cudaEventRecord(c->ev0, s)) != cudaSuccess) return cuda_fail(e, "event");
            if (k == 0) k_peak_ffma<<<blocks, kPeakThreads, 0, s>>>(out.as<float>(), it32, 0.999999f, 1e-7f);
            if (k == 1) k_peak_ffma2<<<blocks, kPeakThreads, 0, s>>>(out.as<float>(), it32, 0.999999f, 1e-7f);
            if (k == 2) k_peak_mufu<<<blocks, kPeakThreads, 0, s>>>(out.as<float>(), itmufu);
            if (k == 3) k_peak_dfma<<<blocks, kPeakThreads, 0, s>>>(out.as<double>(), it64, 0.999999, 1e-7);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "peak kernel");
            if ((e = cudaEventRecord(c->ev1, s)) != cudaSuccess) return cuda_fail(e, "event");
            if ((e = cudaEventSynchronize(c->ev1)) != cudaSuccess) return cuda_fail(e, "peak kernel");
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, c->ev0, c->ev1)) != cudaSuccess) return cuda_fail(e, "event");
            if (rep > 0 && ms > 0.f) best[k] = std::max(best[k], ops[k] / (1e-3 * ms));
        }
    }
    for (int k = 0; k < 4; ++k) rates[k] = best[k];
    return NEBEM_OK;
}
