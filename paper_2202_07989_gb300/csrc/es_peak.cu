// ALU throughput microbenchmark: the denominators of the flux kernels' roofline.
//
// The residual of the method is bound by the plain FP32 / FP64 pipes (no step is a dense
// contraction), so the roofline compares the flux kernels' flops per second with the
// measured fused multiply-add throughput of those pipes on the same GPU.  Every thread runs
// NCH independent multiply-add chains x <- x b + c (b slightly below 1, so the chains
// converge and never reach a subnormal or an infinity); the chain values are summed and
// written at the end, so no operation can be dropped.
#include "../../include/es.h"
#include "es_common.cuh"

namespace {

constexpr int PEAK_TPB = 256;
constexpr int NCH = 16;       // independent chains per thread

__global__ void __launch_bounds__(PEAK_TPB) peak_ffma_kernel(int iters, double* sink)
{
    float x[NCH];
    const float b = 0.999f, c = 1.0e-3f * (1 + (threadIdx.x & 7));
#pragma unroll
    for (int q = 0; q < NCH; ++q) x[q] = 0.5f + 0.01f * q + 1.0e-6f * threadIdx.x;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < NCH; ++q) x[q] = fmaf(x[q], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < NCH; ++q) s += x[q];
    sink[(long long)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

// paired FP32: each instruction forms two independent fused multiply-adds (FFMA2)
__global__ void __launch_bounds__(PEAK_TPB) peak_ffma2_kernel(int iters, double* sink)
{
    float2 x[NCH];
    const float2 b = make_float2(0.999f, 0.998f);
    const float2 c = make_float2(1.0e-3f * (1 + (threadIdx.x & 7)), 2.0e-3f);
#pragma unroll
    for (int q = 0; q < NCH; ++q) x[q] = make_float2(0.5f + 0.01f * q, 0.25f + 1.0e-6f * threadIdx.x);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < NCH; ++q) x[q] = __ffma2_rn(x[q], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < NCH; ++q) s += x[q].x + x[q].y;
    sink[(long long)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

__global__ void __launch_bounds__(PEAK_TPB) peak_dfma_kernel(int iters, double* sink)
{
    double x[NCH];
    const double b = 0.999, c = 1.0e-3 * (1 + (threadIdx.x & 7));
#pragma unroll
    for (int q = 0; q < NCH; ++q) x[q] = 0.5 + 0.01 * q + 1.0e-6 * threadIdx.x;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < NCH; ++q) x[q] = fma(x[q], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < NCH; ++q) s += x[q];
    sink[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" es_status es_alu_peak(int kind, int grid, int iters, double* sink, void* stream)
{
    if (kind < 0 || kind > 2 || grid <= 0 || iters <= 0 || !sink) return ES_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == 0) peak_ffma_kernel<<<grid, PEAK_TPB, 0, st>>>(iters, sink);
    else if (kind == 1) peak_ffma2_kernel<<<grid, PEAK_TPB, 0, st>>>(iters, sink);
    else peak_dfma_kernel<<<grid, PEAK_TPB, 0, st>>>(iters, sink);
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

extern "C" long long es_alu_peak_flops(int kind, int grid, int iters)
{
    if (kind < 0 || kind > 2 || grid <= 0 || iters <= 0) return 0;
    return (long long)grid * PEAK_TPB * iters * NCH * 2 * (kind == 1 ? 2 : 1);
}
