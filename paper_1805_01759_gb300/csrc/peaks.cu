// Arithmetic-pipe microbenchmarks: the peaks against which the iteration kernel's and
// the refit's rooflines are stated (the FP32 FMA pipe, its packed-pair form, the FP64
// FMA pipe and the special-function unit).  Each thread runs `iters` trips of a loop of
// independent dependency chains, so that the pipe, not the latency of one chain, bounds
// the rate; the results are folded into one value per thread and written to a sink so
// that nothing is optimised away.  Not part of the paper's method.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bpdn_bench.h"
#include "bpdn_internal.h"

namespace bpdn {
namespace {

constexpr int kChains = 8;  // independent accumulators per thread

// FFMA: 8 chains x 2 flops per trip
__global__ void k_ffma(int64_t iters, float a, float b, float *sink)
{
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = (float)(threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FFMA2 (fma.rn.f32x2): 8 chains x 2 lanes x 2 flops per trip
__global__ void k_ffma2(int64_t iters, float a, float b, float *sink)
{
    unsigned long long acc[kChains];
    float2 av = make_float2(a, a), bv = make_float2(b, b);
    const unsigned long long ap = *reinterpret_cast<unsigned long long *>(&av);
    const unsigned long long bp = *reinterpret_cast<unsigned long long *>(&bv);
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float2 v = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
        acc[c] = *reinterpret_cast<unsigned long long *>(&v);
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[c]) : "l"(ap), "l"(bp));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float2 v = *reinterpret_cast<float2 *>(&acc[c]);
        s += v.x + v.y;
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// DFMA: 8 chains x 2 flops per trip
__global__ void k_dfma(int64_t iters, double a, double b, float *sink)
{
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = (double)(threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = fma(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// MUFU: 8 chains x one reciprocal square root per trip (the prox's |v|^-1)
__global__ void k_mufu(int64_t iters, float a, float b, float *sink)
{
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = 1.f + (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = rsqrtf(acc[c]) + b;
    }
    float s = a;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace bpdn

using namespace bpdn;

extern "C" int bpdn_bench_peak(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, float *d_sink,
                               double *ops_per_thread_trip, void *cuda_stream)
{
    if (kind < 0 || kind > 3)
        return set_error(BPDN_EINVAL, "kind must be 0 (FFMA), 1 (FFMA2), 2 (DFMA) or 3 (MUFU)");
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1)
        return set_error(BPDN_EINVAL, "blocks >= 1, threads a multiple of 32 in [32, 1024], iters >= 1");
    if (!d_sink)
        return set_error(BPDN_EINVAL, "sink is NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double ops = 0.0;
    switch (kind) {
    case 0: k_ffma<<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, d_sink); ops = 2.0 * kChains; break;
    case 1: k_ffma2<<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, d_sink); ops = 4.0 * kChains; break;
    case 2: k_dfma<<<blocks, threads, 0, s>>>(iters, 0.999, 1e-3, d_sink); ops = 2.0 * kChains; break;
    default: k_mufu<<<blocks, threads, 0, s>>>(iters, 0.f, 0.5f, d_sink); ops = (double)kChains; break;
    }
    if (ops_per_thread_trip)
        *ops_per_thread_trip = ops;
    return check_cuda(cudaGetLastError(), "peak kernel");
}
