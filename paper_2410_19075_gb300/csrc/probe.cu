// Peak-throughput probes of the arithmetic pipes the stage kernels use, timed on
// the device so that the roofline denominators are measured on the GPU the
// library runs on (sim_probe_peak in include/sim.h).
//
//   kind 0  FP64 fused multiply-add (DFMA), the node right-hand sides and RK4
//   kind 1  64-bit unsigned multiply-high (mul.hi.u64), the fixed-point
//           elementary functions
//   kind 2  32-bit integer multiply-add (IMAD)
//   kind 3  int64 -> double conversion (cvt.rn.f64.s64): on GB300 it runs at
//           the FP64 rate, so a conversion costs as much as a DFMA
//   kind 4  64-bit signed multiply-high (mul.hi.s64), about 1.7 unsigned ones
//
// Every thread runs kChains independent dependent chains (enough instruction-
// level parallelism to cover the pipes' latency at full occupancy); the grid
// fills every SM several times.  One warm-up launch, then one timed launch
// bracketed by CUDA events on a private stream.  The result is written only if
// it takes an impossible value, so nothing can be optimised away.
#include <cstdint>

#include "internal.h"
#include "sim.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) probe_dfma(int64_t iters, double a, double b, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_mulhi64(int64_t iters, uint64_t k, unsigned long long *sink)
{
    uint64_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0x9E3779B97F4A7C15ull * (threadIdx.x + 1 + 977 * c);
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __umul64hi(x[c], k) | 1ull;
    }
    uint64_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 2ull) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_imad32(int64_t iters, unsigned a, unsigned b, unsigned *sink)
{
    unsigned x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 7919u + 13u * c;
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 0xFFFFFFFEu && b == 0u) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_cvt(int64_t iters, unsigned long long *sink)
{
    uint64_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0x3FF0000000000000ull + 977ull * (threadIdx.x + 131 * c);
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = (uint64_t)__double_as_longlong(__ll2double_rn((long long)x[c]));
    }
    uint64_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 2ull) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_mulhi64s(int64_t iters, int64_t k, unsigned long long *sink)
{
    int64_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (int64_t)(0x9E3779B97F4A7C15ull * (threadIdx.x + 1 + 977 * c));
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __mul64hi(x[c], k) | 1;
    }
    int64_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 2) sink[0] = (unsigned long long)s;
}

} // namespace

extern "C" int sim_probe_peak(int kind, double *ops_per_s)
{
    if (!ops_per_s || kind < 0 || kind > 4) return simk::report_error(SIM_EINVAL, "sim_probe_peak: unknown kind");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return simk::report_cuda_error(e, "sim_probe_peak: device query");
    // Iterations per thread for roughly 20-80 ms per timed launch on a GB300.
    const int64_t iters = kind == 0 || kind == 3 ? 4096 : kind == 1 || kind == 4 ? 65536 : 262144;
    const unsigned grid = (unsigned)sms * 8;
    void *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&sink, 64);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) { // warm-up, then the timed launch
        e = cudaEventRecord(a, s);
        if (kind == 0)
            probe_dfma<<<grid, kProbeThreads, 0, s>>>(iters, 0.9999999, 1e-7, static_cast<double *>(sink));
        else if (kind == 1)
            probe_mulhi64<<<grid, kProbeThreads, 0, s>>>(iters, 0xF0E1D2C3B4A59687ull,
                                                          static_cast<unsigned long long *>(sink));
        else if (kind == 2)
            probe_imad32<<<grid, kProbeThreads, 0, s>>>(iters, 1664525u, 1013904223u, static_cast<unsigned *>(sink));
        else if (kind == 3)
            probe_cvt<<<grid, kProbeThreads, 0, s>>>(iters, static_cast<unsigned long long *>(sink));
        else
            probe_mulhi64s<<<grid, kProbeThreads, 0, s>>>(iters, (int64_t)0x70E1D2C3B4A59687ll,
                                                           static_cast<unsigned long long *>(sink));
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return simk::report_cuda_error(e, "sim_probe_peak");
    }
    const double ops = (double)grid * kProbeThreads * kChains * (double)iters;
    *ops_per_s = ops / (ms * 1e-3);
    return SIM_OK;
}
