// peaks.cu -- arithmetic-rate probes for the roofline denominators.
//
// The FP64 chain is bound by the GPU's FP64 rate and the double-float chain
// by its FP32 pipe, so their roofline fractions need measured arithmetic
// ceilings next to the measured copy bandwidth.  Each probe is one kernel of
// long dependent chains of a single instruction kind (16 independent chains
// per thread, 8 blocks of 256 threads per SM), timed with CUDA events on the
// caller's stream.  The paper has no counterpart: these are measurement aids.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/vloc.h"

namespace {

constexpr int kChains = 16;
constexpr int kBlockThreads = 256;
constexpr int kBlocksPerSM = 8;

// x <- x * b + c (FMA kinds) or x <- x + c (add kinds); b < 1 keeps the
// chains bounded.  The sum of the chains is stored so nothing is dead code.
__global__ void __launch_bounds__(kBlockThreads) k_peak_dfma(long long iters, double b, double c, double* sink) {
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1e-3 * (threadIdx.x + j);
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], b, c);
    double s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == 12345.678) sink[0] = s;  // never true; keeps the chains live
}
__global__ void __launch_bounds__(kBlockThreads) k_peak_dadd(long long iters, double b, double c, double* sink) {
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1e-3 * (threadIdx.x + j);
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = x[j] + ((i & 1) ? c : -c);
    double s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == 12345.678) sink[0] = s + b;
}
__global__ void __launch_bounds__(kBlockThreads) k_peak_ffma(long long iters, float b, float c, double* sink) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1e-3f * (threadIdx.x + j);
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], b, c);
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == 12345.678f) sink[0] = s;
}
__global__ void __launch_bounds__(kBlockThreads) k_peak_ffma2(long long iters, float b, float c, double* sink) {
    float2 x[kChains];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = make_float2(1e-3f * (threadIdx.x + j), 2e-3f * (threadIdx.x + j));
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], bb, cc);
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
    if (s == 12345.678f) sink[0] = s;
}
__global__ void __launch_bounds__(kBlockThreads) k_peak_fadd2(long long iters, float b, float c, double* sink) {
    float2 x[kChains];
    const float2 cp = make_float2(c, c), cm = make_float2(-c, -c);
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = make_float2(1e-3f * (threadIdx.x + j), 2e-3f * (threadIdx.x + j));
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = __fadd2_rn(x[j], (i & 1) ? cp : cm);
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
    if (s == 12345.678f) sink[0] = s + b;
}

}  // namespace

extern "C" int vloc_alu_peak(int kind, int64_t iters, void* sink, double* flops, double* ms, void* stream) {
    if (kind < 0 || kind >= VLOC_PEAK_NKINDS || iters <= 0 || !sink || !flops || !ms) return VLOC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VLOC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VLOC_ERR_CUDA;
    const unsigned grid = (unsigned)(nsm * kBlocksPerSM);
    // FLOPs per chain step: FMA 2, add 1; paired kinds do two of them
    const double per = (kind == VLOC_PEAK_DFMA || kind == VLOC_PEAK_FFMA) ? 2.0
                       : kind == VLOC_PEAK_FFMA2                            ? 4.0
                       : kind == VLOC_PEAK_FADD2                            ? 2.0
                                                                            : 1.0;
    *flops = per * kChains * (double)iters * grid * kBlockThreads;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return VLOC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return VLOC_ERR_CUDA; }
    double* sk = (double*)sink;
    cudaEventRecord(e0, st);
    switch (kind) {
        case VLOC_PEAK_DFMA: k_peak_dfma<<<grid, kBlockThreads, 0, st>>>(iters, 0.999999, 1e-7, sk); break;
        case VLOC_PEAK_DADD: k_peak_dadd<<<grid, kBlockThreads, 0, st>>>(iters, 0.999999, 1e-7, sk); break;
        case VLOC_PEAK_FFMA: k_peak_ffma<<<grid, kBlockThreads, 0, st>>>(iters, 0.9999f, 1e-5f, sk); break;
        case VLOC_PEAK_FFMA2: k_peak_ffma2<<<grid, kBlockThreads, 0, st>>>(iters, 0.9999f, 1e-5f, sk); break;
        default: k_peak_fadd2<<<grid, kBlockThreads, 0, st>>>(iters, 0.9999f, 1e-5f, sk); break;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return VLOC_ERR_CUDA;
    *ms = t;
    return VLOC_OK;
}
