// Throughput probes for the roofline denominators of the ALU-bound kernels: FP32 FFMA,
// packed FP32x2 FFMA2, FP64 DFMA, the special-function unit (sine) and TF32 mma.sync.
// Each probe runs independent dependency chains on every SM for a few milliseconds and
// reports operations per second measured with CUDA events. Built as its own library: the
// IFGF library does not depend on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ifgf_peaks.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void k_ffma(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live
}

__global__ void k_ffma2(float* out, int iters, float a, float b) {
    float2 x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = make_float2(threadIdx.x * 1e-3f + j, j * 0.5f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
    if (s == 1234.5f) out[blockIdx.x] = s;
}

__global__ void k_dfma(float* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == 1234.5) out[blockIdx.x] = (float)s;
}

__global__ void k_sin(float* out, int iters) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = __sinf(x[j]);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == 1234.5f) out[blockIdx.x] = s;
}

__global__ void k_mma_tf32(float* out, int iters) {
    constexpr int kAcc = 4;
    float c[kAcc][4];
#pragma unroll
    for (int j = 0; j < kAcc; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[j][e] = 0.f;
    const uint32_t a0 = __float_as_uint(1.0f + threadIdx.x * 1e-3f), a1 = __float_as_uint(0.5f);
    const uint32_t b0 = __float_as_uint(0.25f), b1 = __float_as_uint(-0.125f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kAcc; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                : "r"(a0), "r"(a1), "r"(a1), "r"(a0), "r"(b0), "r"(b1));
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kAcc; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
    if (s == 1234.5f) out[blockIdx.x] = s;
}

template <class F>
double time_ms(F launch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

extern "C" {

// out[0] FP32 FFMA TFLOP/s, out[1] FP32x2 FFMA2 TFLOP/s, out[2] FP64 DFMA TFLOP/s,
// out[3] MUFU sine Gop/s, out[4] TF32 mma.sync (m16n8k8) TFLOP/s, out[5] SM count.
// Returns 0, or the CUDA error code of the first failing call.
int ifgf_peaks_measure(double* out) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    float* sink = nullptr;
    const int blocks = sms * 8;
    e = cudaMalloc(&sink, sizeof(float) * blocks);
    if (e != cudaSuccess) return (int)e;
    const double threads = (double)blocks * kThreads;
    const int it = 1 << 14;
    double ms = time_ms([&] { k_ffma<<<blocks, kThreads>>>(sink, it, 0.999f, 1e-3f); });
    out[0] = threads * it * kChains * 2.0 / (ms * 1e-3) / 1e12;
    ms = time_ms([&] { k_ffma2<<<blocks, kThreads>>>(sink, it, 0.999f, 1e-3f); });
    out[1] = threads * it * kChains * 4.0 / (ms * 1e-3) / 1e12;
    const int itd = 1 << 10;
    ms = time_ms([&] { k_dfma<<<blocks, kThreads>>>(sink, itd, 0.999, 1e-3); });
    out[2] = threads * itd * kChains * 2.0 / (ms * 1e-3) / 1e12;
    const int its = 1 << 12;
    ms = time_ms([&] { k_sin<<<blocks, kThreads>>>(sink, its); });
    out[3] = threads * its * kChains / (ms * 1e-3) / 1e9;
    const int itm = 1 << 12;
    ms = time_ms([&] { k_mma_tf32<<<blocks, kThreads>>>(sink, itm); });
    out[4] = threads / 32.0 * itm * 4 * (16.0 * 8 * 8 * 2) / (ms * 1e-3) / 1e12;
    out[5] = sms;
    e = cudaGetLastError();
    cudaFree(sink);
    return (int)e;
}

}  // extern "C"
