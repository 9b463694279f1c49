// Arithmetic peaks of the CUDA cores, measured with our own kernels: long
// chains of dependent fused multiply-adds, many independent chains per thread
// and enough threads to fill every SM.  Used only to state roofline
// denominators for kernels bound by plain ALU arithmetic (the FP64 path, the
// FP32 epilogue of the tensor-core path); nothing in the evaluation path calls
// this library.
//
//   kind 0  FP64 fma.rn.f64
//   kind 1  FP32 fma.rn.f32
//   kind 2  FP32 fma.rn.f32x2 (packed pair: two FMAs per instruction)
//
// peak_probe(kind, iters, &tflops, &ms): one warm-up launch, then one timed
// launch (CUDA events on a private stream); tflops counts 2 flops per FMA.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma64(int iters, double seed, double *out)
{
    double a[kChains];
    const double b = 1.0 - 1e-9 * (threadIdx.x & 7), c = 1e-12 * seed;
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = seed + i;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < kChains; i++) a[i] = fma(a[i], b, c);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i];
    if (s == 12345.678) out[blockIdx.x] = s;  // never true: keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_fma32(int iters, float seed, float *out)
{
    float a[kChains];
    const float b = 1.0f - 1e-6f * (threadIdx.x & 7), c = 1e-7f * seed;
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = seed + i;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < kChains; i++) a[i] = fmaf(a[i], b, c);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_fma32x2(int iters, float seed, float *out)
{
    unsigned long long a[kChains], b, c;
    const float bf = 1.0f - 1e-6f * (threadIdx.x & 7), cf = 1e-7f * seed;
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(bf), "f"(bf));
    asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(cf), "f"(cf));
#pragma unroll
    for (int i = 0; i < kChains; i++) {
        const float x = seed + i, y = seed - i;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[i]) : "f"(x), "f"(y));
    }
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int i = 0; i < kChains; i++) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(b), "l"(c));
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; i++) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[i]));
        s += x + y;
    }
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int peak_probe(int kind, int iters, double *tflops, double *ms_out)
{
    if (kind < 0 || kind > 2 || iters < 1 || !tflops) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -5;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    void *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) return -2;
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(e0, s);
        if (kind == 0) k_fma64<<<blocks, kThreads, 0, s>>>(iters, 1.5, (double *)out);
        else if (kind == 1) k_fma32<<<blocks, kThreads, 0, s>>>(iters, 1.5f, (float *)out);
        else k_fma32x2<<<blocks, kThreads, 0, s>>>(iters, 1.5f, (float *)out);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    const int rc = cudaGetLastError() == cudaSuccess ? 0 : -5;
    const double fmas = (double)blocks * kThreads * kChains * iters * (kind == 2 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(out);
    return rc;
}
