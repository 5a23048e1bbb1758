// ddsg_probe.cu -- measured FMA peaks of the device (no paper counterpart):
// the denominators of the evaluation kernels' ALU rooflines.
//
// Every thread runs 8 independent FMA chains held in registers; the grid
// fills every SM with 8 warps per scheduler. FLOPs = 2 per FMA (4 per paired
// FP32 FMA). The launch is timed with CUDA events after one warm-up launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ddsg_alloc.h"
#include "ddsg_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T a, T b, T *out) {
    T c[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) c[j] = (T)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) c[j] = fma(c[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += c[j];
    if (s == (T)-1.2345) out[0] = s;   // keeps the chains live; never true for these inputs
}

// paired FP32: fma.rn.f32x2 on register pairs
__global__ void __launch_bounds__(kThreads) fma2_chain_kernel(int iters, float a, float b, float *out) {
    uint64_t c[kChains], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        const float x = (float)(threadIdx.x + j);
        asm("mov.b64 %0, {%1, %2};" : "=l"(c[j]) : "f"(x), "f"(x + 0.5f));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(c[j]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(c[j]));
        s += lo + hi;
    }
    if (s == -1.2345f) out[0] = s;
}

}  // namespace

// kind: 0 = FP64 fma, 1 = FP32 fmaf, 2 = paired FP32 (fma.rn.f32x2). Synchronous.
extern "C" int ddsg_probe_fma(int kind, double *tflops, double *ms_out) {
    if (!tflops || kind < 0 || kind > 2) return ddsg::set_error(DDSG_ERR_ARG, "ddsg_probe_fma: bad argument");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return ddsg::set_error(DDSG_ERR_CUDA, "ddsg_probe_fma: no device");
    }
    void *out = nullptr;
    if (ddsg::dev_alloc(&out, 16) != cudaSuccess) {
        cudaGetLastError();
        return ddsg::set_error(DDSG_ERR_OOM, "ddsg_probe_fma: device memory unavailable");
    }
    const int blocks = sms * 8;                  // 8 blocks of 8 warps per SM: 16 warps per scheduler
    const int iters = kind == 0 ? 1 << 12 : 1 << 16;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {          // the first launch warms up
        cudaEventRecord(e0);
        if (kind == 0) fma_chain_kernel<double><<<blocks, kThreads>>>(iters, 0.999999, 1e-7, (double *)out);
        else if (kind == 1) fma_chain_kernel<float><<<blocks, kThreads>>>(iters, 0.999999f, 1e-7f, (float *)out);
        else fma2_chain_kernel<<<blocks, kThreads>>>(iters, 0.999999f, 1e-7f, (float *)out);
        cudaEventRecord(e1);
    }
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) {
        cudaGetLastError();
        return ddsg::set_error(DDSG_ERR_CUDA, "ddsg_probe_fma: the probe launch failed");
    }
    const double fmas = (double)blocks * kThreads * kChains * iters * (kind == 2 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return DDSG_OK;
}
