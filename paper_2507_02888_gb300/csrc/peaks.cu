// Arithmetic peaks of the current GPU, measured: the denominators of the
// ALU-bound rooflines of the mixed (FP32 FMA, MUFU) and plain (FP64 FMA)
// forms.  Each thread runs kChains independent multiply-add chains (enough
// independent work to hide the pipeline latency) over a grid of a few CTAs
// per SM; the result is stored so that no chain can be optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ewald.h"

namespace {

constexpr int kChains = 8, kThreads = 256, kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T seed, T *out) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T m = (T)0.999999, s = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] * m + s;  // one FMA
    }
    T t = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// reciprocal square roots on the special-function unit (one op per step)
__global__ void __launch_bounds__(kThreads) k_mufu_chains(int iters, float seed, float *out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
            a[c] = y;
        }
    }
    float t = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

template <typename F>
cudaError_t best_ms(F launch, cudaStream_t st, float *ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (e) return e;
    *ms = 1e30f;
    for (int rep = 0; rep < 4 && !e; ++rep) {  // the first run warms up
        e = cudaEventRecord(e0, st);
        if (!e) launch();
        if (!e) e = cudaGetLastError();
        if (!e) e = cudaEventRecord(e1, st);
        if (!e) e = cudaEventSynchronize(e1);
        float t = 0;
        if (!e) e = cudaEventElapsedTime(&t, e0, e1);
        if (!e && rep) *ms = std::min(*ms, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" int ewald_measure_peaks(double *fp32_tflops, double *fp64_tflops, double *mufu_tops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return EWALD_ERR_CUDA;
    const int grid = sms * kBlocksPerSm;
    const double threads = (double)grid * kThreads;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) return EWALD_ERR_CUDA;
    void *buf = nullptr;
    if ((e = cudaMalloc(&buf, (size_t)grid * kThreads * sizeof(double)))) {
        cudaStreamDestroy(st);
        return EWALD_ERR_OOM;
    }
    float ms = 0;
    const int it32 = 4096, it64 = 256, itmu = 1024;
    if (!e && fp32_tflops) {
        e = best_ms([&] { k_fma_chains<float><<<grid, kThreads, 0, st>>>(it32, 1.0f, (float *)buf); }, st, &ms);
        if (!e) *fp32_tflops = 2.0 * kChains * it32 * threads / (ms * 1e-3) / 1e12;
    }
    if (!e && fp64_tflops) {
        e = best_ms([&] { k_fma_chains<double><<<grid, kThreads, 0, st>>>(it64, 1.0, (double *)buf); }, st, &ms);
        if (!e) *fp64_tflops = 2.0 * kChains * it64 * threads / (ms * 1e-3) / 1e12;
    }
    if (!e && mufu_tops) {
        e = best_ms([&] { k_mufu_chains<<<grid, kThreads, 0, st>>>(itmu, 2.0f, (float *)buf); }, st, &ms);
        if (!e) *mufu_tops = (double)kChains * itmu * threads / (ms * 1e-3) / 1e12;
    }
    cudaFree(buf);
    cudaStreamDestroy(st);
    return e ? EWALD_ERR_CUDA : EWALD_OK;
}
