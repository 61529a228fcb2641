// Diagnostics: CUDA-core FMA throughput (the ALU roofline denominator of the
// FP64- and FP32-bound kernels).  Many independent FMA chains per thread, grid
// sized to fill every SM; best of three timed runs with CUDA events.
#include "gtqa.h"
#include "gtqa_common.cuh"

#include <cuda_runtime.h>

namespace {

template <typename T, int NACC>
__global__ void fma_chains(T* sink, int iters, T a, T b) {
    T acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[k] = fma(acc[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < NACC; ++k) s += acc[k];
    if (s == (T)-1) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the work
}

template <typename T>
int measure(double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GTQA_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GTQA_ERR_CUDA;
    const int threads = 256, blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 1000 : 20000;
    constexpr int NACC = 8;
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * (size_t)threads * blocks) != cudaSuccess) return GTQA_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chains<T, NACC><<<blocks, threads>>>(sink, 10, (T)0.999, (T)0.001);
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        fma_chains<T, NACC><<<blocks, threads>>>(sink, iters, (T)0.999, (T)0.001);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return GTQA_ERR_CUDA;
    *tflops = 2.0 * NACC * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
    return GTQA_OK;
}

}  // namespace

extern "C" int gtqa_alu_peak(int32_t fp64, double* tflops_out) {
    if (!tflops_out) return GTQA_ERR_INVALID_ARG;
    return fp64 ? measure<double>(tflops_out) : measure<float>(tflops_out);
}

// Diagnostic: the Newton-refined reciprocal / rsqrt / sqrt used by the kernels next to
// CUDA's own 1/x, 1/sqrt(x) and sqrt(x), for accuracy tests.
namespace {
__global__ void math_check_kernel(int n, const double* x, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    out[6 * i + 0] = gtqa::nr_rcp(v);
    out[6 * i + 1] = 1.0 / v;
    out[6 * i + 2] = gtqa::nr_rsqrt(v);
    out[6 * i + 3] = 1.0 / sqrt(v);
    out[6 * i + 4] = gtqa::nr_sqrt(v);
    out[6 * i + 5] = sqrt(v);
}
}  // namespace

extern "C" int gtqa_math_check(int32_t n, const double* x, double* out) {
    if (n < 1 || !x || !out) return GTQA_ERR_INVALID_ARG;
    double *dx = nullptr, *dout = nullptr;
    if (cudaMalloc(&dx, sizeof(double) * n) != cudaSuccess) return GTQA_ERR_OOM;
    if (cudaMalloc(&dout, sizeof(double) * 6 * n) != cudaSuccess) {
        cudaFree(dx);
        return GTQA_ERR_OOM;
    }
    cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    math_check_kernel<<<(n + 127) / 128, 128>>>(n, dx, dout);
    cudaError_t e = cudaMemcpy(out, dout, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dout);
    return e == cudaSuccess ? GTQA_OK : GTQA_ERR_CUDA;
}

// Diagnostic: latency of the bounded grid barrier used by the phase kernels
// (cooperative launch, one block of `threads` per SM, `rounds` barriers).
namespace {
__global__ void barrier_bench_kernel(unsigned long long* cnt, int* err, int rounds) {
    gtqa::GridBarrier gb = gtqa::grid_barrier_init(cnt, err, gridDim.x);
    for (int r = 0; r < rounds; ++r)
        if (!gtqa::grid_sync(gb, 1LL << 22)) return;
}
}  // namespace

extern "C" int gtqa_barrier_bench(int32_t threads, int32_t rounds, double* us_per_barrier) {
    if (threads < 32 || threads > 1024 || rounds < 1 || !us_per_barrier) return GTQA_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GTQA_ERR_CUDA;
    unsigned long long* buf = nullptr;
    if (cudaMalloc(&buf, 2 * sizeof(unsigned long long)) != cudaSuccess) return GTQA_ERR_OOM;
    cudaMemset(buf, 0, 2 * sizeof(unsigned long long));
    unsigned long long* cnt = buf;
    int* err = reinterpret_cast<int*>(buf + 1);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        void* args[] = {&cnt, &err, &rounds};
        cudaEventRecord(e0);
        cudaLaunchCooperativeKernel((const void*)barrier_bench_kernel, dim3(sms), dim3(threads), args, 0, nullptr);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    int herr = 0;
    cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    const cudaError_t ce = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (ce != cudaSuccess) return GTQA_ERR_CUDA;
    if (herr) return herr;
    *us_per_barrier = best * 1e3 / rounds;
    return GTQA_OK;
}
