// FMA-throughput probe (include/m2l_peaks.h): every thread runs 8 independent FMA chains, 16
// trips of the 8 per loop iteration, so the loop's own instructions are about 2% of those issued.
// The grid holds 8 CTAs of 256 threads per SM, 64 resident warps, enough to hide the FMA latency
// on every sub-partition. The result of each thread is stored, so no chain can be removed.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/m2l_peaks.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(T *out, long long iters, T mul, T add) {
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], mul, add);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

template <class T>
int run(long long iters, int reps, double *best, double *median, double *ms_best) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -3;
    const int blocks = sms * 8;
    T *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess) return -3;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // mul slightly below one and a small add keep every value finite and normal
    const T mul = (T)0.9999999, add = (T)1e-7;
    fma_chains_kernel<T><<<blocks, kThreads>>>(out, iters, mul, add);
    std::vector<double> rates;
    double msb = 1e30;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a);
        fma_chains_kernel<T><<<blocks, kThreads>>>(out, iters, mul, add);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kThreads;
        rates.push_back(flops / (ms * 1e-3) / 1e12);
        msb = std::min(msb, (double)ms);
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return -3;
    std::sort(rates.begin(), rates.end());
    if (best) *best = rates.back();
    if (median) *median = rates[rates.size() / 2];
    if (ms_best) *ms_best = msb;
    return 0;
}

}  // namespace

extern "C" int m2l_fma_peak(int fp64, long long iters, int reps, double *best, double *median, double *ms_best) {
    if (iters < 1 || reps < 1 || reps > 64) return -1;
    return fp64 ? run<double>(iters, reps, best, median, ms_best) : run<float>(iters, reps, best, median, ms_best);
}
