// peak.cu -- measured FP64 fused multiply-add rate of the current GPU, the denominator of the
// FP64-pipe roofline of the FP64 kernels (the bench reports their algorithmic flops against it).
//
// Every thread runs CHAINS independent chains x <- fma(x, a, b) (a slightly below 1, so the chains
// stay finite), enough per warp to hide the pipe's latency; the grid fills every SM to the
// occupancy the kernel allows.  Only FP64 FMAs sit in the timed loop; the loop counter and branch
// run on the integer pipes.  Timed with CUDA events on the caller's stream; nothing is allocated
// beyond one small result array, freed before the call returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "feod.h"

namespace {

constexpr int CHAINS = 16;
constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) k_dfma_rate(double *out, int iters, double a, double b)
{
    double x[CHAINS];
    const double seed = 1.0 + 1e-3 * (double)(threadIdx.x + blockDim.x * blockIdx.x);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = seed + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[threadIdx.x + (size_t)blockDim.x * blockIdx.x] = s;
}

}  // namespace

extern "C" fe_status fe_measure_fp64_peak(int reps, double *tflops_best, double *tflops_median, void *stream)
{
    if (reps < 1 || !tflops_best) return FE_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FE_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FE_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_rate, PEAK_THREADS, 0) != cudaSuccess)
        return FE_ERR_CUDA;
    const int grid = sms * std::max(per_sm, 1);
    const int iters = 4096;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)grid * PEAK_THREADS) != cudaSuccess) return FE_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fe_status s = FE_OK;
    std::vector<double> rate;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = FE_ERR_CUDA;
    const double flops = 2.0 * CHAINS * (double)iters * grid * PEAK_THREADS;
    for (int r = -2; r < reps && s == FE_OK; ++r) {         // two untimed warm-up launches
        cudaEventRecord(e0, st);
        k_dfma_rate<<<grid, PEAK_THREADS, 0, st>>>(out, iters, 0.999999, 1e-6);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) { s = FE_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r >= 0 && ms > 0.f) rate.push_back(flops / (ms * 1e-3) / 1e12);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (s != FE_OK) return s;
    if (rate.empty()) return FE_ERR_CUDA;
    std::sort(rate.begin(), rate.end());
    *tflops_best = rate.back();
    if (tflops_median) *tflops_median = rate[rate.size() / 2];
    return FE_OK;
}
