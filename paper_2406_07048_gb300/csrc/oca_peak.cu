// FP64 arithmetic rate of this GPU, measured: the denominator of the
// trajectory kernel's roofline.  That kernel's backward Riccati recursion and
// forward sweep run in FP64, whose rate on this part is a small fraction of
// the FP32 rate and is not among the copy-bandwidth and GEMM peaks measured
// for the rest of the path.
#include <cuda_runtime.h>

#include "oca.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// Every thread advances kChains independent recurrences x <- a x + b by one
// FMA each per iteration; the sum is stored only under a condition the
// recurrences (which stay near b / (1 - a) = 1) never meet, so that the
// compiler keeps them.
__global__ void k_fp64_fma(double *sink, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0) sink[0] = s;
}

}  // namespace

extern "C" oca_status oca_fp64_peak(int device, double *gflops) {
    if (!gflops) return OCA_ERR_INVALID_ARGUMENT;
    *gflops = 0.0;
    int prev = 0, n_sm = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return OCA_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return OCA_ERR_INVALID_ARGUMENT;
    oca_status out = OCA_OK;
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int threads = 256, iters = 8192;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        out = OCA_ERR_CUDA;
    } else {
        const int blocks = 8 * n_sm;  // 2,048 threads per SM
        float best = 0.f;
        for (int rep = 0; rep < 4 && out == OCA_OK; ++rep) {  // the first run warms up
            cudaEventRecord(e0);
            k_fp64_fma<<<blocks, threads>>>(sink, iters, 0.999999, 1e-6);
            cudaEventRecord(e1);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                out = OCA_ERR_CUDA;
            } else if (rep > 0 && (best == 0.f || ms < best)) {
                best = ms;
            }
        }
        if (out == OCA_OK && best > 0.f)
            *gflops = 2.0 * kChains * (double)iters * (double)blocks * threads / (best * 1e-3) / 1e9;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaSetDevice(prev);
    return out;
}
