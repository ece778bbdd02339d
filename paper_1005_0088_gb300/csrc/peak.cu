// FP64 (DFMA) throughput of the current GPU, measured on the device: the denominator of the
// FP64 roofline fractions of the plain FP64 path (GEMMs, pivot sweeps, solves).  GB300 has no
// FP64 tensor path, so the CUDA-core DFMA rate is the ceiling of every FP64 kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "ndsi.h"
#include "handle.hpp"

namespace ndsi {
namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hides the DFMA latency)
constexpr int kPeakThreads = 256;

// Every thread runs kChains independent x <- x * a + b chains for `iters` steps: 2 * kChains *
// iters flops per thread.  The sum is stored so that the chains are not removed.
__global__ void __launch_bounds__(kPeakThreads) k_dfma_rate(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + 1) + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int fp64_rate(cudaStream_t st, double* tflops_out) {
    int dev = 0, sms = 0;
    NDSI_CK(cudaGetDevice(&dev));
    NDSI_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;   // 2048 threads per SM
    const int iters = 8192;
    DevBuf out;
    NDSI_CK(out.alloc(sizeof(double) * blocks * kPeakThreads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NDSI_CK(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    double best = 0.0;
    // a warm-up launch, then the best of five timed launches
    for (int rep = 0; rep < 6 && err == cudaSuccess; ++rep) {
        err = cudaEventRecord(e0, st);
        if (err == cudaSuccess) {
            k_dfma_rate<<<blocks, kPeakThreads, 0, st>>>(out.as<double>(), iters, 0.999999, 1e-7);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0 && ms > 0.0f) {
            const double flops = 2.0 * kChains * static_cast<double>(iters) * blocks * kPeakThreads;
            best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    NDSI_CK(err);
    *tflops_out = best;
    return NDSI_OK;
}

}  // namespace ndsi

using namespace ndsi;

extern "C" int ndsi_fp64_peak(double* tflops_out, void* stream) {
    if (!tflops_out) return fail(NDSI_ERR_INVALID, "ndsi_fp64_peak: NULL output");
    return fp64_rate(static_cast<cudaStream_t>(stream), tflops_out);
}
