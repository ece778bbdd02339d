// Learned chemical-potential seed: spectral-moment features of (H, S) and a small MLP with
// hand-written forward, backward and Adam kernels (FP32).  The paper searches mu iteratively
// (Sec. II.C.3); this network only proposes the starting bracket for that search.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "ndsi.h"
#include "plan.hpp"

namespace ndsi {
namespace {

constexpr int kIn = NDSI_MLP_INPUTS, kHid = NDSI_MLP_HIDDEN;
constexpr int kNW1 = kHid * kIn, kNB1 = kHid, kNW2 = kHid * kHid, kNB2 = kHid, kNW3 = kHid, kNB3 = 1;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kNW1, kOffW2 = kOffB1 + kNB1, kOffB2 = kOffW2 + kNW2,
              kOffW3 = kOffB2 + kNB2, kOffB3 = kOffW3 + kNW3, kNParams = kOffB3 + kNB3;
static_assert(kNParams == NDSI_MLP_PARAMS, "parameter layout");
constexpr int kBatchBlock = 64;  // samples per CTA in the gradient kernel

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__device__ inline float uniform01(uint64_t seed, uint64_t i) {
    return static_cast<float>((splitmix64(seed ^ splitmix64(i)) >> 40) * (1.0 / 16777216.0));
}

// ------------------------------------------------------------------------ features -----------
// y(:, r) = c1 * (A x(:, r)) + c0 * x(:, r) - cp * p(:, r) for R vectors stored row-major
// [n][R]; A = (vals - shift*I) / scale on the CSR pattern.  Also partial sums of z . y per block
// (z = the Rademacher start vectors) for the stochastic trace.
__global__ void __launch_bounds__(256) k_cheb_step(const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col,
                                                   const double* __restrict__ vals, double shift,
                                                   double scale, int64_t n, int R,
                                                   const float* __restrict__ x,
                                                   const float* __restrict__ prev, float c1, float cp,
                                                   float* __restrict__ y, uint64_t seed,
                                                   double* __restrict__ partial) {
    __shared__ double red[256];
    const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    double dot = 0.0;
    if (idx < n * R) {
        const int64_t i = idx / R;
        const int r = static_cast<int>(idx % R);
        float acc = 0.f;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int64_t j = col[k];
            float a = static_cast<float>(vals[k]);
            if (j == i) a -= static_cast<float>(shift);
            acc += a * x[j * R + r];
        }
        acc = acc / static_cast<float>(scale);
        const float v = c1 * acc - (prev ? cp * prev[idx] : 0.f);
        y[idx] = v;
        const float z = (splitmix64(seed ^ splitmix64(static_cast<uint64_t>(idx))) & 1) ? 1.f : -1.f;
        dot = static_cast<double>(z) * v;
    }
    red[threadIdx.x] = dot;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_rademacher(int64_t count, uint64_t seed, float* __restrict__ z) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        z[i] = (splitmix64(seed ^ splitmix64(static_cast<uint64_t>(i))) & 1) ? 1.f : -1.f;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nblocks, double norm,
                               float* __restrict__ out) {
    __shared__ double red[256];
    double v = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v += partial[i];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = static_cast<float>(red[0] * norm);
}

// ----------------------------------------------------------------------------- MLP -----------
__device__ __forceinline__ void mlp_forward_one(const float* __restrict__ P, const float* x, float* h1,
                                                float* h2, float& y) {
    for (int j = 0; j < kHid; ++j) {
        float a = P[kOffB1 + j];
        for (int i = 0; i < kIn; ++i) a = fmaf(P[kOffW1 + j * kIn + i], x[i], a);
        h1[j] = tanhf(a);
    }
    for (int j = 0; j < kHid; ++j) {
        float a = P[kOffB2 + j];
        for (int i = 0; i < kHid; ++i) a = fmaf(P[kOffW2 + j * kHid + i], h1[i], a);
        h2[j] = tanhf(a);
    }
    float a = P[kOffB3];
    for (int i = 0; i < kHid; ++i) a = fmaf(P[kOffW3 + i], h2[i], a);
    y = a;
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params,
                                                     const float* __restrict__ X, int n,
                                                     float* __restrict__ Y) {
    __shared__ float P[kNParams];
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[kIn], h1[kHid], h2[kHid], y;
    for (int i = 0; i < kIn; ++i) x[i] = X[static_cast<int64_t>(s) * kIn + i];
    mlp_forward_one(P, x, h1, h2, y);
    Y[s] = y;
}

// Mean-squared-error gradient of a block of up to 64 samples, written as one partial gradient
// per block (summed in a fixed order by k_mlp_reduce, so the result is deterministic).
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ params,
                                                  const float* __restrict__ X,
                                                  const float* __restrict__ T, int n,
                                                  float* __restrict__ partial,
                                                  float* __restrict__ loss_partial) {
    extern __shared__ float sm[];
    float* P = sm;                              // kNParams
    float* xs = P + kNParams;                   // [64][kIn]
    float* h1s = xs + kBatchBlock * kIn;        // [64][kHid]
    float* h2s = h1s + kBatchBlock * kHid;      // [64][kHid]
    float* dz1 = h2s + kBatchBlock * kHid;      // [64][kHid]
    float* dz2 = dz1 + kBatchBlock * kHid;      // [64][kHid]
    float* dys = dz2 + kBatchBlock * kHid;      // [64]
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) P[i] = params[i];
    const int s0 = blockIdx.x * kBatchBlock;
    const int nb = min(kBatchBlock, n - s0);
    for (int i = threadIdx.x; i < kBatchBlock * kIn; i += blockDim.x) {
        const int b = i / kIn;
        xs[i] = b < nb ? X[static_cast<int64_t>(s0 + b) * kIn + i % kIn] : 0.f;
    }
    __syncthreads();
    // per-sample forward and backward down to dz1 and dz2 (one thread per sample)
    if (threadIdx.x < kBatchBlock) {
        const int b = threadIdx.x;
        float* h1 = h1s + b * kHid;
        float* h2 = h2s + b * kHid;
        float y;
        mlp_forward_one(P, xs + b * kIn, h1, h2, y);
        float dy = 0.f, l = 0.f;
        if (b < nb) {
            const float e = y - T[s0 + b];
            dy = 2.f * e / static_cast<float>(n);
            l = e * e / static_cast<float>(n);
        }
        dys[b] = dy;
        for (int j = 0; j < kHid; ++j) dz2[b * kHid + j] = dy * P[kOffW3 + j] * (1.f - h2[j] * h2[j]);
        for (int i = 0; i < kHid; ++i) {
            float a = 0.f;
            for (int j = 0; j < kHid; ++j) a = fmaf(P[kOffW2 + j * kHid + i], dz2[b * kHid + j], a);
            dz1[b * kHid + i] = a * (1.f - h1[i] * h1[i]);
        }
        loss_partial[blockIdx.x * kBatchBlock + b] = l;
    }
    __syncthreads();
    float* out = partial + static_cast<int64_t>(blockIdx.x) * kNParams;
    for (int p = threadIdx.x; p < kNW1; p += blockDim.x) {          // dW1 = dz1^T x
        const int j = p / kIn, i = p % kIn;
        float a = 0.f;
        for (int b = 0; b < kBatchBlock; ++b) a = fmaf(dz1[b * kHid + j], xs[b * kIn + i], a);
        out[kOffW1 + p] = a;
    }
    for (int p = threadIdx.x; p < kNW2; p += blockDim.x) {          // dW2 = dz2^T h1
        const int j = p / kHid, i = p % kHid;
        float a = 0.f;
        for (int b = 0; b < kBatchBlock; ++b) a = fmaf(dz2[b * kHid + j], h1s[b * kHid + i], a);
        out[kOffW2 + p] = a;
    }
    for (int j = threadIdx.x; j < kHid; j += blockDim.x) {          // db1, db2, dW3
        float a = 0.f, c = 0.f, w = 0.f;
        for (int b = 0; b < kBatchBlock; ++b) {
            a += dz1[b * kHid + j];
            c += dz2[b * kHid + j];
            w = fmaf(dys[b], h2s[b * kHid + j], w);
        }
        out[kOffB1 + j] = a;
        out[kOffB2 + j] = c;
        out[kOffW3 + j] = w;
    }
    if (threadIdx.x == 0) {                                          // db3
        float a = 0.f;
        for (int b = 0; b < kBatchBlock; ++b) a += dys[b];
        out[kOffB3] = a;
    }
}

__global__ void __launch_bounds__(256) k_mlp_reduce(const float* __restrict__ partial, int nblocks,
                                                    float* __restrict__ grad,
                                                    const float* __restrict__ loss_partial, int nloss,
                                                    float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kNParams) {
        float a = 0.f;
        for (int b = 0; b < nblocks; ++b) a += partial[static_cast<int64_t>(b) * kNParams + p];
        grad[p] = a;
    }
    if (p == 0 && loss) {
        float l = 0.f;
        for (int i = 0; i < nloss; ++i) l += loss_partial[i];
        *loss = l;
    }
}

// Adam (Kingma and Ba 2015) with bias correction.
__global__ void k_adam(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNParams) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    params[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Glorot-uniform weights, zero biases, from the counter-based generator.
__global__ void k_mlp_init(float* __restrict__ params, uint64_t seed) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNParams) return;
    float bound = 0.f;
    if (p < kOffB1) bound = sqrtf(6.f / (kIn + kHid));
    else if (p >= kOffW2 && p < kOffB2) bound = sqrtf(6.f / (kHid + kHid));
    else if (p >= kOffW3 && p < kOffB3) bound = sqrtf(6.f / (kHid + 1));
    params[p] = bound * (2.f * uniform01(seed, static_cast<uint64_t>(p)) - 1.f);
}

int mfail(int code, const std::string& m) {
    set_last_error(m);
    return code;
}

#define MLP_CK(call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return mfail(NDSI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool dev_ptr(const void* p) {
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t grad_smem() {
    return sizeof(float) * (kNParams + kBatchBlock * kIn + 4 * kBatchBlock * kHid + kBatchBlock);
}

int grad_launch(const float* params, const float* X, const float* T, int n, float* partial, float* lossp,
                float* grad, float* loss, cudaStream_t st) {
    const int nblk = (n + kBatchBlock - 1) / kBatchBlock;
    k_mlp_grad<<<nblk, 256, grad_smem(), st>>>(params, X, T, n, partial, lossp);
    MLP_CK(cudaGetLastError());
    k_mlp_reduce<<<(kNParams + 255) / 256, 256, 0, st>>>(partial, nblk, grad, lossp, nblk * kBatchBlock, loss);
    MLP_CK(cudaGetLastError());
    return NDSI_OK;
}

}  // namespace

int mlp_features(const Plan& P, const double* Hd, const double* Sd, const int64_t* rowptr_d,
                 const int32_t* col_d, double n_electrons, double kT, int R, uint64_t seed, float* feat_d,
                 cudaStream_t st) {
    const int64_t n = P.n;
    const int64_t cnt = n * R;
    float *buf = nullptr;
    double* partial = nullptr;
    const int nblk = static_cast<int>((cnt + 255) / 256);
    MLP_CK(cudaMalloc(&buf, sizeof(float) * cnt * 4));
    if (cudaMalloc(&partial, sizeof(double) * nblk) != cudaSuccess) {
        cudaFree(buf);
        return mfail(NDSI_ERR_OOM, "ndsi_mu_features: scratch allocation failed");
    }
    float* z = buf;
    float* t[3] = {buf + cnt, buf + 2 * cnt, buf + 3 * cnt};
    cudaError_t e = cudaSuccess;
    auto moments = [&](const double* vals, double shift, double scale, int kmax, int out0) {
        // t0 = z, t1 = A z, t_{k+1} = 2 A t_k - t_{k-1}; moment_k = z . t_k / (R n)
        const float* cur = z;
        const float* prv = nullptr;
        for (int k = 1; k <= kmax && e == cudaSuccess; ++k) {
            float* nxt = t[(k - 1) % 3];
            k_cheb_step<<<nblk, 256, 0, st>>>(rowptr_d, col_d, vals, shift, scale, n, R, cur, prv,
                                              k == 1 ? 1.f : 2.f, 1.f, nxt, seed, partial);
            k_sum_partials<<<1, 256, 0, st>>>(partial, nblk, 1.0 / static_cast<double>(cnt), feat_d + out0 + k - 1);
            e = cudaGetLastError();
            prv = cur;
            cur = nxt;
        }
    };
    k_rademacher<<<1024, 256, 0, st>>>(cnt, seed, z);
    e = cudaGetLastError();
    // fixed energy window [-4, 4] Ha for H; S - I in [-0.75, 0.75] for the overlap
    moments(Hd, 0.0, 4.0, 24, 0);
    moments(Sd, 1.0, 0.75, 6, 24);
    const float extra[2] = {static_cast<float>(n_electrons / (2.0 * n)), static_cast<float>(10.0 * kT)};
    if (e == cudaSuccess) e = cudaMemcpyAsync(feat_d + 30, extra, sizeof(extra), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    cudaFree(partial);
    if (e != cudaSuccess) return mfail(NDSI_ERR_CUDA, std::string("ndsi_mu_features: ") + cudaGetErrorString(e));
    return NDSI_OK;
}

}  // namespace ndsi

using namespace ndsi;

extern "C" {

int ndsi_mlp_init(float* params, uint64_t seed, void* stream) {
    if (!params || !dev_ptr(params)) return mfail(NDSI_ERR_INVALID, "ndsi_mlp_init: params must be device memory");
    k_mlp_init<<<(kNParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, seed);
    MLP_CK(cudaGetLastError());
    return NDSI_OK;
}

int ndsi_mlp_forward(const float* params, const float* X, int32_t n, float* Y, void* stream) {
    if (!params || !X || !Y || n < 1 || !dev_ptr(params) || !dev_ptr(X) || !dev_ptr(Y))
        return mfail(NDSI_ERR_INVALID, "ndsi_mlp_forward: device arrays and n >= 1 required");
    k_mlp_forward<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(params, X, n, Y);
    MLP_CK(cudaGetLastError());
    return NDSI_OK;
}

int ndsi_mlp_grad(const float* params, const float* X, const float* T, int32_t n, float* grad, float* loss,
                  void* stream) {
    if (!params || !X || !T || !grad || n < 1 || !dev_ptr(params) || !dev_ptr(X) || !dev_ptr(T) ||
        !dev_ptr(grad) || (loss && !dev_ptr(loss)))
        return mfail(NDSI_ERR_INVALID, "ndsi_mlp_grad: device arrays and n >= 1 required");
    static bool attr = false;
    if (!attr) {
        MLP_CK(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(grad_smem())));
        attr = true;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nblk = (n + kBatchBlock - 1) / kBatchBlock;
    float *partial = nullptr, *lossp = nullptr;
    MLP_CK(cudaMalloc(&partial, sizeof(float) * (static_cast<size_t>(nblk) * kNParams + nblk * kBatchBlock)));
    lossp = partial + static_cast<size_t>(nblk) * kNParams;
    int rc = grad_launch(params, X, T, n, partial, lossp, grad, loss, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(partial);
    if (rc) return rc;
    MLP_CK(e);
    return NDSI_OK;
}

int ndsi_mlp_train(float* params, const float* X, const float* T, int32_t n, int32_t steps, float lr,
                   float* loss_out, void* stream) {
    if (!params || !X || !T || n < 1 || steps < 1 || !(lr > 0) || !dev_ptr(params) || !dev_ptr(X) || !dev_ptr(T))
        return mfail(NDSI_ERR_INVALID, "ndsi_mlp_train: device arrays, n >= 1, steps >= 1, lr > 0 required");
    static bool attr = false;
    if (!attr) {
        MLP_CK(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(grad_smem())));
        attr = true;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nblk = (n + kBatchBlock - 1) / kBatchBlock;
    float* work = nullptr;
    const size_t nwork = static_cast<size_t>(nblk) * kNParams + nblk * kBatchBlock + 3 * kNParams + 1;
    MLP_CK(cudaMalloc(&work, sizeof(float) * nwork));
    float* partial = work;
    float* lossp = partial + static_cast<size_t>(nblk) * kNParams;
    float* grad = lossp + nblk * kBatchBlock;
    float* m = grad + kNParams;
    float* v = m + kNParams;
    float* loss = v + kNParams;
    cudaError_t e = cudaMemsetAsync(m, 0, sizeof(float) * 2 * kNParams, st);
    int rc = NDSI_OK;
    const float b1 = 0.9f, b2 = 0.999f;
    double p1 = 1.0, p2 = 1.0;
    for (int s = 0; s < steps && rc == NDSI_OK && e == cudaSuccess; ++s) {
        rc = grad_launch(params, X, T, n, partial, lossp, grad, loss, st);
        p1 *= b1;
        p2 *= b2;
        k_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(params, grad, m, v, lr, b1, b2, 1e-8f,
                                                       static_cast<float>(1.0 - p1), static_cast<float>(1.0 - p2));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(work);
    if (rc) return rc;
    MLP_CK(e);
    return NDSI_OK;
}

}  // extern "C"
