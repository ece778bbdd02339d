// Residue sum and electron count from caller-held G, with no device allocation.
//
// This is the static-memory variant of the residue-sum kernel used by ndsi_density.  That path
// keeps its per-block partial traces in a buffer it allocates; here the partials live in a
// fixed file-scope __device__ array, so the entry point needs no cudaMalloc or cudaFree.  It
// serves callers that cannot allocate device memory themselves: code running under a host
// framework that owns the whole device-memory budget (an extra cudaMalloc would fail or break
// its accounting) and latency-critical callers for whom cudaMalloc/cudaFree, which can
// synchronise the device, are not acceptable.  Such a caller holds G, the weights, S and the
// outputs in memory it already owns.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "ndsi.h"
#include "plan.hpp"

namespace ndsi {
namespace {

constexpr int kStaticThreads = 256;
// One partial trace per 256-entry block: at most 2^15 blocks, i.e. nnz <= 8,388,608.
constexpr int kStaticMaxBlocks = 32768;
constexpr int64_t kStaticMaxNnz = static_cast<int64_t>(kStaticMaxBlocks) * kStaticThreads;

// Shared by every call on a device; held by every GPU that loads the library until exit.
static __device__ __align__(256) double g_static_partials[kStaticMaxBlocks];

// Device address of g_static_partials, resolved once per device.
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {};

// rho_k = sum_q Re(c_q G_q(k)) and one partial of sum_k rho_k S_k per block.
__global__ void __launch_bounds__(kStaticThreads) k_residue_sum_static(
    const double2* __restrict__ G, int64_t nnz, int np, const double2* __restrict__ c,
    const double* __restrict__ S, double* __restrict__ rho, double* __restrict__ partials) {
    __shared__ double red[kStaticThreads / 32];
    const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    double tr = 0.0;
    if (k < nnz) {
        double sum = 0.0;
        for (int q = 0; q < np; ++q) {
            const double2 g = G[static_cast<int64_t>(q) * nnz + k];
            const double2 w = c[q];
            sum += w.x * g.x - w.y * g.y;
        }
        rho[k] = sum;
        tr = sum * S[k];
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kStaticThreads / 32 ? red[threadIdx.x] : 0.0;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

// Fixed-order sum of the partials written by the launch above.
__global__ void __launch_bounds__(1024) k_reduce_static(const double* __restrict__ partials, int n,
                                                        double* __restrict__ out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) *out = w;
    }
}

// Memory the kernels may read or write on device `dev`: device memory of that device, or
// managed memory.  Device memory of another GPU is refused (the kernels would fault on it).
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// G and c are read as complex pairs (16-byte loads).
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int static_fail(int code, const std::string& msg) {
    set_last_error(msg);
    return code;
}

}  // namespace
}  // namespace ndsi

using namespace ndsi;

extern "C" int ndsi_residue_sum_static(const double* G, const double* c, int32_t n_points,
                                       const double* S, int64_t nnz, double* rho_out,
                                       double* n_elec_out, void* stream) {
    if (!G || !c || !S || !rho_out || n_points < 1 || nnz < 1)
        return static_fail(NDSI_ERR_INVALID, "ndsi_residue_sum_static: invalid argument");
    if (nnz > kStaticMaxNnz)
        return static_fail(NDSI_ERR_INVALID,
                           "ndsi_residue_sum_static: nnz = " + std::to_string(nnz) +
                               " exceeds the static scratch limit of " +
                               std::to_string(kStaticMaxNnz) + " pattern entries");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return static_fail(NDSI_ERR_CUDA, "ndsi_residue_sum_static: no usable current device");
    if (!on_device(G, dev) || !on_device(c, dev) || !on_device(S, dev) || !on_device(rho_out, dev) ||
        (n_elec_out && !on_device(n_elec_out, dev)))
        return static_fail(NDSI_ERR_INVALID,
                           "ndsi_residue_sum_static: every array must be in device memory of the current device");
    if (!aligned16(G) || !aligned16(c))
        return static_fail(NDSI_ERR_INVALID, "ndsi_residue_sum_static: G and c must be 16-byte aligned");
    double* partials = nullptr;
    {
        // First call on this device: resolve the array's device address with the device current.
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_partials);
            if (e != cudaSuccess || !p)
                return static_fail(NDSI_ERR_CUDA, std::string("ndsi_residue_sum_static: "
                                                              "cudaGetSymbolAddress: ") +
                                                      cudaGetErrorString(e));
            g_static_ptr[dev] = static_cast<double*>(p);
        }
        partials = g_static_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nblk = static_cast<int>((nnz + kStaticThreads - 1) / kStaticThreads);
    // Every partial read by k_reduce_static is written first by this launch, so nothing in the
    // array needs clearing; values left by an earlier call are overwritten.
    k_residue_sum_static<<<nblk, kStaticThreads, 0, st>>>(reinterpret_cast<const double2*>(G), nnz,
                                                          n_points, reinterpret_cast<const double2*>(c),
                                                          S, rho_out, partials);
    if (n_elec_out) k_reduce_static<<<1, 1024, 0, st>>>(partials, nblk, n_elec_out);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return static_fail(NDSI_ERR_CUDA, std::string("ndsi_residue_sum_static: launch: ") +
                                              cudaGetErrorString(e));
    return NDSI_OK;
}
