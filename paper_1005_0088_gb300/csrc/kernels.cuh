// Device kernels of the FP64 numeric phase (shared declarations).
#pragma once

#include <cuda_runtime.h>

#include "plan.hpp"

namespace ndsi {

// Error bits latched in the device status word.
constexpr int kStatusSingular = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusBadItem = 4;  // a schedule item outside what its kernel handles (skipped)

struct DevTables {
    NodeDev* nodes = nullptr;
    int64_t* asm_map = nullptr;
    int64_t* out_map = nullptr;
    int32_t* inv_map = nullptr;
    int32_t* rel_map = nullptr;
    int64_t* scatter_idx = nullptr;
    GemmItem* gemm_items = nullptr;
    GemmTile* gemm_tiles = nullptr;
    CopyItem* copy_items = nullptr;
    DiagItem* diag_items = nullptr;
    NodeTile* node_tiles = nullptr;
    int32_t* entry_sys = nullptr;  // system of each pattern entry
    int64_t* rowptr = nullptr;   // CSR pattern (original order), for the moment features
    int32_t* col = nullptr;
    int* status = nullptr;
    void* blob = nullptr;  // single allocation holding all of the above
};

// Pole-batched workspace: `np` slabs of fronts and of scratch.
struct Workspace {
    double2* fronts = nullptr;
    double2* scr = nullptr;
    int64_t front_stride = 0;   // complex elements per pole slab
    int64_t scr_stride = 0;
    int32_t np_cap = 0;         // poles the buffers hold
};

// Spectral-moment features of (H, S) for the learned mu seed (mlp.cu).
int mlp_features(const Plan& P, const double* Hd, const double* Sd, const int64_t* rowptr_d,
                 const int32_t* col_d, double n_electrons, double kT, int R, uint64_t seed, float* feat_d,
                 cudaStream_t st);

// One-time kernel attributes (large dynamic shared memory).
cudaError_t kernels_init();

// Launch one schedule step over `np` poles whose slabs start at the workspace base.
// z holds the points of every system: z[sys * zstride + pole].
cudaError_t launch_step(const Plan& P, const DevTables& T, const Launch& l, const Workspace& W,
                        const double* H, const double* S, const double2* z, int64_t zstride, int np,
                        cudaStream_t st);

// rho(k) (+)= sum_q Re(c_q G_q(k)) over the pattern; `partials` receives per-block sums of
// rho(k) S(k) when `want_trace` is set (nblocks = accumulate_blocks(nnz)).
// (entries [k0, k0+count); count < 0 = the whole pattern)
cudaError_t launch_accumulate(const Plan& P, const DevTables& T, const Workspace& W, int np,
                              const double2* c, const double* S, double* rho, int accumulate,
                              int want_trace, double* partials, cudaStream_t st, int64_t k0 = 0,
                              int64_t count = -1);
int accumulate_blocks(int64_t nnz);
cudaError_t launch_reduce(const double* partials, int nblocks, double* out, cudaStream_t st);

// Gershgorin data of (H, S): out[0] = order key of max_i sum_j |H_ij|, out[1] = order key of
// max_i (sum_{j != i} |S_ij| - S_ii); keys decode with gershgorin_value.  out must be zeroed.
cudaError_t launch_gershgorin(const DevTables& T, int64_t n, const double* H, const double* S,
                              unsigned long long* out, cudaStream_t st);
double gershgorin_value(unsigned long long key);

// Per point q of a chunk: out[q] = sum over the pattern of Im G_q(k) S_k = Im Tr(G(z_q) S) (the
// density of states of Eq. 42 up to -2/pi).  partials: np x accumulate_blocks(nnz) doubles.
// The same over one range of pattern entries (out_map and S offset to its first entry; F holds np
// point slabs of `stride` complex elements): out[q] = sum_k Im F_q[out_map[k]] S[k].
cudaError_t launch_point_traces_range(const int64_t* out_map, int64_t nnz, const double2* F, int64_t stride, int np,
                                      const double* S, double* partials, double* out, cudaStream_t st);
cudaError_t launch_point_traces(const Plan& P, const DevTables& T, const Workspace& W, int np,
                                const double* S, double* partials, double* out, cudaStream_t st);

// G_out[q*nnz + k] = G_q(k) for the np poles of the workspace.
cudaError_t launch_gather_pattern(const Plan& P, const DevTables& T, const Workspace& W, int np,
                                  double2* G_out, int64_t q0, cudaStream_t st);

}  // namespace ndsi
