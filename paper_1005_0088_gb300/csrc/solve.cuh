// Solves with the nested-dissection factorisation, and the dense kernels of the block
// shift-invert eigensolver (App. B).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "plan.hpp"

namespace ndsi {

// One supernode as the triangular solves see it: its front (f = s + r rows, column-major, lower
// storage) and the basis index of each front row.
struct SolveNode {
    int64_t front_off;  // complex elements within a point's slab of fronts
    int64_t row_off;    // offset into the row table (f entries)
    int32_t f, s, r, pad;
};

// A kSolveTile x kSolveTile tile of one node's front: forward tiles at (front row i0, column j0)
// of the first s columns (lower tiles only inside the J x J block), backward tiles at (row s + i0
// of R(J), column j0).
struct SolveTile {
    int32_t node, i0, j0, pad;
};

constexpr int kSolveTile = 64;
constexpr int kSolveRhs = 8;  // right-hand sides per block (grid.y covers the rest)

struct SolveTables {
    SolveNode* nodes = nullptr;
    int32_t* rows = nullptr;       // basis index of every front row, per node
    SolveTile* fwd = nullptr;      // forward tiles, grouped by level (leaves first)
    SolveTile* bwd = nullptr;      // backward tiles, grouped by level
    std::vector<int64_t> fwd_first, bwd_first;  // [n_levels + 1] host offsets per level
    void* blob = nullptr;
};

// Host construction and upload of the solve tables; freeing.
cudaError_t solve_tables_build(const Plan& P, SolveTables& T);
void solve_tables_free(SolveTables& T);

// X = (zS - H)^{-1} Y with the factors of one point held in `fronts` (after the factor phase:
// A_J^{-1} in the node's diagonal block, L_RJ = X_RJ A_J^{-1} below it).  Y and X are complex,
// n x k, row-major (the k right-hand sides of a basis index are adjacent), original basis order.
// Y is overwritten (the forward elimination works in it).  Every tile accumulates into X and Y
// with FP64 atomics, so the rounding order (not the result beyond it) varies from run to run.
cudaError_t launch_solve(const Plan& P, const SolveTables& T, const double2* fronts, double2* Y, double2* X, int k,
                         cudaStream_t st);

// Y[:, 0:m] = A X[:, 0:m] for the real CSR matrix A on the pattern (values in pattern order);
// X and Y are n x ld row-major.
cudaError_t launch_spmm(const int64_t* rowptr, const int32_t* col, const double* A, int64_t n, const double* X,
                        int ldx, double* Y, int ldy, int m, cudaStream_t st);

// R = Y - (z S - H) X for complex n x k blocks (row-major), H and S real on the CSR pattern: the
// residual of one step of iterative refinement.
cudaError_t launch_shifted_residual(const int64_t* rowptr, const int32_t* col, const double* H, const double* S,
                                    int64_t n, double2 z, const double2* X, const double2* Y, double2* R, int k,
                                    cudaStream_t st);

// X += D for count complex values.
cudaError_t launch_complex_add(double2* X, const double2* D, int64_t count, cudaStream_t st);

// B = A + 0i for count real values.
cudaError_t launch_real_to_complex(const double* A, int64_t count, double2* B, cudaStream_t st);

// V (n x 2k, real) = [Re B | Im B] of the complex n x k block B.
cudaError_t launch_split_complex(const double2* B, int64_t n, int k, double* V, cudaStream_t st);

// Gram matrices V^T HV and V^T SV (m x m each, m <= 64): per-block partial sums then a reduction
// into out[0:m*m] (H) and out[m*m:2*m*m] (S).
int gram_blocks(int64_t n);
cudaError_t launch_gram(const double* V, const double* HV, const double* SV, int64_t n, int m, double* partials,
                        double* out, cudaStream_t st);

// C (n x k) = V (n x m) Y (m x k, row-major, device); and per-block partial sums of the squared
// residuals |(HV - e_c SV) Y[:, c]|^2 (partials: gram_blocks(n) x k).
cudaError_t launch_ritz(const double* V, const double* HV, const double* SV, int64_t n, int m, const double* Y,
                        const double* e, int k, double* C, double* partials, cudaStream_t st);

}  // namespace ndsi
