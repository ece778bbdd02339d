// Small dense symmetric eigenproblems on the host: the projected problems of the block
// shift-invert eigensolver (App. B, Eq. B3).
#pragma once

#include <vector>

namespace ndsi {

// Symmetric eigendecomposition by cyclic Jacobi rotations: A (n x n, row-major) is overwritten;
// eigenvalues in w (unordered), eigenvectors as the columns of V (row-major).
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V);

// Rayleigh-Ritz in the span of m vectors with Gram matrices Hs = V^T H V and Ss = V^T S V
// (row-major m x m): Ritz values e and coefficients Y (m x e.size(), row-major), Y^T Ss Y = I;
// directions whose S-Gram eigenvalue is below 1e-12 of the largest are dropped.
void rayleigh_ritz(int m, const std::vector<double>& Hs, const std::vector<double>& Ss, std::vector<double>& e,
                   std::vector<double>& Y);

}  // namespace ndsi
