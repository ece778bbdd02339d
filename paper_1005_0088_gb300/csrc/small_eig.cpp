// Small dense symmetric eigenproblems on the host (see small_eig.hpp).
#include "small_eig.hpp"

#include <algorithm>
#include <cmath>

namespace ndsi {

// Symmetric eigendecomposition by cyclic Jacobi rotations (Golub & Van Loan, Matrix
// Computations, Sec. 8.5): A (n x n, row-major) is overwritten; eigenvalues in w, eigenvectors as
// the columns of V (row-major).  For the small projected problems of the eigensolver only.
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
    V.assign(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, all = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                all += A[p * n + q] * A[p * n + q];
                if (p != q) off += A[p * n + q] * A[p * n + q];
            }
        if (off <= 1e-32 * all) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q of A J
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q of J^T (A J)
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

// Rayleigh-Ritz of (B3) in the span of the m columns whose Gram matrices are Hs = V^T H V and
// Ss = V^T S V (row-major m x m): columns are scaled to unit S-norm, directions with an S-Gram
// eigenvalue below 1e-12 of the largest are dropped, and the reduced standard problem is solved.
// Returns the Ritz values e and coefficients Y (m x e.size(), row-major) with Y^T Ss Y = I.
void rayleigh_ritz(int m, const std::vector<double>& Hs, const std::vector<double>& Ss, std::vector<double>& e,
                   std::vector<double>& Y) {
    std::vector<double> d(m);
    for (int a = 0; a < m; ++a) d[a] = Ss[a * m + a] > 0 ? 1.0 / std::sqrt(Ss[a * m + a]) : 0.0;
    std::vector<double> Sn(static_cast<size_t>(m) * m), Hn(static_cast<size_t>(m) * m);
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            Sn[a * m + b] = 0.5 * (Ss[a * m + b] + Ss[b * m + a]) * d[a] * d[b];
            Hn[a * m + b] = 0.5 * (Hs[a * m + b] + Hs[b * m + a]) * d[a] * d[b];
        }
    std::vector<double> lam, Q;
    jacobi_eig(m, Sn, lam, Q);
    double lmax = 0.0;
    for (double l : lam) lmax = std::max(lmax, l);
    std::vector<int> keep;
    for (int i = 0; i < m; ++i)
        if (lam[i] > 1e-12 * lmax) keep.push_back(i);
    const int r = static_cast<int>(keep.size());
    std::vector<double> T(static_cast<size_t>(m) * r);  // m x r: Q_keep Lambda^{-1/2}
    for (int a = 0; a < m; ++a)
        for (int j = 0; j < r; ++j) T[a * r + j] = Q[a * m + keep[j]] / std::sqrt(lam[keep[j]]);
    std::vector<double> HT(static_cast<size_t>(m) * r, 0.0), Ht(static_cast<size_t>(r) * r, 0.0);
    for (int a = 0; a < m; ++a)
        for (int j = 0; j < r; ++j) {
            double acc = 0.0;
            for (int b = 0; b < m; ++b) acc += Hn[a * m + b] * T[b * r + j];
            HT[a * r + j] = acc;
        }
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
            double acc = 0.0;
            for (int a = 0; a < m; ++a) acc += T[a * r + i] * HT[a * r + j];
            Ht[i * r + j] = acc;
        }
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < i; ++j) Ht[i * r + j] = Ht[j * r + i] = 0.5 * (Ht[i * r + j] + Ht[j * r + i]);
    std::vector<double> W;
    jacobi_eig(r, Ht, e, W);
    Y.assign(static_cast<size_t>(m) * r, 0.0);
    for (int a = 0; a < m; ++a)
        for (int j = 0; j < r; ++j) {
            double acc = 0.0;
            for (int i = 0; i < r; ++i) acc += T[a * r + i] * W[i * r + j];
            Y[a * r + j] = d[a] * acc;
        }
}

}  // namespace ndsi
