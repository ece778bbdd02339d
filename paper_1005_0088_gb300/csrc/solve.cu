// Triangular solves with the nested-dissection factors, and the dense kernels of the block
// shift-invert eigensolver.
//
// After the factor phase a node J's front holds A_J^{-1} (its diagonal block after the Schur
// updates of its descendants; lower storage) and L_RJ = X_RJ A_J^{-1} below it, so that
// zS - H = L D L^T with unit block-lower L (blocks L_RJ) and D = diag(A_J).  The product with
// (zS - H)^{-1} is then the three steps of App. B (B8-B15) in the supernodal form:
//   forward, leaves first:   y_R(J) -= L_RJ y_J            (y_J is final once J's subtree is done)
//   diagonal:                w_J = A_J^{-1} y_J             (fused into the forward launch)
//   backward, root first:    x_J = w_J - L_RJ^T x_R(J)      (x_R(J) is final: ancestors done)
// Nodes of one tree level run in one launch.  The forward scatter goes to ancestor rows that
// several nodes of the level may share, so it uses FP64 atomics; every other write has one owner.
#include "solve.cuh"

#include <algorithm>

namespace ndsi {

namespace {

__device__ __forceinline__ double2 cmac(double2 acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}

constexpr int kFwdChunk = 32;  // columns of y_J staged in shared memory at a time

// One tile of kSolveFwdRows front rows of node J, kSolveRhs right-hand sides (grid.y): rows of
// J get w = A_J^{-1} y_J (written to X), rows of R(J) subtract L_RJ y_J from Y (atomics).
__global__ void __launch_bounds__(kSolveFwdRows) k_solve_fwd(const SolveNode* __restrict__ nodes,
                                                            const int32_t* __restrict__ rows,
                                                            const SolveTile* __restrict__ tiles,
                                                            const double2* __restrict__ F, double2* Y,
                                                            double2* __restrict__ X, int k) {
    __shared__ double2 zs[kFwdChunk][kSolveRhs];
    const SolveTile t = tiles[blockIdx.x];
    const SolveNode nd = nodes[t.node];
    const int i = t.i0 + threadIdx.x;
    const int c0 = blockIdx.y * kSolveRhs;
    const int nc = min(kSolveRhs, k - c0);
    const int32_t* rb = rows + nd.row_off;
    const double2* Fn = F + nd.front_off;
    double2 acc[kSolveRhs];
#pragma unroll
    for (int c = 0; c < kSolveRhs; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int j0 = 0; j0 < nd.s; j0 += kFwdChunk) {
        const int jn = min(kFwdChunk, nd.s - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < kFwdChunk * kSolveRhs; e += blockDim.x) {
            const int jj = e / kSolveRhs, cc = e % kSolveRhs;
            zs[jj][cc] = (jj < jn && cc < nc) ? Y[static_cast<int64_t>(rb[j0 + jj]) * k + c0 + cc]
                                              : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (i < nd.f) {
            for (int jj = 0; jj < jn; ++jj) {
                const int j = j0 + jj;
                // rows of R(J): L_RJ(i - s, j); rows of J: A_J^{-1}(i, j) from the lower triangle
                const double2 a = (i >= nd.s || j <= i) ? Fn[i + static_cast<int64_t>(j) * nd.f]
                                                        : Fn[j + static_cast<int64_t>(i) * nd.f];
#pragma unroll
                for (int c = 0; c < kSolveRhs; ++c) acc[c] = cmac(acc[c], a, zs[jj][c]);
            }
        }
    }
    if (i >= nd.f) return;
    const int64_t row = static_cast<int64_t>(rb[i]) * k + c0;
    if (i < nd.s) {
        for (int c = 0; c < nc; ++c) X[row + c] = acc[c];
    } else {
        for (int c = 0; c < nc; ++c) {
            atomicAdd(&Y[row + c].x, -acc[c].x);
            atomicAdd(&Y[row + c].y, -acc[c].y);
        }
    }
}

// One warp per row i of node J: x_J(i) -= sum_t L_RJ(t, i) x_R(J)(t), lanes over t.
__global__ void __launch_bounds__(32 * kSolveBwdRows) k_solve_bwd(const SolveNode* __restrict__ nodes,
                                                                 const int32_t* __restrict__ rows,
                                                                 const SolveTile* __restrict__ tiles,
                                                                 const double2* __restrict__ F, double2* X,
                                                                 int k) {
    const SolveTile t = tiles[blockIdx.x];
    const SolveNode nd = nodes[t.node];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = t.i0 + warp;
    if (i >= nd.s) return;
    const int c0 = blockIdx.y * kSolveRhs;
    const int nc = min(kSolveRhs, k - c0);
    const int32_t* rb = rows + nd.row_off;
    const double2* Lcol = F + nd.front_off + nd.s + static_cast<int64_t>(i) * nd.f;
    double2 acc[kSolveRhs];
#pragma unroll
    for (int c = 0; c < kSolveRhs; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int tt = lane; tt < nd.r; tt += 32) {
        const double2 l = Lcol[tt];
        const double2* xr = X + static_cast<int64_t>(rb[nd.s + tt]) * k + c0;
#pragma unroll
        for (int c = 0; c < kSolveRhs; ++c)
            if (c < nc) acc[c] = cmac(acc[c], l, xr[c]);
    }
#pragma unroll
    for (int c = 0; c < kSolveRhs; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc[c].x += __shfl_down_sync(0xffffffffu, acc[c].x, o);
            acc[c].y += __shfl_down_sync(0xffffffffu, acc[c].y, o);
        }
    }
    if (lane == 0) {
        double2* xi = X + static_cast<int64_t>(rb[i]) * k + c0;
        for (int c = 0; c < nc; ++c) xi[c] = make_double2(xi[c].x - acc[c].x, xi[c].y - acc[c].y);
    }
}

// One warp per row of the CSR matrix, lanes over the m columns.
__global__ void __launch_bounds__(256) k_spmm(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                              const double* __restrict__ A, int64_t n,
                                              const double* __restrict__ X, int ldx, double* __restrict__ Y,
                                              int ldy, int m) {
    const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    for (int c = lane; c < m; c += 32) {
        double acc = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) acc = fma(A[e], X[static_cast<int64_t>(col[e]) * ldx + c], acc);
        Y[i * ldy + c] = acc;
    }
}

__global__ void __launch_bounds__(256) k_split_complex(const double2* __restrict__ B, int64_t n, int k,
                                                       double* __restrict__ V) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    const int64_t i = e / k;
    const int c = static_cast<int>(e - i * k);
    const double2 b = B[e];
    V[i * 2 * k + c] = b.x;
    V[i * 2 * k + k + c] = b.y;
}

__global__ void __launch_bounds__(256) k_real_to_complex(const double* __restrict__ A, int64_t count,
                                                         double2* __restrict__ B) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < count) B[e] = make_double2(A[e], 0.0);
}

// One warp per row, lanes over the right-hand sides: R = Y - (z S - H) X.
__global__ void __launch_bounds__(256) k_shifted_residual(const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ H, const double* __restrict__ S,
                                                          int64_t n, double2 z, const double2* __restrict__ X,
                                                          const double2* __restrict__ Y, double2* __restrict__ R,
                                                          int k) {
    const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    for (int c = lane; c < k; c += 32) {
        double2 acc = Y[i * k + c];
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            // (z S - H)_ie = (z.x S - H) + i z.y S
            const double2 a = make_double2(z.x * S[e] - H[e], z.y * S[e]);
            const double2 x = X[static_cast<int64_t>(col[e]) * k + c];
            acc.x -= a.x * x.x - a.y * x.y;
            acc.y -= a.x * x.y + a.y * x.x;
        }
        R[i * k + c] = acc;
    }
}

__global__ void __launch_bounds__(256) k_complex_add(double2* __restrict__ X, const double2* __restrict__ D,
                                                     int64_t count) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < count) X[e] = make_double2(X[e].x + D[e].x, X[e].y + D[e].y);
}

constexpr int kGramRows = 16;
constexpr int kGramMax = 64;
constexpr int kGramPairs = kGramMax * kGramMax / 256;  // pairs per thread at m = 64

// Partial Gram sums over a contiguous range of rows per block; thread p owns pairs p, p+256, ...
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ V, const double* __restrict__ HV,
                                              const double* __restrict__ SV, int64_t n, int m,
                                              double* __restrict__ partials) {
    __shared__ double vs[kGramRows][kGramMax], hs[kGramRows][kGramMax], ss[kGramRows][kGramMax];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * per;
    const int64_t r1 = min(n, r0 + per);
    double ah[kGramPairs], as[kGramPairs];
#pragma unroll
    for (int q = 0; q < kGramPairs; ++q) ah[q] = as[q] = 0.0;
    for (int64_t rb = r0; rb < r1; rb += kGramRows) {
        const int nr = static_cast<int>(r1 - rb < kGramRows ? r1 - rb : kGramRows);
        __syncthreads();
        for (int e = threadIdx.x; e < kGramRows * m; e += blockDim.x) {
            const int rr = e / m, cc = e % m;
            const bool ok = rr < nr;
            const int64_t g = (rb + rr) * m + cc;
            vs[rr][cc] = ok ? V[g] : 0.0;
            hs[rr][cc] = ok ? HV[g] : 0.0;
            ss[rr][cc] = ok ? SV[g] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kGramPairs; ++q) {
            const int p = threadIdx.x + q * 256;
            if (p < m * m) {
                const int a = p / m, b = p % m;
                double h = ah[q], s = as[q];
                for (int rr = 0; rr < nr; ++rr) {
                    h = fma(vs[rr][a], hs[rr][b], h);
                    s = fma(vs[rr][a], ss[rr][b], s);
                }
                ah[q] = h;
                as[q] = s;
            }
        }
    }
    double* out = partials + static_cast<int64_t>(blockIdx.x) * 2 * m * m;
#pragma unroll
    for (int q = 0; q < kGramPairs; ++q) {
        const int p = threadIdx.x + q * 256;
        if (p < m * m) {
            out[p] = ah[q];
            out[m * m + p] = as[q];
        }
    }
}

__global__ void __launch_bounds__(256) k_gram_reduce(const double* __restrict__ partials, int nblk, int len,
                                                     double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partials[static_cast<int64_t>(b) * len + e];
    out[e] = s;
}

constexpr int kRitzMaxK = 32;

// Thread per row (grid-stride): C(i, :) = V(i, :) Y and the squared residual of every column,
// reduced per block into partials[block][c].
__global__ void __launch_bounds__(256) k_ritz(const double* __restrict__ V, const double* __restrict__ HV,
                                              const double* __restrict__ SV, int64_t n, int m,
                                              const double* __restrict__ Yg, const double* __restrict__ eg, int k,
                                              double* __restrict__ C, double* __restrict__ partials) {
    __shared__ double Ys[kGramMax * kRitzMaxK];
    __shared__ double es[kRitzMaxK];
    __shared__ double red[8][kRitzMaxK];
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) Ys[e] = Yg[e];
    if (threadIdx.x < k) es[threadIdx.x] = eg[threadIdx.x];
    __syncthreads();
    double rs[kRitzMaxK];
#pragma unroll
    for (int c = 0; c < kRitzMaxK; ++c) rs[c] = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double* v = V + i * m;
        const double* hv = HV + i * m;
        const double* sv = SV + i * m;
#pragma unroll
        for (int c = 0; c < kRitzMaxK; ++c) {
            if (c < k) {
                double cv = 0.0, hc = 0.0, sc = 0.0;
                for (int a = 0; a < m; ++a) {
                    const double y = Ys[a * k + c];
                    cv = fma(v[a], y, cv);
                    hc = fma(hv[a], y, hc);
                    sc = fma(sv[a], y, sc);
                }
                C[i * k + c] = cv;
                const double r = hc - es[c] * sc;
                rs[c] = fma(r, r, rs[c]);
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < kRitzMaxK; ++c) {
        double v = rs[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        partials[static_cast<int64_t>(blockIdx.x) * k + threadIdx.x] = s;
    }
}

}  // namespace

cudaError_t solve_tables_build(const Plan& P, SolveTables& T) {
    const int32_t nn = P.n_nodes;
    std::vector<SolveNode> nodes(nn);
    std::vector<int32_t> rows;
    for (int32_t j = 0; j < nn; ++j) {
        SolveNode& d = nodes[j];
        d.front_off = P.front_off[j];
        d.row_off = static_cast<int64_t>(rows.size());
        d.f = P.f[j];
        d.s = P.s[j];
        d.r = P.r[j];
        d.pad = 0;
        for (int32_t i = 0; i < P.s[j]; ++i) rows.push_back(P.perm_basis[P.node_first[j] + i]);
        for (int64_t q = P.sstruct_ptr[j]; q < P.sstruct_ptr[j + 1]; ++q) rows.push_back(P.perm_basis[P.struct_basis[q]]);
    }
    std::vector<SolveTile> fwd, bwd;
    T.fwd_first.assign(P.n_levels + 1, 0);
    T.bwd_first.assign(P.n_levels + 1, 0);
    for (int32_t L = 0; L < P.n_levels; ++L) {
        T.fwd_first[L] = static_cast<int64_t>(fwd.size());
        T.bwd_first[L] = static_cast<int64_t>(bwd.size());
        for (int32_t j : P.level_nodes[L]) {
            if (P.s[j] == 0) continue;
            for (int32_t i0 = 0; i0 < P.f[j]; i0 += kSolveFwdRows) fwd.push_back(SolveTile{j, i0});
            if (P.r[j] > 0)
                for (int32_t i0 = 0; i0 < P.s[j]; i0 += kSolveBwdRows) bwd.push_back(SolveTile{j, i0});
        }
    }
    T.fwd_first[P.n_levels] = static_cast<int64_t>(fwd.size());
    T.bwd_first[P.n_levels] = static_cast<int64_t>(bwd.size());
    auto al = [](size_t b) { return (std::max<size_t>(b, 16) + 255) / 256 * 256; };
    const size_t b0 = al(sizeof(SolveNode) * nodes.size()), b1 = al(sizeof(int32_t) * rows.size()),
                 b2 = al(sizeof(SolveTile) * fwd.size()), b3 = al(sizeof(SolveTile) * bwd.size());
    cudaError_t e = cudaMalloc(&T.blob, b0 + b1 + b2 + b3);
    if (e != cudaSuccess) return e;
    char* base = static_cast<char*>(T.blob);
    T.nodes = reinterpret_cast<SolveNode*>(base);
    T.rows = reinterpret_cast<int32_t*>(base + b0);
    T.fwd = reinterpret_cast<SolveTile*>(base + b0 + b1);
    T.bwd = reinterpret_cast<SolveTile*>(base + b0 + b1 + b2);
    if (!nodes.empty() && (e = cudaMemcpy(T.nodes, nodes.data(), sizeof(SolveNode) * nodes.size(), cudaMemcpyHostToDevice)))
        return e;
    if (!rows.empty() && (e = cudaMemcpy(T.rows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice)))
        return e;
    if (!fwd.empty() && (e = cudaMemcpy(T.fwd, fwd.data(), sizeof(SolveTile) * fwd.size(), cudaMemcpyHostToDevice)))
        return e;
    if (!bwd.empty() && (e = cudaMemcpy(T.bwd, bwd.data(), sizeof(SolveTile) * bwd.size(), cudaMemcpyHostToDevice)))
        return e;
    return cudaSuccess;
}

void solve_tables_free(SolveTables& T) {
    if (T.blob) cudaFree(T.blob);
    T = SolveTables{};
}

cudaError_t launch_solve(const Plan& P, const SolveTables& T, const double2* fronts, double2* Y, double2* X, int k,
                         cudaStream_t st) {
    const unsigned gy = static_cast<unsigned>((k + kSolveRhs - 1) / kSolveRhs);
    for (int32_t L = 0; L < P.n_levels; ++L) {
        const int64_t cnt = T.fwd_first[L + 1] - T.fwd_first[L];
        if (cnt == 0) continue;
        k_solve_fwd<<<dim3(static_cast<unsigned>(cnt), gy), kSolveFwdRows, 0, st>>>(T.nodes, T.rows, T.fwd + T.fwd_first[L],
                                                                                     fronts, Y, X, k);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int32_t L = P.n_levels - 1; L >= 0; --L) {
        const int64_t cnt = T.bwd_first[L + 1] - T.bwd_first[L];
        if (cnt == 0) continue;
        k_solve_bwd<<<dim3(static_cast<unsigned>(cnt), gy), 32 * kSolveBwdRows, 0, st>>>(
            T.nodes, T.rows, T.bwd + T.bwd_first[L], fronts, X, k);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_spmm(const int64_t* rowptr, const int32_t* col, const double* A, int64_t n, const double* X,
                        int ldx, double* Y, int ldy, int m, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n * 32 + 255) / 256;
    k_spmm<<<static_cast<unsigned>(blocks), 256, 0, st>>>(rowptr, col, A, n, X, ldx, Y, ldy, m);
    return cudaGetLastError();
}

cudaError_t launch_split_complex(const double2* B, int64_t n, int k, double* V, cudaStream_t st) {
    const int64_t total = n * k;
    if (total == 0) return cudaSuccess;
    k_split_complex<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(B, n, k, V);
    return cudaGetLastError();
}

cudaError_t launch_real_to_complex(const double* A, int64_t count, double2* B, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_real_to_complex<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(A, count, B);
    return cudaGetLastError();
}

cudaError_t launch_shifted_residual(const int64_t* rowptr, const int32_t* col, const double* H, const double* S,
                                    int64_t n, double2 z, const double2* X, const double2* Y, double2* R, int k,
                                    cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_shifted_residual<<<static_cast<unsigned>((n * 32 + 255) / 256), 256, 0, st>>>(rowptr, col, H, S, n, z, X, Y, R,
                                                                                     k);
    return cudaGetLastError();
}

cudaError_t launch_complex_add(double2* X, const double2* D, int64_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_complex_add<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(X, D, count);
    return cudaGetLastError();
}

int gram_blocks(int64_t n) { return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + 63) / 64, 304))); }

cudaError_t launch_gram(const double* V, const double* HV, const double* SV, int64_t n, int m, double* partials,
                        double* out, cudaStream_t st) {
    if (m < 1 || m > kGramMax) return cudaErrorInvalidValue;
    const int nb = gram_blocks(n);
    k_gram<<<nb, 256, 0, st>>>(V, HV, SV, n, m, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int len = 2 * m * m;
    k_gram_reduce<<<(len + 255) / 256, 256, 0, st>>>(partials, nb, len, out);
    return cudaGetLastError();
}

cudaError_t launch_ritz(const double* V, const double* HV, const double* SV, int64_t n, int m, const double* Y,
                        const double* e, int k, double* C, double* partials, cudaStream_t st) {
    if (m < 1 || m > kGramMax || k < 1 || k > kRitzMaxK) return cudaErrorInvalidValue;
    k_ritz<<<gram_blocks(n), 256, 0, st>>>(V, HV, SV, n, m, Y, e, k, C, partials);
    return cudaGetLastError();
}

}  // namespace ndsi
