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

constexpr int kT = kSolveTile;
constexpr int kTP = kSolveTile + 1;  // padded tile row (conflict-free column reads)

constexpr int kSolveThreads = 256;

// Stage a kT x kT tile of the front (column-major, rows r0.., columns c0..) into shared memory as
// t[c][r] with asynchronous 16-byte copies (every copy of a thread in flight at once); entries
// outside rows [0, rows) or columns [0, cols) are zero-filled.  Ends with the copies complete and
// a block barrier.
__device__ __forceinline__ void load_tile(double2 (*t)[kTP], const double2* __restrict__ Fn, int64_t ld, int r0,
                                          int rows, int c0, int cols) {
#pragma unroll
    for (int u = 0; u < kT * kT / kSolveThreads; ++u) {
        const int e = threadIdx.x + u * kSolveThreads;
        const int r = e % kT, c = e / kT;
        const bool ok = r0 + r < rows && c0 + c < cols;
        const double2* src = ok ? Fn + (r0 + r) + static_cast<int64_t>(c0 + c) * ld : Fn;
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&t[c][r]));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0)
                     : "memory");
    }
}

__device__ __forceinline__ void load_tile_wait() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
}

// Right-hand-side values c + id of kT rows staged for the three-multiplication complex product:
// (a + ib)(c + id) = [c(a + b) - b(c + d)] + i[c(a + b) + a(d - c)], so a dot product over a tile
// takes three real FMAs per complex term (c, d - c and c + d stored per value).
struct RhsTile {
    double c[kT][kSolveRhs], dmc[kT][kSolveRhs], cpd[kT][kSolveRhs];
};

// Stage kT rows (basis indices rb[i0 + r], r < n) of a complex n x k row-major block, RHS c0..
__device__ __forceinline__ void load_rows(RhsTile& v, const double2* X, const int32_t* rb, int i0, int n, int k,
                                          int c0, int nc) {
    for (int e = threadIdx.x; e < kT * kSolveRhs; e += kSolveThreads) {
        const int r = e / kSolveRhs, c = e % kSolveRhs;
        const double2 x = (i0 + r < n && c < nc) ? X[static_cast<int64_t>(rb[i0 + r]) * k + c0 + c]
                                                 : make_double2(0.0, 0.0);
        v.c[r][c] = x.x;
        v.dmc[r][c] = x.y - x.x;
        v.cpd[r][c] = x.x + x.y;
    }
}

__device__ __forceinline__ void atomic_add2(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

constexpr int kRq = kSolveRhs / 4;  // right-hand sides per thread (four thread quarters)

// Three-multiplication accumulators of kRq complex dot products.
struct Acc3 {
    double p1[kRq], p2[kRq], p3[kRq];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int u = 0; u < kRq; ++u) p1[u] = p2[u] = p3[u] = 0.0;
    }
    __device__ __forceinline__ void add(double2 a, const RhsTile& v, int row, int col0) {
        const double ab = a.x + a.y;
#pragma unroll
        for (int u = 0; u < kRq; ++u) {
            p1[u] = fma(v.c[row][col0 + u], ab, p1[u]);
            p2[u] = fma(a.x, v.dmc[row][col0 + u], p2[u]);
            p3[u] = fma(a.y, v.cpd[row][col0 + u], p3[u]);
        }
    }
    __device__ __forceinline__ double2 get(int u, double sg) const {
        return make_double2(sg * (p1[u] - p3[u]), sg * (p1[u] + p2[u]));
    }
};

// Forward tile (i0, j0) of node J: front rows i0.. against y_J rows j0..  Rows of R(J) subtract
// L_RJ y_J from Y; rows of J accumulate w = A_J^{-1} y_J into X from the lower triangle only
// (element (i, j), i >= j, serves row i directly and, for i > j, row j transposed).
__global__ void __launch_bounds__(kSolveThreads) k_solve_fwd(const SolveNode* __restrict__ nodes,
                                                             const int32_t* __restrict__ rows,
                                                             const SolveTile* __restrict__ tiles,
                                                             const double2* __restrict__ F, double2* Y, double2* X,
                                                             int k) {
    extern __shared__ double2 solve_smem[];
    auto t = reinterpret_cast<double2 (*)[kTP]>(solve_smem);
    RhsTile& yc = *reinterpret_cast<RhsTile*>(solve_smem + kT * kTP);
    RhsTile& yr = *(&yc + 1);
    const SolveTile tl = tiles[blockIdx.x];
    const SolveNode nd = nodes[tl.node];
    const int c0 = blockIdx.y * kSolveRhs;
    const int nc = min(kSolveRhs, k - c0);
    const int32_t* rb = rows + nd.row_off;
    load_tile(t, F + nd.front_off, nd.f, tl.i0, nd.f, tl.j0, nd.s);
    load_rows(yc, Y, rb, tl.j0, nd.s, k, c0, nc);
    const bool sym = tl.i0 < nd.s;  // the tile has rows of J
    if (sym) load_rows(yr, Y, rb, tl.i0, nd.s, k, c0, nc);
    load_tile_wait();
    const int q = threadIdx.x >> 6, r = threadIdx.x & (kT - 1);  // 4 quarters of kRq RHS, 64 rows
    if (kRq * q >= nc) return;  // a whole quarter (two warps) without right-hand sides
    // direct part: row i0 + r
    {
        const int i = tl.i0 + r;
        if (i < nd.f) {
            Acc3 acc;
            acc.zero();
            const int jmax = i < nd.s ? min(kT, i - tl.j0 + 1) : kT;  // J rows: lower triangle only
            for (int c = 0; c < jmax; ++c) acc.add(t[c][r], yc, c, kRq * q);
            double2* dst = (i < nd.s ? X : Y) + static_cast<int64_t>(rb[i]) * k + c0;
            const double sg = i < nd.s ? 1.0 : -1.0;
#pragma unroll
            for (int u = 0; u < kRq; ++u)
                if (kRq * q + u < nc && jmax > 0) atomic_add2(dst + kRq * q + u, acc.get(u, sg));
        }
    }
    // transposed part (J rows only): column j0 + r gets sum over rows i > j of A(i, j) y_i
    if (sym) {
        const int j = tl.j0 + r;
        if (j < nd.s) {
            const int rmin = max(0, j - tl.i0 + 1), rmax = min(kT, nd.s - tl.i0);
            if (rmin < rmax) {
                Acc3 acc;
                acc.zero();
                for (int rr = rmin; rr < rmax; ++rr) acc.add(t[r][rr], yr, rr, kRq * q);
                double2* dst = X + static_cast<int64_t>(rb[j]) * k + c0;
#pragma unroll
                for (int u = 0; u < kRq; ++u)
                    if (kRq * q + u < nc) atomic_add2(dst + kRq * q + u, acc.get(u, 1.0));
            }
        }
    }
}

// Backward tile (i0, j0) of node J: x_J(j0 + c) -= sum over R rows s + i0 + t of L_RJ(t, c) x_R(t).
__global__ void __launch_bounds__(kSolveThreads) k_solve_bwd(const SolveNode* __restrict__ nodes,
                                                             const int32_t* __restrict__ rows,
                                                             const SolveTile* __restrict__ tiles,
                                                             const double2* __restrict__ F, double2* X, int k) {
    extern __shared__ double2 solve_smem[];
    auto t = reinterpret_cast<double2 (*)[kTP]>(solve_smem);
    RhsTile& xr = *reinterpret_cast<RhsTile*>(solve_smem + kT * kTP);
    const SolveTile tl = tiles[blockIdx.x];
    const SolveNode nd = nodes[tl.node];
    const int c0 = blockIdx.y * kSolveRhs;
    const int nc = min(kSolveRhs, k - c0);
    const int32_t* rb = rows + nd.row_off;
    load_tile(t, F + nd.front_off, nd.f, nd.s + tl.i0, nd.f, tl.j0, nd.s);
    load_rows(xr, X, rb + nd.s, tl.i0, nd.r, k, c0, nc);
    load_tile_wait();
    const int q = threadIdx.x >> 6, c = threadIdx.x & (kT - 1);
    const int j = tl.j0 + c;
    if (j >= nd.s || kRq * q >= nc) return;
    Acc3 acc;
    acc.zero();
    const int tmax = min(kT, nd.r - tl.i0);
    for (int tt = 0; tt < tmax; ++tt) acc.add(t[c][tt], xr, tt, kRq * q);
    double2* dst = X + static_cast<int64_t>(rb[j]) * k + c0;
#pragma unroll
    for (int u = 0; u < kRq; ++u)
        if (kRq * q + u < nc) atomic_add2(dst + kRq * q + u, acc.get(u, -1.0));
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
            const int32_t s = P.s[j], f = P.f[j], r = P.r[j];
            if (s == 0) continue;
            for (int32_t i0 = 0; i0 < f; i0 += kSolveTile)
                for (int32_t j0 = 0; j0 < s; j0 += kSolveTile)
                    if (i0 + kSolveTile > s || j0 <= i0) fwd.push_back(SolveTile{j, i0, j0, 0});
            for (int32_t i0 = 0; i0 < r; i0 += kSolveTile)
                for (int32_t j0 = 0; j0 < s; j0 += kSolveTile) bwd.push_back(SolveTile{j, i0, j0, 0});
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

constexpr size_t kFwdSmem = sizeof(double2) * kT * kTP + 2 * sizeof(RhsTile);
constexpr size_t kBwdSmem = sizeof(double2) * kT * kTP + sizeof(RhsTile);

cudaError_t launch_solve(const Plan& P, const SolveTables& T, const double2* fronts, double2* Y, double2* X, int k,
                         cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_solve_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kFwdSmem))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_solve_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kBwdSmem))) != cudaSuccess)
        return e;
    const unsigned gy = static_cast<unsigned>((k + kSolveRhs - 1) / kSolveRhs);
    e = cudaMemsetAsync(X, 0, sizeof(double2) * static_cast<size_t>(P.n) * k, st);
    if (e != cudaSuccess) return e;
    for (int32_t L = 0; L < P.n_levels; ++L) {
        const int64_t cnt = T.fwd_first[L + 1] - T.fwd_first[L];
        if (cnt == 0) continue;
        k_solve_fwd<<<dim3(static_cast<unsigned>(cnt), gy), kSolveThreads, kFwdSmem, st>>>(T.nodes, T.rows, T.fwd + T.fwd_first[L], fronts,
                                                                           Y, X, k);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int32_t L = P.n_levels - 1; L >= 0; --L) {
        const int64_t cnt = T.bwd_first[L + 1] - T.bwd_first[L];
        if (cnt == 0) continue;
        k_solve_bwd<<<dim3(static_cast<unsigned>(cnt), gy), kSolveThreads, kBwdSmem, st>>>(T.nodes, T.rows, T.bwd + T.bwd_first[L], fronts,
                                                                           X, k);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
