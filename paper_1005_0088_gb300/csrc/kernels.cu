// FP64 kernels of the per-pole factor / selected-inversion path.
//
// Front layout: every supernode J owns a dense f x f complex front (f = |J| + |struct(J)|),
// column-major, J's columns first; only the lower triangle is kept valid.  All poles of a chunk
// are batched in one launch (grid.y = pole), each pole owning one slab of fronts and one slab
// of scratch.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "kernels.cuh"

namespace ndsi {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// ---------------------------------------------------------------------------------------------
// Front assembly: F_J = sum over children c of U_c (extend-add through the inverse relative
// index maps), written for the lower triangle of every front of a level.  Zero where no child
// contributes; the original entries are added afterwards by k_scatter.  One CTA per 32 x 32 tile
// (lanes = rows, 8 warps x 4 columns): the tile's column indices into each child are staged in
// shared memory first, so a thread's four column loads are independent and in flight together.
__global__ void __launch_bounds__(256) k_assemble(const NodeDev* __restrict__ nodes,
                                                  const NodeTile* __restrict__ tiles, int64_t first,
                                                  const int32_t* __restrict__ inv_map,
                                                  double2* __restrict__ F, int64_t stride) {
    static_assert(kNodeTile == 32, "one lane per tile row, 8 warps x 4 columns");
    constexpr int kCols = kNodeTile / 8;
    const NodeTile t = tiles[first + blockIdx.x];
    const NodeDev nd = nodes[t.node];
    double2* Fp = F + static_cast<int64_t>(blockIdx.y) * stride;
    __shared__ NodeDev ch[2];
    __shared__ int ibs[2][kNodeTile];
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (tx < nd.nchild && ty == 0) ch[tx] = nodes[nd.child[tx]];
    if (ty < nd.nchild) ibs[ty][tx] = t.j0 + tx < nd.f ? inv_map[nd.inv_off[ty] + t.j0 + tx] : -1;
    __syncthreads();
    const int a = t.i0 + tx;
    if (a >= nd.f) return;
    double2 v[kCols];
#pragma unroll
    for (int u = 0; u < kCols; ++u) v[u] = make_double2(0.0, 0.0);
    for (int c = 0; c < nd.nchild; ++c) {
        const int ia = inv_map[nd.inv_off[c] + a];
        if (ia < 0) continue;
        const NodeDev& cd = ch[c];
        const double2* U = Fp + cd.front_off + cd.s + ia + static_cast<int64_t>(cd.s) * cd.f;
#pragma unroll
        for (int u = 0; u < kCols; ++u) {
            const int q = ty + 8 * u;
            const int ib = ibs[c][q];
            if (ib >= 0 && t.j0 + q <= a) v[u] = cadd(v[u], U[static_cast<int64_t>(ib) * cd.f]);
        }
    }
#pragma unroll
    for (int u = 0; u < kCols; ++u) {
        const int b = t.j0 + ty + 8 * u;
        if (b <= a && b < nd.f) Fp[nd.front_off + a + static_cast<int64_t>(b) * nd.f] = v[u];
    }
}

// X = z S - H on the level's entries (each front element receives at most one entry).
// z[sys * zstride + pole] is the point of the entry's system (systems of a batch have their own
// mu and kT).
__global__ void __launch_bounds__(256) k_scatter(const int64_t* __restrict__ idx, int64_t first,
                                                 int64_t count, const int64_t* __restrict__ asm_map,
                                                 const int32_t* __restrict__ entry_sys,
                                                 const double* __restrict__ H,
                                                 const double* __restrict__ S,
                                                 const double2* __restrict__ z, int64_t zstride,
                                                 double2* __restrict__ F, int64_t stride) {
    double2* Fp = F + static_cast<int64_t>(blockIdx.y) * stride;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = idx[first + e];
        const int64_t off = asm_map[k];
        const double2 zq = z[entry_sys[k] * zstride + blockIdx.y];
        const double h = H[k], s = S[k];
        double2 v = Fp[off];
        v.x += zq.x * s - h;
        v.y += zq.y * s;
        Fp[off] = v;
    }
}

// FP64 inverse of a complex-symmetric pivot block (Gauss-Jordan sweeps without pivoting).
// No pivoting is needed: for Im z != 0 and S SPD, Im(X) = Im(z) S is definite, so every leading
// block and every Schur complement of X is nonsingular.  A zero or non-finite pivot sets the
// singular bit of the status word.
template <int NB>
__global__ void __launch_bounds__(256) k_diaginv(const DiagItem* __restrict__ items, int64_t first,
                                                 double2* __restrict__ F, int64_t stride,
                                                 int* __restrict__ status) {
    extern __shared__ double2 smem_dinv[];
    double2 (*a)[NB + 1] = reinterpret_cast<double2 (*)[NB + 1]>(smem_dinv);
    const DiagItem d = items[first + blockIdx.x];
    double2* A = F + static_cast<int64_t>(blockIdx.y) * stride + d.off;
    const int nb = d.nb, ld = d.ld;
    const int tid = threadIdx.x;
    if (nb > NB) {
        if (tid == 0) atomicOr(status, kStatusBadItem);
        return;
    }
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        a[i][j] = i >= j ? A[i + static_cast<int64_t>(j) * ld] : A[j + static_cast<int64_t>(i) * ld];
    }
    __syncthreads();
    constexpr int kPer = (NB * NB + 255) / 256;
    for (int t = 0; t < nb; ++t) {
        const double2 p = a[t][t];
        const double den = p.x * p.x + p.y * p.y;
        if (tid == 0 && !(den > 0.0 && isfinite(den))) atomicOr(status, kStatusSingular);
        const double2 ip = make_double2(p.x / den, -p.y / den);
        double2 nv[kPer];
        #pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int e = tid + u * 256;
            if (e < nb * nb) {
                const int i = e % nb, j = e / nb;
                if (i == t && j == t) {
                    nv[u] = ip;
                } else if (i == t) {
                    nv[u] = cmul(a[t][j], ip);
                } else if (j == t) {
                    const double2 v = cmul(a[i][t], ip);
                    nv[u] = make_double2(-v.x, -v.y);
                } else {
                    const double2 v = cmul(cmul(a[i][t], ip), a[t][j]);
                    nv[u] = make_double2(a[i][j].x - v.x, a[i][j].y - v.y);
                }
            }
        }
        __syncthreads();
        #pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int e = tid + u * 256;
            if (e < nb * nb) a[e % nb][e / nb] = nv[u];
        }
        __syncthreads();
    }
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        if (i >= j) A[i + static_cast<int64_t>(j) * ld] = a[i][j];
    }
}

// Register-resident variant for blocks of up to N = 16 or 32: one warp per (block, pole) running
// the symmetric sweep, the sign convention of Gauss-Jordan elimination that keeps a symmetric
// matrix symmetric.  Pivoting on t with p = a_tt maps a_tt -> -1/p, a_it and a_ti -> a_it/p and
// a_ik -> a_ik - a_it a_tk / p; after all pivots the block holds -A^{-1}.  Because every
// intermediate matrix is symmetric only the N(N+1)/2 lower-triangle elements are updated, half
// the FP64 work of the full elimination.  They are packed onto the lanes: virtual column c
// (c < N/2) is rows c..N-1 of column c followed by rows N-1-c..N-1 of column N-1-c (N+1
// elements), split evenly over 64/N lanes.  Every lane runs the same instruction stream (no
// divergent pivot lane); column t of the current matrix and its scaled copy pass through shared
// memory.  N = 16 serves launches whose pivot blocks are all at most 16 wide (small separators
// and the ragged last block of a front) at about a third of the N = 32 cost.
template <int N>
__global__ void __launch_bounds__(32) k_diaginv_sweep(const DiagItem* __restrict__ items, int64_t first,
                                                      double2* __restrict__ F, int64_t stride,
                                                      int* __restrict__ status) {
    constexpr int VC = N / 2;                  // virtual columns
    constexpr int LPC = 32 / VC;               // lanes per virtual column
    constexpr int SLOTS = (N + 1 + LPC - 1) / LPC;
    __shared__ double2 cs[33], ds[33];
    const int lane = threadIdx.x;
    const DiagItem d = items[first + blockIdx.x];
    double2* A = F + static_cast<int64_t>(blockIdx.y) * stride + d.off;
    const int nb = d.nb, ld = d.ld;
    if (nb > N) {
        if (lane == 0) atomicOr(status, kStatusBadItem);
        return;
    }
    const int c = lane % VC, vbase = (lane / VC) * SLOTS;
    int rc[SLOTS];  // row | column << 8 of each slot (32 = unused slot)
    double2 a[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const int v = vbase + s;
        int i = 32, k = 32;
        if (v < N - c) {
            i = c + v;
            k = c;
        } else if (v <= N) {
            i = v - 1;
            k = N - 1 - c;
        }
        rc[s] = i | (k << 8);
        a[s] = make_double2(0.0, 0.0);
        if (i < nb && k < nb) a[s] = A[i + static_cast<int64_t>(k) * ld];
    }
    if (lane == 0) {
        cs[32] = make_double2(0.0, 0.0);
        ds[32] = make_double2(0.0, 0.0);
    }
    bool bad = false;
    for (int t = 0; t < nb; ++t) {
        // column t (= row t) of the current matrix
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            const int i = rc[s] & 255, k = rc[s] >> 8;
            if (k == t) cs[i] = a[s];
            if (i == t) cs[k] = a[s];
        }
        __syncwarp();
        const double2 p = cs[t];
        const double den = p.x * p.x + p.y * p.y;
        bad |= !(den > 0.0 && isfinite(den));
        const double rden = 1.0 / den;
        const double2 ip = make_double2(p.x * rden, -p.y * rden);
        if (lane < N) ds[lane] = cmul(cs[lane], ip);
        __syncwarp();
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            const int i = rc[s] & 255, k = rc[s] >> 8;
            const double2 cv = cs[i], dk = ds[k];
            double2 g = make_double2(a[s].x - (cv.x * dk.x - cv.y * dk.y), a[s].y - (cv.x * dk.y + cv.y * dk.x));
            if (k == t) g = i == t ? make_double2(-ip.x, -ip.y) : ds[i];
            else if (i == t) g = dk;
            a[s] = g;
        }
        __syncwarp();
    }
    if (bad && lane == 0) atomicOr(status, kStatusSingular);
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const int i = rc[s] & 255, k = rc[s] >> 8;
        if (i < nb && k < nb) A[i + static_cast<int64_t>(k) * ld] = make_double2(-a[s].x, -a[s].y);
    }
}

// ---------------------------------------------------------------------------------------------
// Batched complex FP64 GEMM on the CUDA cores: C = alpha op(A) op(B) + beta C for every tile of
// a schedule step.  TILE x TILE output tile (32, or 16 for launches of small items, where a 32
// tile would spend its multiply-adds on padding), K step 16, 64 threads with (TILE/8)^2 outputs
// each.  The complex product uses three real products per element (Re = P1 - P2,
// Im = P3 - P1 - P2 with P1 = Ar Br, P2 = Ai Bi, P3 = (Ar + Ai)(Br + Bi)): GB300's FP64 rate is
// the bound here, and the third real product saves a quarter of the DFMAs.
constexpr int BK = 16;

template <int OP>
__device__ __forceinline__ double2 load_op(const double2* __restrict__ X, int ld, int r, int c) {
    if (OP == OP_N) return X[r + static_cast<int64_t>(c) * ld];
    if (OP == OP_T) return X[c + static_cast<int64_t>(r) * ld];
    const int hi = r > c ? r : c, lo = r > c ? c : r;
    return X[hi + static_cast<int64_t>(lo) * ld];
}

template <int OPA, int OPB, int TILE>
__global__ void __launch_bounds__(64) k_gemm_f64(const GemmItem* __restrict__ items,
                                                 const GemmTile* __restrict__ tiles, int64_t tfirst,
                                                 int64_t ifirst, const double2* __restrict__ Abuf,
                                                 int64_t sA, const double2* __restrict__ Bbuf,
                                                 int64_t sB, double2* __restrict__ Cbuf, int64_t sC,
                                                 double alpha, double beta, int lower) {
    constexpr int MT = TILE / 8;           // outputs per thread along each edge
    constexpr int LD = TILE * BK / 64;     // operand elements each thread stages per K step
    __shared__ double As[3][BK][TILE + 1];
    __shared__ double Bs[3][BK][TILE + 1];
    const GemmTile t = tiles[tfirst + blockIdx.x];
    const GemmItem it = items[ifirst + t.item];
    const int64_t pole = blockIdx.y;
    const double2* A = Abuf + pole * sA + it.a_off;
    const double2* B = Bbuf + pole * sB + it.b_off;
    double2* C = Cbuf + pole * sC + it.c_off;
    const int tid = threadIdx.x;
    const int tx = tid % 8, ty = tid / 8;
    double p1[MT][MT], p2[MT][MT], p3[MT][MT];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) p1[i][j] = p2[i][j] = p3[i][j] = 0.0;
    for (int k0 = 0; k0 < it.K; k0 += BK) {
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int e = tid + 64 * u;
            int lm, lk;
            if (OPA == OP_T) {
                lk = e % BK;
                lm = e / BK;
            } else {
                lm = e % TILE;
                lk = e / TILE;
            }
            const int m = t.m0 + lm, k = k0 + lk;
            const double2 v = (m < it.M && k < it.K) ? load_op<OPA>(A, it.lda, m, k) : make_double2(0.0, 0.0);
            As[0][lk][lm] = v.x;
            As[1][lk][lm] = v.y;
            As[2][lk][lm] = v.x + v.y;
        }
#pragma unroll
        for (int u = 0; u < LD; ++u) {
            const int e = tid + 64 * u;
            int ln, lk;
            if (OPB == OP_T) {
                ln = e % TILE;
                lk = e / TILE;
            } else {
                lk = e % BK;
                ln = e / BK;
            }
            const int n = t.n0 + ln, k = k0 + lk;
            const double2 v = (n < it.N && k < it.K) ? load_op<OPB>(B, it.ldb, k, n) : make_double2(0.0, 0.0);
            Bs[0][lk][ln] = v.x;
            Bs[1][lk][ln] = v.y;
            Bs[2][lk][ln] = v.x + v.y;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < BK; ++kk) {
            double ar[MT], ai[MT], as[MT], br[MT], bi[MT], bs[MT];
#pragma unroll
            for (int i = 0; i < MT; ++i) {
                ar[i] = As[0][kk][tx + 8 * i];
                ai[i] = As[1][kk][tx + 8 * i];
                as[i] = As[2][kk][tx + 8 * i];
            }
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                br[j] = Bs[0][kk][ty + 8 * j];
                bi[j] = Bs[1][kk][ty + 8 * j];
                bs[j] = Bs[2][kk][ty + 8 * j];
            }
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int j = 0; j < MT; ++j) {
                    p1[i][j] = fma(ar[i], br[j], p1[i][j]);
                    p2[i][j] = fma(ai[i], bi[j], p2[i][j]);
                    p3[i][j] = fma(as[i], bs[j], p3[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < MT; ++j) {
        const int n = t.n0 + ty + 8 * j;
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            const int m = t.m0 + tx + 8 * i;
            if (m < it.M && n < it.N && (!lower || m >= n)) {
                double2* c = C + m + static_cast<int64_t>(n) * it.ldc;
                const double re = p1[i][j] - p2[i][j];
                const double im = p3[i][j] - p1[i][j] - p2[i][j];
                double2 v = make_double2(alpha * re, alpha * im);
                if (beta != 0.0) {
                    const double2 old = *c;
                    v.x += beta * old.x;
                    v.y += beta * old.y;
                }
                *c = v;
            }
        }
    }
}

// dst = scale * src for the blocks of a step (SCR -> FRONT).
__global__ void __launch_bounds__(256) k_copy(const CopyItem* __restrict__ items, int64_t first,
                                              const double2* __restrict__ src, int64_t s_src,
                                              double2* __restrict__ dst, int64_t s_dst, double scale) {
    const CopyItem c = items[first + blockIdx.x];
    const double2* S = src + static_cast<int64_t>(blockIdx.y) * s_src + c.src_off;
    double2* D = dst + static_cast<int64_t>(blockIdx.y) * s_dst + c.dst_off;
    // the block's rows x cols elements (column-major, < 2^31) in gridDim.z contiguous ranges, so
    // that short columns still occupy every thread
    const uint32_t rows = static_cast<uint32_t>(c.rows);
    const uint32_t total = rows * static_cast<uint32_t>(c.cols);
    const uint32_t per = (total + gridDim.z - 1) / gridDim.z;
    const uint32_t e0 = blockIdx.z * per, e1 = min(total, e0 + per);
#pragma unroll 4
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const uint32_t j = e / rows, i = e - j * rows;
        const double2 v = S[i + static_cast<int64_t>(j) * c.lds];
        D[i + static_cast<int64_t>(j) * c.ldd] = make_double2(scale * v.x, scale * v.y);
    }
}

// G_RR of a node from the full (lower-valid) G front of its parent (Eq. 38's reuse of
// ancestor blocks), through the node's relative index map.
__global__ void __launch_bounds__(256) k_gather(const NodeDev* __restrict__ nodes,
                                                const NodeTile* __restrict__ tiles, int64_t first,
                                                const int32_t* __restrict__ rel_map,
                                                double2* __restrict__ F, int64_t stride) {
    const NodeTile t = tiles[first + blockIdx.x];
    const NodeDev nd = nodes[t.node];
    const NodeDev pd = nodes[nd.parent];
    double2* Fp = F + static_cast<int64_t>(blockIdx.y) * stride;
    const int i = t.i0 + threadIdx.x;
    if (i >= nd.r) return;
    const int ra = rel_map[nd.rel_off + i];
    for (int q = threadIdx.y; q < kNodeTile; q += blockDim.y) {
        const int j = t.j0 + q;
        if (j > i) continue;
        const int rb = rel_map[nd.rel_off + j];
        Fp[nd.front_off + (nd.s + i) + static_cast<int64_t>(nd.s + j) * nd.f] =
            Fp[pd.front_off + ra + static_cast<int64_t>(rb) * pd.f];
    }
}

// Residue sum of Eq. 8 on the pattern: rho_k (+)= sum_q Re(c_q G_q(k)); per-block partial sums
// of rho_k S_k for Tr(rho S) (Eq. 40), reduced in a fixed order by k_reduce.
constexpr int kAccThreads = 256;

__global__ void __launch_bounds__(kAccThreads) k_accumulate(const int64_t* __restrict__ out_map,
                                                            int64_t k0, int64_t nnz,
                                                            const double2* __restrict__ F,
                                                            int64_t stride, int np,
                                                            const double2* __restrict__ c,
                                                            const double* __restrict__ S,
                                                            double* __restrict__ rho, int accumulate,
                                                            int want_trace,
                                                            double* __restrict__ partials) {
    __shared__ double red[kAccThreads / 32];
    const int64_t k = k0 + blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    double tr = 0.0;
    if (k < k0 + nnz) {
        const int64_t off = out_map[k];
        double sum = accumulate ? rho[k] : 0.0;
        for (int q = 0; q < np; ++q) {
            const double2 g = F[static_cast<int64_t>(q) * stride + off];
            const double2 w = c[q];
            sum += w.x * g.x - w.y * g.y;
        }
        rho[k] = sum;
        tr = sum * S[k];
    }
    if (!want_trace) return;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kAccThreads / 32 ? red[threadIdx.x] : 0.0;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) k_reduce(const double* __restrict__ partials, int n,
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

__global__ void __launch_bounds__(256) k_gather_pattern(const int64_t* __restrict__ out_map,
                                                        int64_t nnz,
                                                        const double2* __restrict__ F,
                                                        int64_t stride, double2* __restrict__ G,
                                                        int64_t q0) {
    const int64_t q = blockIdx.y;
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nnz;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        G[(q0 + q) * nnz + k] = F[q * stride + out_map[k]];
}

template <int OPA, int OPB>
cudaError_t gemm_launch(const Plan& P, const DevTables& T, const Launch& l, const Workspace& W,
                        int np, cudaStream_t st) {
    const double2* bufs[2] = {W.fronts, W.scr};
    const int64_t strides[2] = {W.front_stride, W.scr_stride};
    dim3 grid(static_cast<unsigned>(l.tcount), static_cast<unsigned>(np));
    if (l.tile == kGemmTileSmall)
        k_gemm_f64<OPA, OPB, kGemmTileSmall><<<grid, 64, 0, st>>>(
            T.gemm_items, T.gemm_tiles, l.tfirst, l.first, bufs[l.bufA], strides[l.bufA], bufs[l.bufB],
            strides[l.bufB], const_cast<double2*>(bufs[l.bufC]), strides[l.bufC], l.alpha, l.beta, l.lower);
    else
        k_gemm_f64<OPA, OPB, kGemmTile><<<grid, 64, 0, st>>>(
            T.gemm_items, T.gemm_tiles, l.tfirst, l.first, bufs[l.bufA], strides[l.bufA], bufs[l.bufB],
            strides[l.bufB], const_cast<double2*>(bufs[l.bufC]), strides[l.bufC], l.alpha, l.beta, l.lower);
    (void)P;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(const Plan& P, const DevTables& T, const Launch& l, const Workspace& W,
                        const double* H, const double* S, const double2* z, int64_t zstride, int np,
                        cudaStream_t st) {
    switch (l.kind) {
        case L_ASSEMBLE: {
            dim3 grid(static_cast<unsigned>(l.count), static_cast<unsigned>(np));
            k_assemble<<<grid, dim3(32, 8), 0, st>>>(T.nodes, T.node_tiles, l.first, T.inv_map, W.fronts,
                                                    W.front_stride);
            return cudaGetLastError();
        }
        case L_SCATTER: {
            const int64_t blocks = (l.count + 255) / 256;
            dim3 grid(static_cast<unsigned>(blocks < 4096 ? blocks : 4096), static_cast<unsigned>(np));
            k_scatter<<<grid, 256, 0, st>>>(T.scatter_idx, l.first, l.count, T.asm_map, T.entry_sys, H, S, z,
                                            zstride, W.fronts, W.front_stride);
            return cudaGetLastError();
        }
        case L_DIAGINV: {
            dim3 grid(static_cast<unsigned>(l.count), static_cast<unsigned>(np));
            const int b = P.block;
            const size_t sm = static_cast<size_t>(b) * (b + 1) * sizeof(double2);
            if (b <= 32) {
                if (l.tile == 16)
                    k_diaginv_sweep<16><<<grid, 32, 0, st>>>(T.diag_items, l.first, W.fronts, W.front_stride, T.status);
                else
                    k_diaginv_sweep<32><<<grid, 32, 0, st>>>(T.diag_items, l.first, W.fronts, W.front_stride, T.status);
            } else {
                k_diaginv<64><<<grid, 256, sm, st>>>(T.diag_items, l.first, W.fronts, W.front_stride, T.status);
            }
            return cudaGetLastError();
        }
        case L_GEMM: {
            if (l.opA == OP_N && l.opB == OP_S) return gemm_launch<OP_N, OP_S>(P, T, l, W, np, st);
            if (l.opA == OP_N && l.opB == OP_T) return gemm_launch<OP_N, OP_T>(P, T, l, W, np, st);
            if (l.opA == OP_S && l.opB == OP_N) return gemm_launch<OP_S, OP_N>(P, T, l, W, np, st);
            if (l.opA == OP_T && l.opB == OP_N) return gemm_launch<OP_T, OP_N>(P, T, l, W, np, st);
            return cudaErrorInvalidValue;
        }
        case L_COPY: {
            // column slices per item: launches of few items (the upper tree levels) would
            // otherwise leave most SMs idle
            const unsigned zc = l.count * np < 4 * 152 ? 32u : 8u;
            dim3 grid(static_cast<unsigned>(l.count), static_cast<unsigned>(np), zc);
            k_copy<<<grid, 256, 0, st>>>(T.copy_items, l.first, W.scr, W.scr_stride, W.fronts, W.front_stride,
                                         l.alpha);
            return cudaGetLastError();
        }
        case L_GATHER: {
            dim3 grid(static_cast<unsigned>(l.count), static_cast<unsigned>(np));
            k_gather<<<grid, dim3(32, 8), 0, st>>>(T.nodes, T.node_tiles, l.first, T.rel_map, W.fronts,
                                                  W.front_stride);
            return cudaGetLastError();
        }
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t kernels_init() {
    const int sm64 = 64 * 65 * static_cast<int>(sizeof(double2));
    return cudaFuncSetAttribute(k_diaginv<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm64);
}

int accumulate_blocks(int64_t nnz) { return static_cast<int>((nnz + kAccThreads - 1) / kAccThreads); }

cudaError_t launch_accumulate(const Plan& P, const DevTables& T, const Workspace& W, int np,
                              const double2* c, const double* S, double* rho, int accumulate,
                              int want_trace, double* partials, cudaStream_t st, int64_t k0, int64_t count) {
    if (count < 0) {
        k0 = 0;
        count = P.nnz;
    }
    const int blocks = accumulate_blocks(count);
    k_accumulate<<<blocks, kAccThreads, 0, st>>>(T.out_map, k0, count, W.fronts, W.front_stride, np, c, S, rho,
                                                 accumulate, want_trace, partials);
    return cudaGetLastError();
}

// Order-preserving map of doubles to unsigned keys (larger double -> larger key).
__host__ __device__ inline unsigned long long order_key(double x) {
    unsigned long long u;
    memcpy(&u, &x, sizeof(u));
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(256) k_gershgorin(const int64_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, int64_t n,
                                                    const double* __restrict__ H,
                                                    const double* __restrict__ S,
                                                    unsigned long long* __restrict__ out) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    double h = 0.0, soff = 0.0, sdiag = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        h += fabs(H[k]);
        if (col[k] == i) sdiag = S[k];
        else soff += fabs(S[k]);
    }
    atomicMax(&out[0], order_key(h));
    atomicMax(&out[1], order_key(soff - sdiag));
}

cudaError_t launch_gershgorin(const DevTables& T, int64_t n, const double* H, const double* S,
                              unsigned long long* out, cudaStream_t st) {
    const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
    k_gershgorin<<<blocks, 256, 0, st>>>(T.rowptr, T.col, n, H, S, out);
    return cudaGetLastError();
}

double gershgorin_value(unsigned long long key) {
    const unsigned long long u = (key >> 63) ? (key & 0x7FFFFFFFFFFFFFFFull) : ~key;
    double x;
    memcpy(&x, &u, sizeof(x));
    return x;
}

__global__ void __launch_bounds__(kAccThreads) k_point_traces(const int64_t* __restrict__ out_map, int64_t nnz,
                                                              const double2* __restrict__ F, int64_t stride,
                                                              const double* __restrict__ S,
                                                              double* __restrict__ partials) {
    __shared__ double red[kAccThreads / 32];
    const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    double v = 0.0;
    if (k < nnz) v = F[static_cast<int64_t>(blockIdx.y) * stride + out_map[k]].y * S[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < kAccThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) partials[static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x] = w;
    }
}

cudaError_t launch_point_traces_range(const int64_t* out_map, int64_t nnz, const double2* F, int64_t stride, int np,
                                      const double* S, double* partials, double* out, cudaStream_t st) {
    if (nnz <= 0 || np <= 0) return cudaSuccess;
    const int nb = accumulate_blocks(nnz);
    k_point_traces<<<dim3(static_cast<unsigned>(nb), static_cast<unsigned>(np)), kAccThreads, 0, st>>>(
        out_map, nnz, F, stride, S, partials);
    cudaError_t e = cudaGetLastError();
    for (int q = 0; q < np && e == cudaSuccess; ++q) {
        k_reduce<<<1, 1024, 0, st>>>(partials + static_cast<int64_t>(q) * nb, nb, out + q);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_point_traces(const Plan& P, const DevTables& T, const Workspace& W, int np, const double* S,
                                double* partials, double* out, cudaStream_t st) {
    return launch_point_traces_range(T.out_map, P.nnz, W.fronts, W.front_stride, np, S, partials, out, st);
}

cudaError_t launch_reduce(const double* partials, int nblocks, double* out, cudaStream_t st) {
    k_reduce<<<1, 1024, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_pattern(const Plan& P, const DevTables& T, const Workspace& W, int np,
                                  double2* G_out, int64_t q0, cudaStream_t st) {
    const int64_t blocks = (P.nnz + 255) / 256;
    dim3 grid(static_cast<unsigned>(blocks < 2048 ? blocks : 2048), static_cast<unsigned>(np));
    k_gather_pattern<<<grid, 256, 0, st>>>(T.out_map, P.nnz, W.fronts, W.front_stride, G_out, q0);
    return cudaGetLastError();
}

}  // namespace ndsi
