// C-ABI entry points of App. B: solves with the factors of a pole and selected eigenstates near
// an energy by block shift-invert iteration.
#include "handle.hpp"

namespace ndsi {

namespace {

int ensure_solve_tables(ndsi_plan* h) {
    if (h->ST.blob) return NDSI_OK;
    cudaError_t e = solve_tables_build(h->P, h->ST);
    if (e != cudaSuccess) {
        cudaGetLastError();
        solve_tables_free(h->ST);
        return fail(e == cudaErrorMemoryAllocation ? NDSI_ERR_OOM : NDSI_ERR_CUDA,
                    std::string("solve tables: ") + cudaGetErrorString(e));
    }
    return NDSI_OK;
}

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

// Uniform [-1, 1) numbers from a counter (splitmix64 finaliser) for the starting block.
double counter_uniform(uint64_t seed, uint64_t i) {
    uint64_t x = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return static_cast<double>(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Density of states from the retarded Green function (Eq. 41): D(E_k) = -(2/pi) Im Tr(G(E_k +
// i eta) S) for nE energies, one batched sweep of factorisation + selected inversion (chunked to
// the workspace) and a per-point trace on the pattern.  Host energies in, host D out.
}  // namespace
}  // namespace ndsi

extern "C" {

using namespace ndsi;

int ndsi_factors_solve(ndsi_factors* f, int32_t pole, const double* Y, int32_t k, double* X_out, void* stream) {
    if (!f || !f->plan || !Y || !X_out || k < 1 || pole < 0 || pole >= f->np)
        return fail(NDSI_ERR_INVALID, "ndsi_factors_solve: invalid argument");
    if (f->inverted) return fail(NDSI_ERR_INVALID, "ndsi_factors_solve: ndsi_selinv has overwritten the factors");
    ndsi_plan* h = f->plan;
    if (h->P.n_systems != 1) return fail(NDSI_ERR_INVALID, "ndsi_factors_solve: batched plan");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_solve_tables(h);
    if (rc) return rc;
    const int64_t elems = h->P.n * static_cast<int64_t>(k);
    const size_t bytes = sizeof(double2) * static_cast<size_t>(elems);
    if (f->solve_cap < elems) {  // kept with the factors: repeated solves allocate nothing
        if (f->solve_buf) cudaFree(f->solve_buf);
        f->solve_buf = nullptr;
        f->solve_cap = 0;
        NDSI_CK(cudaMalloc(&f->solve_buf, 2 * bytes));
        f->solve_cap = elems;
    }
    double2* yw = f->solve_buf;
    const bool x_dev = is_device_ptr(X_out);
    double2* xd = x_dev ? reinterpret_cast<double2*>(X_out) : f->solve_buf + f->solve_cap;
    NDSI_CK(cudaMemcpyAsync(yw, Y, bytes, cudaMemcpyDefault, st));
    NDSI_CK(launch_solve(h->P, h->ST, f->W.fronts + static_cast<int64_t>(pole) * f->W.front_stride, yw, xd, k, st));
    if (!x_dev) NDSI_CK(cudaMemcpyAsync(X_out, xd, bytes, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    return NDSI_OK;
}

int ndsi_eigenstates(ndsi_plan* h, const double* H, const double* S, double xi, double eta, int32_t n_states,
                     int32_t block, int32_t max_iter, double tol, uint64_t seed, double* eps_out, double* C_out,
                     double* resid_out, int32_t* iters_out, void* stream) {
    if (!h || !H || !S || !eps_out || !C_out || !std::isfinite(xi) || !(eta > 0) || !std::isfinite(eta) ||
        n_states < 1 || block < n_states || block > 32 || max_iter < 1 || !(tol > 0))
        return fail(NDSI_ERR_INVALID, "ndsi_eigenstates: invalid argument");
    if (h->P.n_systems != 1) return fail(NDSI_ERR_INVALID, "ndsi_eigenstates: batched plan");
    const int64_t n = h->P.n;
    if (block > n) return fail(NDSI_ERR_INVALID, "ndsi_eigenstates: block larger than the matrix");
    if (is_device_ptr(eps_out) || (resid_out && is_device_ptr(resid_out)))
        return fail(NDSI_ERR_INVALID, "ndsi_eigenstates: eps_out and resid_out are host arrays");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (!rc) rc = ensure_solve_tables(h);
    if (rc) return rc;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    // factor z S - H at z = xi + i eta (one point): A_J^{-1} and L_RJ stay in the workspace fronts
    const int32_t np = std::max<int32_t>(1, h->W.np_cap);
    rc = alloc_workspace(h->W, h->P, np);
    if (rc) return rc;
    if (h->P.opt.precision == NDSI_PREC_SPLIT) NDSI_CK(split_alloc(h->SB, h->SP.steps, h->P.opt.split_slices, np));
    if (!h->point_z) NDSI_CK(cudaMalloc(&h->point_z, sizeof(double2)));
    const double2 z = make_double2(xi, eta);
    NDSI_CK(cudaMemcpyAsync(h->point_z, &z, sizeof(double2), cudaMemcpyHostToDevice, st));
    rc = run_phase(h, h->W, h->SB, 0, Hd, Sd, h->point_z, 1, 1, st);
    if (rc) return rc;
    // buffers: complex right-hand sides and solutions, V = [Re B | Im B], H V, S V, the block C
    const int mmax = 2 * block;
    const int nb = gram_blocks(n);
    DevBuf yb, xb, rb, vb, hvb, svb, cb, gp, gram, yc, ec, rp;
    // the split path's factors are accurate to ~1e-9 relative: one refinement step per solve
    // restores FP64 accuracy, so the iteration converges to the pencil's own eigenpairs
    const int refine = h->P.opt.precision == NDSI_PREC_SPLIT ? 1 : 0;
    NDSI_CK(yb.alloc(sizeof(double2) * n * block));
    if (refine) NDSI_CK(rb.alloc(sizeof(double2) * n * block));
    NDSI_CK(xb.alloc(sizeof(double2) * n * block));
    NDSI_CK(vb.alloc(sizeof(double) * n * mmax));
    NDSI_CK(hvb.alloc(sizeof(double) * n * mmax));
    NDSI_CK(svb.alloc(sizeof(double) * n * mmax));
    NDSI_CK(cb.alloc(sizeof(double) * n * block));
    NDSI_CK(gp.alloc(sizeof(double) * nb * 2 * mmax * mmax));
    NDSI_CK(gram.alloc(sizeof(double) * 2 * mmax * mmax));
    NDSI_CK(yc.alloc(sizeof(double) * mmax * block));
    NDSI_CK(ec.alloc(sizeof(double) * block));
    NDSI_CK(rp.alloc(sizeof(double) * nb * block));
    int m = block;
    {
        std::vector<double> c0(static_cast<size_t>(n) * m);
        for (size_t i = 0; i < c0.size(); ++i) c0[i] = counter_uniform(seed, i);
        NDSI_CK(cudaMemcpyAsync(cb.p, c0.data(), sizeof(double) * c0.size(), cudaMemcpyHostToDevice, st));
        NDSI_CK(cudaStreamSynchronize(st));
    }
    std::vector<double> e, Y, res(block, 0.0), gh(2 * mmax * mmax);
    std::vector<int> order;
    int it = 0;
    bool done = false;
    while (!done && it < max_iter) {
        ++it;
        // (B2): b = (z S - H)^{-1} S c, the shift-invert product with the factors of z
        NDSI_CK(launch_spmm(h->T.rowptr, h->T.col, Sd, n, cb.as<double>(), m, vb.as<double>(), m, m, st));
        NDSI_CK(launch_real_to_complex(vb.as<double>(), n * m, yb.as<double2>(), st));
        NDSI_CK(launch_solve(h->P, h->ST, h->W.fronts, yb.as<double2>(), xb.as<double2>(), m, st));
        for (int r = 0; r < refine; ++r) {
            // iterative refinement in FP64: x += (zS - H)^{-1} (y - (zS - H) x)
            NDSI_CK(launch_real_to_complex(vb.as<double>(), n * m, yb.as<double2>(), st));
            NDSI_CK(launch_shifted_residual(h->T.rowptr, h->T.col, Hd, Sd, n, z, xb.as<double2>(), yb.as<double2>(),
                                            rb.as<double2>(), m, st));
            NDSI_CK(launch_solve(h->P, h->ST, h->W.fronts, rb.as<double2>(), yb.as<double2>(), m, st));
            NDSI_CK(launch_complex_add(xb.as<double2>(), yb.as<double2>(), n * m, st));
        }
        // (B3) in the real span of Re b and Im b
        const int m2 = 2 * m;
        NDSI_CK(launch_split_complex(xb.as<double2>(), n, m, vb.as<double>(), st));
        NDSI_CK(launch_spmm(h->T.rowptr, h->T.col, Hd, n, vb.as<double>(), m2, hvb.as<double>(), m2, m2, st));
        NDSI_CK(launch_spmm(h->T.rowptr, h->T.col, Sd, n, vb.as<double>(), m2, svb.as<double>(), m2, m2, st));
        NDSI_CK(launch_gram(vb.as<double>(), hvb.as<double>(), svb.as<double>(), n, m2, gp.as<double>(), gram.as<double>(),
                            st));
        NDSI_CK(cudaMemcpyAsync(gh.data(), gram.p, sizeof(double) * 2 * m2 * m2, cudaMemcpyDeviceToHost, st));
        NDSI_CK(cudaStreamSynchronize(st));
        rc = check_status(h, st);
        if (rc) return rc;
        for (double v : gh)
            if (!std::isfinite(v)) return fail(NDSI_ERR_SINGULAR, "ndsi_eigenstates: non-finite projected matrices");
        std::vector<double> Hs(gh.begin(), gh.begin() + m2 * m2), Ss(gh.begin() + m2 * m2, gh.begin() + 2 * m2 * m2);
        std::vector<double> ev, Yall;
        rayleigh_ritz(m2, Hs, Ss, ev, Yall);
        const int r = static_cast<int>(ev.size());
        if (r < n_states) return fail(NDSI_ERR_SINGULAR, "ndsi_eigenstates: search space collapsed");
        // keep the block's worth of Ritz pairs nearest xi
        order.resize(r);
        for (int i = 0; i < r; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return std::fabs(ev[a] - xi) < std::fabs(ev[b] - xi); });
        const int mn = std::min(m, r);
        e.resize(mn);
        Y.assign(static_cast<size_t>(m2) * mn, 0.0);
        for (int j = 0; j < mn; ++j) {
            e[j] = ev[order[j]];
            for (int a = 0; a < m2; ++a) Y[a * mn + j] = Yall[a * r + order[j]];
        }
        NDSI_CK(cudaMemcpyAsync(yc.p, Y.data(), sizeof(double) * Y.size(), cudaMemcpyHostToDevice, st));
        NDSI_CK(cudaMemcpyAsync(ec.p, e.data(), sizeof(double) * mn, cudaMemcpyHostToDevice, st));
        NDSI_CK(launch_ritz(vb.as<double>(), hvb.as<double>(), svb.as<double>(), n, m2, yc.as<double>(), ec.as<double>(), mn,
                            cb.as<double>(), rp.as<double>(), st));
        std::vector<double> part(static_cast<size_t>(nb) * mn);
        NDSI_CK(cudaMemcpyAsync(part.data(), rp.p, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st));
        NDSI_CK(cudaStreamSynchronize(st));
        m = mn;
        done = true;
        for (int j = 0; j < m; ++j) {
            double s2 = 0.0;
            for (int b = 0; b < nb; ++b) s2 += part[static_cast<size_t>(b) * m + j];
            res[j] = std::sqrt(s2);
            if (j < n_states && !(res[j] < tol)) done = false;
        }
    }
    // the n_states pairs nearest xi, ascending in energy, largest component of each made positive
    std::vector<int> sel(n_states);
    for (int j = 0; j < n_states; ++j) sel[j] = j;
    std::stable_sort(sel.begin(), sel.end(), [&](int a, int b) { return e[a] < e[b]; });
    std::vector<double> Ch(static_cast<size_t>(n) * m), out(static_cast<size_t>(n) * n_states);
    NDSI_CK(cudaMemcpyAsync(Ch.data(), cb.p, sizeof(double) * Ch.size(), cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    for (int j = 0; j < n_states; ++j) {
        const int c = sel[j];
        int64_t imax = 0;
        for (int64_t i = 1; i < n; ++i)
            if (std::fabs(Ch[i * m + c]) > std::fabs(Ch[imax * m + c])) imax = i;
        const double sg = Ch[imax * m + c] < 0 ? -1.0 : 1.0;
        for (int64_t i = 0; i < n; ++i) out[static_cast<size_t>(j) * n + i] = sg * Ch[i * m + c];
        eps_out[j] = e[c];
        if (resid_out) resid_out[j] = res[c];
    }
    NDSI_CK(cudaMemcpy(C_out, out.data(), sizeof(double) * out.size(), cudaMemcpyDefault));
    if (iters_out) *iters_out = it;
    if (!done) return fail(NDSI_ERR_TIMEOUT, "ndsi_eigenstates: not converged within max_iter (best pairs returned)");
    return NDSI_OK;
}

}  // extern "C"
