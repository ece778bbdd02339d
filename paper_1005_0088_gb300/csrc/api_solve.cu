// C-ABI entry points of App. B: solves with the factors of a pole and selected eigenstates near
// an energy by block shift-invert iteration.
#include "handle.hpp"
#include "small_eig.hpp"

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

// Uniform [-1, 1) numbers from a counter (splitmix64 finaliser) for the starting block.
double counter_uniform(uint64_t seed, uint64_t i) {
    uint64_t x = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return static_cast<double>(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

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
