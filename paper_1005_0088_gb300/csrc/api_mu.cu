// C-ABI entry points of the chemical-potential search (Sec. II.C.3): density of states from the
// retarded Green function (Eq. 41), single-system and lockstep batched searches.
#include "handle.hpp"

namespace ndsi {

namespace {

// Gershgorin bounds of the pencil (H, S) over basis rows [i0, i1) (host values on the pattern):
// every generalised eigenvalue lies in [elo, ehi] when S is diagonally dominant there.
void pencil_bounds(const Plan& P, const std::vector<double>& hv, const std::vector<double>& sv, int64_t i0, int64_t i1,
                   double* elo, double* ehi) {
    double hlo = 1e300, hhi = -1e300, slo = 1e300, shi = -1e300;
    for (int64_t i = i0; i < i1; ++i) {
        double hd = 0, sd = 0, hr = 0, sr = 0;
        for (int64_t k = P.rowptr[i]; k < P.rowptr[i + 1]; ++k) {
            if (P.col[k] == i) {
                hd = hv[k];
                sd = sv[k];
            } else {
                hr += std::fabs(hv[k]);
                sr += std::fabs(sv[k]);
            }
        }
        hlo = std::min(hlo, hd - hr);
        hhi = std::max(hhi, hd + hr);
        slo = std::min(slo, sd - sr);
        shi = std::max(shi, sd + sr);
    }
    if (slo > 0) {
        *elo = hlo / (hlo < 0 ? slo : shi);
        *ehi = hhi / (hhi > 0 ? slo : shi);
    } else {
        *elo = hlo < 0 ? hlo * 4 : -1.0;  // S not diagonally dominant: generous guess
        *ehi = hhi > 0 ? hhi * 4 : 1.0;
    }
}

// Callbacks of the lockstep search over the systems of a batched plan: one batched contour sweep
// per evaluation round, one batched retarded-Green-function sweep for the density of states.
struct FindMuBatchCtx {
    ndsi_plan* h;
    const double *Hd, *Sd;
    const double* kT;
    int32_t n_poles;
    const double* n_electrons;
    double *rho_d, *ne_d;
    cudaStream_t st;
    std::vector<double> last_mu;
};

int find_mu_eval_batch(void* c, int32_t ns, const int32_t* active, const double* mu, double* dn) {
    (void)active;
    FindMuBatchCtx& x = *static_cast<FindMuBatchCtx*>(c);
    int r = density_impl(x.h, x.Hd, x.Sd, mu, x.kT, x.n_poles, x.rho_d, x.ne_d, x.st);
    if (r) return r;
    std::vector<double> ne(ns);
    if (cudaMemcpy(ne.data(), x.ne_d, sizeof(double) * ns, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(NDSI_ERR_CUDA, "ndsi_find_mu_batched: readback failed");
    x.last_mu.assign(mu, mu + ns);
    for (int32_t sy = 0; sy < ns; ++sy) dn[sy] = ne[sy] - x.n_electrons[sy];
    return NDSI_OK;
}

int find_mu_dos_batch(void* c, int32_t ns, const int32_t* active, const double* E, int32_t n, const double* eta,
                      double* D) {
    (void)ns;
    (void)active;
    FindMuBatchCtx& x = *static_cast<FindMuBatchCtx*>(c);
    return dos_sweep_systems(x.h, x.Hd, x.Sd, E, n, eta, D, x.st);
}

// Callbacks of the chemical-potential search: DeltaN from one contour evaluation, and the
// density of states from one sweep of the retarded Green function.
struct FindMuCtx {
    ndsi_plan* h;
    const double *Hd, *Sd;
    double kT;
    int32_t n_poles;
    double n_electrons;
    double *rho_d, *ne_d;
    cudaStream_t st;
    double last_mu;
    bool have_last;
};

int find_mu_eval(void* c, double mu, double* dn) {
    FindMuCtx& x = *static_cast<FindMuCtx*>(c);
    int r = density_impl(x.h, x.Hd, x.Sd, &mu, &x.kT, x.n_poles, x.rho_d, x.ne_d, x.st);
    if (r) return r;
    double ne = 0;
    if (cudaMemcpy(&ne, x.ne_d, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(NDSI_ERR_CUDA, "ndsi_find_mu: readback failed");
    x.last_mu = mu;
    x.have_last = true;
    *dn = ne - x.n_electrons;
    return NDSI_OK;
}

int find_mu_dos(void* c, const double* E, int32_t n, double eta, double* D) {
    FindMuCtx& x = *static_cast<FindMuCtx*>(c);
    return dos_sweep(x.h, x.Hd, x.Sd, E, n, eta, D, x.st);
}

}  // namespace

// Density of states of every system of the plan on its own grid (E and D row-major systems x nE,
// eta per system): one sweep over the points, traces per system on its pattern range.
int dos_sweep_systems(ndsi_plan* h, const double* Hd, const double* Sd, const double* E, int nE, const double* eta,
                      double* D, cudaStream_t st) {
    const int32_t ns = h->P.n_systems;
    const int64_t npts = static_cast<int64_t>(ns) * nE;
    std::vector<double2> z(npts);
    for (int32_t sy = 0; sy < ns; ++sy)
        for (int k = 0; k < nE; ++k) z[static_cast<size_t>(sy) * nE + k] = make_double2(E[static_cast<size_t>(sy) * nE + k], eta[sy]);
    const int64_t per_pole = bytes_per_pole(h);
    const int64_t cap = workspace_cap(h);
    if (cap < per_pole) return fail(NDSI_ERR_OOM, "ndsi_dos: one point does not fit the workspace cap");
    const int32_t chunk = static_cast<int32_t>(std::min<int64_t>(nE, std::max<int64_t>(1, cap / per_pole)));
    int rc = alloc_workspace(h->W, h->P, std::max<int32_t>(chunk, h->W.np_cap));
    if (rc) return rc;
    if (h->P.opt.precision == NDSI_PREC_SPLIT)
        NDSI_CK(split_alloc(h->SB, h->SP.steps, h->P.opt.split_slices, std::max<int32_t>(chunk, h->W.np_cap)));
    // trace partials: one chunk of points times the blocks of the largest system's pattern range
    int64_t nb = 1;
    for (int32_t sy = 0; sy < ns; ++sy)
        nb = std::max<int64_t>(nb, accumulate_blocks(h->P.sys_nnz_first[sy + 1] - h->P.sys_nnz_first[sy]));
    const int64_t part_need = static_cast<int64_t>(chunk) * nb;
    if (h->dos_cap < npts || h->dos_part_cap < part_need) {
        if (h->dos_part) cudaFree(h->dos_part);
        if (h->dos_tr) cudaFree(h->dos_tr);
        if (h->dos_z) cudaFree(h->dos_z);
        h->dos_part = h->dos_tr = nullptr;
        h->dos_z = nullptr;
        h->dos_cap = h->dos_part_cap = 0;
        NDSI_CK(cudaMalloc(&h->dos_part, sizeof(double) * static_cast<size_t>(part_need)));
        NDSI_CK(cudaMalloc(&h->dos_tr, sizeof(double) * (npts + 1)));
        NDSI_CK(cudaMalloc(&h->dos_z, sizeof(double2) * npts));
        h->dos_cap = npts;
        h->dos_part_cap = part_need;
    }
    NDSI_CK(cudaMemcpyAsync(h->dos_z, z.data(), sizeof(double2) * npts, cudaMemcpyHostToDevice, st));
    for (int q0 = 0; q0 < nE; q0 += chunk) {
        const int np = std::min(chunk, nE - q0);
        rc = run_phase(h, h->W, h->SB, 0, Hd, Sd, h->dos_z + q0, nE, np, st);
        if (!rc) rc = run_phase(h, h->W, h->SB, 1, Hd, Sd, h->dos_z + q0, nE, np, st);
        if (rc) return rc;
        for (int32_t sy = 0; sy < ns; ++sy) {
            const int64_t k0 = h->P.sys_nnz_first[sy], k1 = h->P.sys_nnz_first[sy + 1];
            NDSI_CK(launch_point_traces_range(h->T.out_map + k0, k1 - k0, h->W.fronts, h->W.front_stride, np, Sd + k0,
                                              h->dos_part, h->dos_tr + static_cast<int64_t>(sy) * nE + q0, st));
        }
    }
    std::vector<double> tr(npts);
    NDSI_CK(cudaMemcpyAsync(tr.data(), h->dos_tr, sizeof(double) * npts, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    rc = check_status(h, st);
    if (rc) return rc;
    for (int64_t k = 0; k < npts; ++k) D[k] = (-2.0 / M_PI) * tr[k];
    return NDSI_OK;
}

// Density of states from the retarded Green function (Eq. 41) of a single-system plan.
int dos_sweep(ndsi_plan* h, const double* Hd, const double* Sd, const double* E, int nE, double eta,
              double* D, cudaStream_t st) {
    return dos_sweep_systems(h, Hd, Sd, E, nE, &eta, D, st);
}

}  // namespace ndsi

extern "C" {

using namespace ndsi;

int ndsi_dos(ndsi_plan* h, const double* H, const double* S, const double* energies, int32_t n_energies,
             double eta, double* dos_out, void* stream) {
    if (!h || !H || !S || !energies || !dos_out || n_energies < 1 || !(eta > 0) || !std::isfinite(eta))
        return fail(NDSI_ERR_INVALID, "ndsi_dos: invalid argument");
    if (h->P.n_systems != 1) return fail(NDSI_ERR_INVALID, "ndsi_dos: batched plan");
    if (is_device_ptr(energies) || is_device_ptr(dos_out))
        return fail(NDSI_ERR_INVALID, "ndsi_dos: energies and dos_out are host arrays");
    for (int32_t k = 0; k < n_energies; ++k)
        if (!std::isfinite(energies[k])) return fail(NDSI_ERR_INVALID, "ndsi_dos: energy not finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    return dos_sweep(h, Hd, Sd, energies, n_energies, eta, dos_out, st);
}

int ndsi_find_mu(ndsi_plan* h, const double* H, const double* S, double kT, int32_t n_poles,
                 double n_electrons, double mu_lo, double mu_hi, double tol_electrons, int32_t max_iter,
                 double* rho_out, double* mu_out, double* n_elec_out, int32_t* iters_out, void* stream) {
    if (!h || !H || !S || !rho_out || !mu_out || n_poles < 1 || !(kT > 0) || !(tol_electrons > 0) ||
        max_iter < 1 || !std::isfinite(n_electrons) || h->P.n_systems != 1)
        return fail(NDSI_ERR_INVALID, "ndsi_find_mu: invalid argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const int64_t nnz = h->P.nnz;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    // Gershgorin bounds of H and S -> bounds of the pencil's spectrum (host, O(nnz))
    std::vector<double> hv(nnz), sv(nnz);
    NDSI_CK(cudaMemcpyAsync(hv.data(), Hd, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaMemcpyAsync(sv.data(), Sd, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    double elo, ehi;
    pencil_bounds(h->P, hv, sv, 0, h->P.n, &elo, &ehi);
    rc = ensure_stage(h, 3 * nnz + 8);
    if (rc) return rc;
    const bool rho_dev = is_device_ptr(rho_out);
    double* rho_d = rho_dev ? rho_out : h->stage + 2 * nnz;
    double* ne_d = h->stage + 3 * nnz;
    FindMuCtx ctx{h, Hd, Sd, kT, n_poles, n_electrons, rho_d, ne_d, st, 0.0, false};
    double mu = 0, dn = 0;
    int32_t iters = 0;
    std::string err;
    rc = mu_search(find_mu_eval, find_mu_dos, &ctx, elo, ehi, kT, n_electrons, n_poles + 1, mu_lo, mu_hi,
                   tol_electrons, max_iter, &mu, &dn, &iters, err);
    if (rc && rc != NDSI_ERR_TIMEOUT) return err.empty() ? rc : fail(rc, "ndsi_find_mu: " + err);
    // rho_out must hold rho(mu): evaluate once more if the last trial was another point
    if (!ctx.have_last || ctx.last_mu != mu) {
        double dn2 = 0;
        const int r2 = find_mu_eval(&ctx, mu, &dn2);
        if (r2) return r2;
    }
    *mu_out = mu;
    if (n_elec_out) *n_elec_out = n_electrons + dn;
    if (iters_out) *iters_out = iters;
    if (!rho_dev) NDSI_CK(cudaMemcpyAsync(rho_out, rho_d, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    if (rc) return fail(rc, "ndsi_find_mu: not converged within max_iter evaluations");
    return NDSI_OK;
}

int ndsi_find_mu_batched(ndsi_plan* h, const double* H, const double* S, const double* kT, int32_t n_poles,
                         const double* n_electrons, const double* mu_lo, const double* mu_hi, double tol_electrons,
                         int32_t max_iter, double* rho_out, double* mu_out, double* n_elec_out, int32_t* rounds_out,
                         void* stream) {
    if (!h || !H || !S || !kT || !n_electrons || !rho_out || !mu_out || n_poles < 1 || !(tol_electrons > 0) ||
        max_iter < 1)
        return fail(NDSI_ERR_INVALID, "ndsi_find_mu_batched: invalid argument");
    const int32_t ns = h->P.n_systems;
    for (int32_t sy = 0; sy < ns; ++sy)
        if (!(kT[sy] > 0) || !std::isfinite(n_electrons[sy]))
            return fail(NDSI_ERR_INVALID, "ndsi_find_mu_batched: kT <= 0 or non-finite electron count");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload_tables(h);
    if (rc) return rc;
    const int64_t nnz = h->P.nnz;
    const double *Hd, *Sd;
    rc = device_inputs(h, H, S, &Hd, &Sd, st);
    if (rc) return rc;
    std::vector<double> hv(nnz), sv(nnz);
    NDSI_CK(cudaMemcpyAsync(hv.data(), Hd, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaMemcpyAsync(sv.data(), Sd, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    std::vector<double> elo(ns), ehi(ns);
    for (int32_t sy = 0; sy < ns; ++sy)
        pencil_bounds(h->P, hv, sv, h->P.sys_n_first[sy], h->P.sys_n_first[sy + 1], &elo[sy], &ehi[sy]);
    rc = ensure_stage(h, 3 * nnz + 8 + ns);
    if (rc) return rc;
    const bool rho_dev = is_device_ptr(rho_out);
    double* rho_d = rho_dev ? rho_out : h->stage + 2 * nnz;
    double* ne_d = h->stage + 3 * nnz;
    FindMuBatchCtx ctx{h, Hd, Sd, kT, n_poles, n_electrons, rho_d, ne_d, st, {}};
    std::vector<double> mu(ns), dn(ns);
    int32_t rounds = 0;
    std::string err;
    rc = mu_search_batched(ns, find_mu_eval_batch, find_mu_dos_batch, &ctx, elo.data(), ehi.data(), kT, n_electrons,
                           n_poles + 1, mu_lo, mu_hi, tol_electrons, max_iter, mu.data(), dn.data(), nullptr, &rounds,
                           err);
    if (rc && rc != NDSI_ERR_TIMEOUT) return err.empty() ? rc : fail(rc, "ndsi_find_mu_batched: " + err);
    // rho_out must hold rho at the returned mu of every system
    if (ctx.last_mu != mu) {
        std::vector<double> dn2(ns);
        const int r2 = find_mu_eval_batch(&ctx, ns, nullptr, mu.data(), dn2.data());
        if (r2) return r2;
    }
    for (int32_t sy = 0; sy < ns; ++sy) {
        mu_out[sy] = mu[sy];
        if (n_elec_out) n_elec_out[sy] = n_electrons[sy] + dn[sy];
    }
    if (rounds_out) *rounds_out = rounds;
    if (!rho_dev) NDSI_CK(cudaMemcpyAsync(rho_out, rho_d, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    NDSI_CK(cudaStreamSynchronize(st));
    if (rc) return fail(rc, "ndsi_find_mu_batched: " + err);
    return NDSI_OK;
}

}  // extern "C"
