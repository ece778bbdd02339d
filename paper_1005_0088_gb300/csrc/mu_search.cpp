// Chemical-potential search (Sec. II.C.3) over caller-supplied evaluations of DeltaN(mu) and,
// optionally, of the density of states from the retarded Green function.  Host code only: the
// GPU entry point ndsi_find_mu drives it with contour sweeps, the tests with the oracle.
//
// DeltaN(mu) = Tr(rho(mu) S) - N (Eq. 40) is increasing in mu.  The search keeps every exact
// evaluation and
//   * starts, without a caller bracket, from the mu where the density-of-states model holds N
//     (procedure (2), Eqs. 41-43: D(E) on a grid over the spectral bounds, one sweep), or from
//     the middle of the bounds when no model is supplied;
//   * while every evaluation has one sign, steps from the best point by the model anchored at it
//     (mu with DeltaN_i + integral D [f(E - mu) - f(E - mu_i)] = 0) or, when that stalls, by a
//     doubling step towards the root;
//   * once both signs are present, takes the Muller step of procedure (4) (Eqs. 45-46) through
//     the three points of smallest |DeltaN| with both signs, else the linear step of procedure (3)
//     (Eq. 44, read with the denominator DeltaN_i - DeltaN_j) through the two smallest, else the
//     anchored model step, accepting a step anywhere strictly inside the bracket; a step that
//     does not at least halve the smallest |DeltaN| is followed by one bisection.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "ndsi.h"
#include "plan.hpp"

namespace ndsi {

namespace {

double fermi(double x) {
    if (x > 0) {
        const double e = std::exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + std::exp(x));
}

struct DosModel {
    std::vector<double> E, wd;  // grid and trapezoid weight x D(E)
    double kT = 0;
    bool on() const { return !E.empty(); }
    // integral D(E) f((E - mu)/kT) dE over the grid
    double count(double mu) const {
        double s = 0;
        for (size_t k = 0; k < E.size(); ++k) s += wd[k] * fermi((E[k] - mu) / kT);
        return s;
    }
    // the mu in [lo, hi] where target - count(mu) changes sign, by bisection
    double solve(double target, double lo, double hi) const {
        for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo)); ++it) {
            const double m = 0.5 * (lo + hi);
            (count(m) < target ? lo : hi) = m;
        }
        return 0.5 * (lo + hi);
    }
};

using Pt = std::pair<double, double>;  // (mu, DeltaN)

// Eqs. 45-46 through three points with the smallest |DeltaN|, both signs present; NaN if the
// quadratic has no real root.
double muller_step(const std::vector<Pt>& pts) {
    if (pts.size() < 3) return std::nan("");
    std::vector<Pt> q(pts);
    std::stable_sort(q.begin(), q.end(), [](const Pt& x, const Pt& y) { return std::fabs(x.second) < std::fabs(y.second); });
    std::vector<Pt> sel(q.begin(), q.begin() + 3);
    bool pos = false, neg = false;
    for (const Pt& t : sel) (t.second > 0 ? pos : neg) = true;
    if (!(pos && neg)) {
        for (size_t i = 3; i < q.size(); ++i)
            if ((q[i].second > 0 && !pos) || (q[i].second < 0 && !neg)) {
                sel[2] = q[i];
                break;
            }
    }
    std::sort(sel.begin(), sel.end());
    const double m0 = sel[0].first, m1 = sel[1].first, m2 = sel[2].first;
    const double h1 = m1 - m0, h2 = m2 - m1;
    if (!(h1 > 0 && h2 > 0)) return std::nan("");
    const double d1 = (sel[1].second - sel[0].second) / h1;
    const double d2 = (sel[2].second - sel[1].second) / h2;
    // DeltaN ~ a t^2 + b t + c with t = mu - m2
    const double a = (d2 - d1) / (h1 + h2);
    const double b = a * h2 + d2;
    const double c = sel[2].second;
    const double disc = b * b - 4.0 * a * c;
    if (disc < 0) return std::nan("");
    const double sq = std::sqrt(disc);
    double t;
    if (b >= 0) t = -2.0 * c / (b + sq);  // the positive-slope root, cancellation-free form
    else if (a != 0) t = (-b + sq) / (2.0 * a);
    else return std::nan("");
    return m2 + t;
}

// Eq. 44 through the two points with the smallest |DeltaN|.
double linear_step(const std::vector<Pt>& pts) {
    if (pts.size() < 2) return std::nan("");
    std::vector<Pt> q(pts);
    std::stable_sort(q.begin(), q.end(), [](const Pt& x, const Pt& y) { return std::fabs(x.second) < std::fabs(y.second); });
    const double mi = q[0].first, fi = q[0].second, mj = q[1].first, fj = q[1].second;
    if (fi == fj) return std::nan("");
    return (mj * fi - mi * fj) / (fi - fj);
}

}  // namespace

int mu_search(ndsi_mu_eval_fn eval, ndsi_mu_dos_fn dos, void* ctx, double elo, double ehi, double kT, double n_electrons,
              int32_t n_grid, double mu_lo, double mu_hi, double tol, int32_t max_iter, double* mu_out,
              double* dn_out, int32_t* evals_out, std::string& err) {
    if (!eval || !(elo < ehi) || !(kT > 0) || !(tol > 0) || max_iter < 1 || !std::isfinite(n_electrons)) {
        err = "mu search: invalid argument";
        return NDSI_ERR_INVALID;
    }
    std::vector<Pt> pts;
    int32_t evals = 0;
    Pt best(0.0, std::numeric_limits<double>::infinity());
    auto evaluate = [&](double mu) -> int {
        double dn = 0;
        const int rc = eval(ctx, mu, &dn);
        ++evals;
        if (rc) return rc;
        if (!std::isfinite(dn)) {
            err = "mu search: non-finite electron count";
            return NDSI_ERR_SINGULAR;
        }
        pts.emplace_back(mu, dn);
        if (std::fabs(dn) < std::fabs(best.second)) best = Pt(mu, dn);
        return NDSI_OK;
    };
    auto finish = [&](int rc) {
        if (mu_out) *mu_out = best.first;
        if (dn_out) *dn_out = best.second;
        if (evals_out) *evals_out = evals;
        return rc;
    };
    DosModel model;
    model.kT = kT;
    int rc;
    double grow = std::max(4.0 * kT, 1e-3);
    if (mu_lo < mu_hi) {
        const double a = std::min(std::max(mu_lo, elo), ehi), b = std::max(std::min(mu_hi, ehi), elo);
        if ((rc = evaluate(a))) return finish(rc);
        if (std::fabs(best.second) >= tol && b > a)
            if ((rc = evaluate(b))) return finish(rc);
        grow = std::max(grow, b - a);
    } else {
        double mu0 = 0.5 * (elo + ehi);
        if (dos && n_grid >= 2) {
            // procedure (2): the density of states on the grid, one sweep of n_grid points with
            // eta two grid spacings (the trapezoid rule then resolves the broadened D)
            const double dE = (ehi - elo) / (n_grid - 1);
            std::vector<double> D(n_grid);
            model.E.resize(n_grid);
            for (int k = 0; k < n_grid; ++k) model.E[k] = elo + k * dE;
            rc = dos(ctx, model.E.data(), n_grid, 2.0 * dE, D.data());
            ++evals;
            if (rc) return finish(rc);
            model.wd.resize(n_grid);
            for (int k = 0; k < n_grid; ++k) model.wd[k] = (k == 0 || k == n_grid - 1 ? 0.5 : 1.0) * dE * D[k];
            mu0 = model.solve(n_electrons, elo - 10.0 * kT, ehi + 10.0 * kT);
            mu0 = std::min(std::max(mu0, elo), ehi);
        }
        if ((rc = evaluate(mu0))) return finish(rc);
    }
    bool force_bisect = false, last_model = false;
    double last_model_from = std::numeric_limits<double>::infinity();
    while (std::fabs(best.second) >= tol && evals < max_iter) {
        double a = -std::numeric_limits<double>::infinity(), b = std::numeric_limits<double>::infinity();
        for (const Pt& t : pts) {
            if (t.second < 0) a = std::max(a, t.first);
            if (t.second > 0) b = std::min(b, t.first);
        }
        const double fb = best.second, mb = best.first;
        double c = std::nan("");
        if (!(std::isfinite(a) && std::isfinite(b))) {
            // one sign only: the anchored model step while it makes progress, else a doubling step
            const bool up = fb < 0;
            if (model.on() && !(last_model && std::fabs(fb) > 0.5 * std::fabs(last_model_from))) {
                // DeltaN_i + count(mu) - count(mu_i) = 0  <=>  count(mu) = count(mu_i) - DeltaN_i
                c = model.solve(model.count(mb) - fb, elo - 10.0 * kT, ehi + 10.0 * kT);
                if (!(up ? c > mb : c < mb)) c = std::nan("");
            }
            last_model = std::isfinite(c);
            last_model_from = fb;
            if (!std::isfinite(c)) {
                // step from the farthest point evaluated in the direction of the root
                double edge = mb;
                for (const Pt& t : pts) edge = up ? std::max(edge, t.first) : std::min(edge, t.first);
                if ((up && edge >= ehi) || (!up && edge <= elo)) {
                    err = "mu search: no sign change of DeltaN within the spectral bounds";
                    return finish(NDSI_ERR_INVALID);
                }
                c = up ? edge + grow : edge - grow;
                grow *= 2.0;
            }
            c = std::min(std::max(c, elo), ehi);
            if ((rc = evaluate(c))) return finish(rc);
            continue;
        }
        // (a >= b only if DeltaN is not monotone at the rounding level: no further refinement)
        if (!(a < b) || b - a <= 1e-15 * std::max(1.0, std::fabs(a))) break;
        auto inside = [&](double x) { return x > a && x < b; };
        bool interp = false;
        if (!force_bisect) {
            c = muller_step(pts);
            if (!inside(c)) c = linear_step(pts);
            if (!inside(c) && model.on()) c = model.solve(model.count(mb) - fb, a, b);
            interp = inside(c);
        }
        if (!interp) c = 0.5 * (a + b);
        if ((rc = evaluate(c))) return finish(rc);
        force_bisect = interp && std::fabs(pts.back().second) > 0.5 * std::fabs(fb);
    }
    if (std::fabs(best.second) >= tol) {
        err = "mu search: not converged within max_iter evaluations";
        return finish(NDSI_ERR_TIMEOUT);
    }
    return finish(NDSI_OK);
}

// ---- many searches in lockstep ---------------------------------------------------------------
// One worker thread per system runs mu_search; its evaluation and density-of-states requests are
// collected by the calling thread, which answers every pending request of one kind with one
// batched callback (one batched sweep on the GPU) and releases the workers again.  Callbacks
// run only on the calling thread.
namespace {

struct Lockstep {
    enum State { RUNNING, WAIT_EVAL, WAIT_DOS, DONE };
    struct Slot {
        State state = RUNNING;
        double mu = 0, dn = 0, last_mu = 0;
        const double* E = nullptr;
        int32_t nE = 0;
        double eta = 0;
        double* D = nullptr;
        int rc = NDSI_OK;
    };
    std::mutex m;
    std::condition_variable cv_coord, cv_work;
    std::vector<Slot> slots;
    int fail_rc = NDSI_OK;  // first callback error: every later request returns it
};

struct WorkerCtx {
    Lockstep* L;
    int32_t sy;
};

int lockstep_eval(void* c, double mu, double* dn) {
    WorkerCtx& w = *static_cast<WorkerCtx*>(c);
    std::unique_lock<std::mutex> lk(w.L->m);
    Lockstep::Slot& s = w.L->slots[w.sy];
    s.mu = mu;
    s.state = Lockstep::WAIT_EVAL;
    w.L->cv_coord.notify_one();
    w.L->cv_work.wait(lk, [&] { return s.state == Lockstep::RUNNING; });
    *dn = s.dn;
    return s.rc;
}

int lockstep_dos(void* c, const double* E, int32_t n, double eta, double* D) {
    WorkerCtx& w = *static_cast<WorkerCtx*>(c);
    std::unique_lock<std::mutex> lk(w.L->m);
    Lockstep::Slot& s = w.L->slots[w.sy];
    s.E = E;
    s.nE = n;
    s.eta = eta;
    s.D = D;
    s.state = Lockstep::WAIT_DOS;
    w.L->cv_coord.notify_one();
    w.L->cv_work.wait(lk, [&] { return s.state == Lockstep::RUNNING; });
    return s.rc;
}

}  // namespace

int mu_search_batched(int32_t ns, ndsi_mu_eval_batch_fn eval, ndsi_mu_dos_batch_fn dos, void* ctx,
                      const double* elo, const double* ehi, const double* kT, const double* n_electrons,
                      int32_t n_grid, const double* mu_lo, const double* mu_hi, double tol, int32_t max_iter,
                      double* mu_out, double* dn_out, int32_t* evals_out, int32_t* rounds_out, std::string& err) {
    if (ns < 1 || !eval || !elo || !ehi || !kT || !n_electrons || !mu_out) {
        err = "mu search: invalid argument";
        return NDSI_ERR_INVALID;
    }
    Lockstep L;
    L.slots.resize(ns);
    std::vector<WorkerCtx> wc(ns);
    std::vector<int> rcs(ns, NDSI_OK);
    std::vector<std::string> errs(ns);
    std::vector<double> mu(ns, 0.0), dn(ns, 0.0);
    std::vector<int32_t> ev(ns, 0);
    std::vector<std::thread> threads;
    threads.reserve(ns);
    for (int32_t sy = 0; sy < ns; ++sy) {
        wc[sy] = WorkerCtx{&L, sy};
        threads.emplace_back([&, sy]() {
            const double lo = mu_lo ? mu_lo[sy] : 0.0, hi = mu_hi ? mu_hi[sy] : 0.0;
            const int rc = mu_search(lockstep_eval, dos ? lockstep_dos : nullptr, &wc[sy], elo[sy], ehi[sy], kT[sy],
                                     n_electrons[sy], n_grid, lo, hi, tol, max_iter, &mu[sy], &dn[sy], &ev[sy],
                                     errs[sy]);
            std::lock_guard<std::mutex> lk(L.m);
            rcs[sy] = rc;
            L.slots[sy].state = Lockstep::DONE;
            L.cv_coord.notify_one();
        });
    }
    int32_t rounds = 0;
    std::vector<double> bmu(ns), bdn(ns), etas(ns);
    std::vector<int32_t> active(ns);
    {
        std::unique_lock<std::mutex> lk(L.m);
        for (;;) {
            L.cv_coord.wait(lk, [&] {
                for (const auto& s : L.slots)
                    if (s.state == Lockstep::RUNNING) return false;
                return true;
            });
            bool any_dos = false, any_eval = false;
            for (const auto& s : L.slots) {
                any_dos |= s.state == Lockstep::WAIT_DOS;
                any_eval |= s.state == Lockstep::WAIT_EVAL;
            }
            if (!any_dos && !any_eval) break;
            int rc = L.fail_rc;
            if (any_dos) {
                // one batched density-of-states call; every waiting system brings its own grid
                int32_t nE = 0;
                for (const auto& s : L.slots)
                    if (s.state == Lockstep::WAIT_DOS) nE = std::max(nE, s.nE);
                std::vector<double> E(static_cast<size_t>(ns) * nE, 0.0), D(static_cast<size_t>(ns) * nE, 0.0);
                for (int32_t sy = 0; sy < ns; ++sy) {
                    const auto& s = L.slots[sy];
                    active[sy] = s.state == Lockstep::WAIT_DOS;
                    etas[sy] = active[sy] ? s.eta : 1.0;
                    for (int32_t k = 0; k < nE; ++k)
                        E[static_cast<size_t>(sy) * nE + k] =
                            active[sy] ? s.E[std::min(k, s.nE - 1)] : elo[sy] + (ehi[sy] - elo[sy]) * k / std::max(1, nE - 1);
                }
                if (!rc) rc = dos(ctx, ns, active.data(), E.data(), nE, etas.data(), D.data());
                ++rounds;
                for (int32_t sy = 0; sy < ns; ++sy) {
                    auto& s = L.slots[sy];
                    if (s.state != Lockstep::WAIT_DOS) continue;
                    for (int32_t k = 0; k < s.nE; ++k) s.D[k] = D[static_cast<size_t>(sy) * nE + k];
                    s.rc = rc;
                    s.state = Lockstep::RUNNING;
                }
            } else {
                // one batched evaluation; systems without a request are evaluated at their last mu
                for (int32_t sy = 0; sy < ns; ++sy) {
                    const auto& s = L.slots[sy];
                    active[sy] = s.state == Lockstep::WAIT_EVAL;
                    bmu[sy] = active[sy] ? s.mu : s.last_mu;
                }
                if (!rc) rc = eval(ctx, ns, active.data(), bmu.data(), bdn.data());
                ++rounds;
                for (int32_t sy = 0; sy < ns; ++sy) {
                    auto& s = L.slots[sy];
                    if (s.state != Lockstep::WAIT_EVAL) continue;
                    s.dn = bdn[sy];
                    s.last_mu = s.mu;
                    s.rc = rc;
                    s.state = Lockstep::RUNNING;
                }
            }
            if (rc && !L.fail_rc) L.fail_rc = rc;
            L.cv_work.notify_all();
        }
    }
    for (auto& t : threads) t.join();
    int rc = NDSI_OK;
    for (int32_t sy = 0; sy < ns; ++sy) {
        mu_out[sy] = mu[sy];
        if (dn_out) dn_out[sy] = dn[sy];
        if (evals_out) evals_out[sy] = ev[sy];
        if (rcs[sy] && (!rc || rc == NDSI_ERR_TIMEOUT)) {
            rc = rcs[sy];
            err = "system " + std::to_string(sy) + ": " + errs[sy];
        }
    }
    if (L.fail_rc && !rc) rc = L.fail_rc;
    if (rounds_out) *rounds_out = rounds;
    return rc;
}

}  // namespace ndsi

extern "C" int ndsi_mu_search(ndsi_mu_eval_fn eval, ndsi_mu_dos_fn dos, void* ctx, double elo, double ehi, double kT,
                              double n_electrons, int32_t n_grid, double mu_lo, double mu_hi, double tol_electrons,
                              int32_t max_iter, double* mu_out, double* dn_out, int32_t* evals_out) {
    std::string err;
    const int rc = ndsi::mu_search(eval, dos, ctx, elo, ehi, kT, n_electrons, n_grid, mu_lo, mu_hi, tol_electrons,
                                   max_iter, mu_out, dn_out, evals_out, err);
    if (rc) ndsi::set_last_error(err);
    return rc;
}

extern "C" int ndsi_mu_search_batched(int32_t n_systems, ndsi_mu_eval_batch_fn eval, ndsi_mu_dos_batch_fn dos,
                                      void* ctx, const double* elo, const double* ehi, const double* kT,
                                      const double* n_electrons, int32_t n_grid, const double* mu_lo,
                                      const double* mu_hi, double tol_electrons, int32_t max_iter, double* mu_out,
                                      double* dn_out, int32_t* evals_out, int32_t* rounds_out) {
    std::string err;
    const int rc = ndsi::mu_search_batched(n_systems, eval, dos, ctx, elo, ehi, kT, n_electrons, n_grid, mu_lo, mu_hi,
                                           tol_electrons, max_iter, mu_out, dn_out, evals_out, rounds_out, err);
    if (rc) ndsi::set_last_error(err.empty() ? "mu search failed" : err);
    return rc;
}
