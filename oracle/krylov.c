/*
 * krylov.c - columns of (alpha S - gamma H)^{-1} by Krylov iterations, for the sampled-column
 * oracle of the density matrix (Eq. 8) on systems too large for a dense or a sparse-direct route.
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by oracle/krylov.py; the library never links it and shares
 * no code with it.
 *
 * H and S are real symmetric on one CSR pattern (Sec. II.A), so A = alpha S - gamma H is complex
 * symmetric (A^T = A) for complex alpha and real gamma.  Each system A x = e_j is solved by the
 * conjugate orthogonal conjugate gradient method (COCG: conjugate gradients with the bilinear form
 * x^T y in place of the inner product x^H y; van der Vorst and Melissen, IEEE Trans. Magn. 26
 * (1990) 706).  With real alpha and gamma = 0 (A = S, symmetric positive definite) every quantity
 * stays real and COCG is plain conjugate gradients.
 *
 * Per iteration, for every system k:
 *     q = A p;  a = rho / (p^T q);  x += a p;  r -= a q;
 *     rho' = r^T r;  b = rho' / rho;  rho = rho';  p = r + b p.
 * Up to KRY_B systems advance together so that one pass over the matrix serves all of them.  A
 * system whose recursively updated residual norm falls below tol has its true residual e_j - A x
 * recomputed; it is finished if that is below tol as well, and otherwise the iteration restarts
 * from x with the true residual.  Sums over the basis are taken per thread over fixed row ranges
 * and combined in thread order, so a run with a given thread count is reproducible.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KRY_B 16          /* systems advanced together */
#define KRY_MAX_THREADS 256

typedef struct {
    int64_t n;
    const int64_t* rowptr;
    const int32_t* col;
    const double* H;
    const double* S;
} csr_pair;

static int n_threads_used(void) {
#ifdef _OPENMP
    int t = omp_get_max_threads();
    return t < KRY_MAX_THREADS ? t : KRY_MAX_THREADS;
#else
    return 1;
#endif
}

/* Q[:,k] = (alpha_k S - gamma_k H) P[:,k] for all k, and pq_k = sum_i P_ik Q_ik (complex, no
 * conjugation).  Blocks are row-major [n][KRY_B], real and imaginary parts in separate arrays. */
static void block_apply(const csr_pair* m, const double* ar, const double* ai, const double* g,
                        const double* Pr, const double* Pi, double* Qr, double* Qi,
                        double* pq_r, double* pq_i, int nt) {
    static double part[KRY_MAX_THREADS][2][KRY_B];
    #pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double lr[KRY_B], li[KRY_B];
        for (int k = 0; k < KRY_B; ++k) lr[k] = li[k] = 0.0;
        #pragma omp for schedule(static)
        for (int64_t i = 0; i < m->n; ++i) {
            double sr[KRY_B], si[KRY_B], hr[KRY_B], hi[KRY_B];
            for (int k = 0; k < KRY_B; ++k) sr[k] = si[k] = hr[k] = hi[k] = 0.0;
            for (int64_t e = m->rowptr[i]; e < m->rowptr[i + 1]; ++e) {
                const double s = m->S[e], h = m->H[e];
                const double* pr = Pr + (int64_t)m->col[e] * KRY_B;
                const double* pi = Pi + (int64_t)m->col[e] * KRY_B;
                for (int k = 0; k < KRY_B; ++k) {
                    sr[k] += s * pr[k];
                    si[k] += s * pi[k];
                    hr[k] += h * pr[k];
                    hi[k] += h * pi[k];
                }
            }
            double* qr = Qr + i * KRY_B;
            double* qi = Qi + i * KRY_B;
            const double* pr = Pr + i * KRY_B;
            const double* pi = Pi + i * KRY_B;
            for (int k = 0; k < KRY_B; ++k) {
                qr[k] = ar[k] * sr[k] - ai[k] * si[k] - g[k] * hr[k];
                qi[k] = ar[k] * si[k] + ai[k] * sr[k] - g[k] * hi[k];
                lr[k] += pr[k] * qr[k] - pi[k] * qi[k];
                li[k] += pr[k] * qi[k] + pi[k] * qr[k];
            }
        }
        for (int k = 0; k < KRY_B; ++k) {
            part[tid][0][k] = lr[k];
            part[tid][1][k] = li[k];
        }
    }
    for (int k = 0; k < KRY_B; ++k) {
        double a = 0.0, b = 0.0;
        for (int t = 0; t < nt; ++t) {
            a += part[t][0][k];
            b += part[t][1][k];
        }
        pq_r[k] = a;
        pq_i[k] = b;
    }
}

/* True residual of slot k: T = e_j - (alpha S - gamma H) X[:,k]; returns ||T||_2 and, when
 * write_r is set, stores T into R[:,k]. */
static double true_residual(const csr_pair* m, double ar, double ai, double g, int64_t j,
                            const double* Xr, const double* Xi, double* Rr, double* Ri, int k,
                            int write_r, int nt) {
    static double part[KRY_MAX_THREADS];
    #pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double acc = 0.0;
        #pragma omp for schedule(static)
        for (int64_t i = 0; i < m->n; ++i) {
            double sr = 0.0, si = 0.0, hr = 0.0, hi = 0.0;
            for (int64_t e = m->rowptr[i]; e < m->rowptr[i + 1]; ++e) {
                const int64_t c = (int64_t)m->col[e] * KRY_B + k;
                sr += m->S[e] * Xr[c];
                si += m->S[e] * Xi[c];
                hr += m->H[e] * Xr[c];
                hi += m->H[e] * Xi[c];
            }
            double tr = (i == j ? 1.0 : 0.0) - (ar * sr - ai * si - g * hr);
            double ti = -(ar * si + ai * sr - g * hi);
            if (write_r) {
                Rr[i * KRY_B + k] = tr;
                Ri[i * KRY_B + k] = ti;
            }
            acc += tr * tr + ti * ti;
        }
        part[tid] = acc;
    }
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += part[t];
    return sqrt(s);
}

/*
 * Solve (alpha_t S - gamma_t H) x_t = e_{cols[t]} for t = 0..n_tasks-1.
 *   alpha      - interleaved complex double[2*n_tasks];  gamma - double[n_tasks].
 *   cols       - int32[n_tasks], 0 <= cols[t] < n.
 *   tol        - relative residual target ||e_j - A x|| <= tol (||e_j|| = 1).
 *   max_iter   - iteration limit per task (restarts included).
 *   X_out      - interleaved complex double[2*n_tasks*n], task-major.
 *   iters_out  - int64[n_tasks] iterations used;  relres_out - double[n_tasks] final true residual.
 * Returns 0, or the number of tasks that did not reach tol within max_iter (their best x is
 * still written), or -1 for bad arguments / no memory.
 */
int krylov_columns(int64_t n, const int64_t* rowptr, const int32_t* col, const double* H,
                   const double* S, int32_t n_tasks, const double* alpha, const double* gamma,
                   const int32_t* cols, double tol, int64_t max_iter, double* X_out,
                   int64_t* iters_out, double* relres_out) {
    if (n < 1 || n_tasks < 0 || !rowptr || !col || !H || !S || !alpha || !gamma || !cols ||
        !X_out || !iters_out || !relres_out || !(tol > 0.0))
        return -1;
    for (int32_t t = 0; t < n_tasks; ++t)
        if (cols[t] < 0 || cols[t] >= n) return -1;
    const csr_pair m = {n, rowptr, col, H, S};
    const int nt = n_threads_used();
    const size_t blk = (size_t)n * KRY_B;
    double* buf = (double*)calloc(8 * blk, sizeof(double));
    if (!buf) return -1;
    double *Xr = buf, *Xi = buf + blk, *Rr = buf + 2 * blk, *Ri = buf + 3 * blk;
    double *Pr = buf + 4 * blk, *Pi = buf + 5 * blk, *Qr = buf + 6 * blk, *Qi = buf + 7 * blk;

    int32_t task[KRY_B];
    double ar[KRY_B], ai[KRY_B], g[KRY_B], rho_r[KRY_B], rho_i[KRY_B];
    int64_t it[KRY_B];
    int32_t next = 0, failed = 0;

    /* Put task t (or nothing, t = -1) into slot k: x = 0, r = p = e_j, rho = 1. */
    #define LOAD_SLOT(k, t)                                                         \
        do {                                                                        \
            task[k] = (t);                                                          \
            for (int64_t i_ = 0; i_ < n; ++i_) {                                    \
                Xr[i_ * KRY_B + k] = Xi[i_ * KRY_B + k] = 0.0;                      \
                Rr[i_ * KRY_B + k] = Ri[i_ * KRY_B + k] = 0.0;                      \
                Pr[i_ * KRY_B + k] = Pi[i_ * KRY_B + k] = 0.0;                      \
            }                                                                       \
            it[k] = 0;                                                              \
            if ((t) >= 0) {                                                         \
                ar[k] = alpha[2 * (t)];                                             \
                ai[k] = alpha[2 * (t) + 1];                                         \
                g[k] = gamma[t];                                                    \
                Rr[(int64_t)cols[t] * KRY_B + k] = 1.0;                             \
                Pr[(int64_t)cols[t] * KRY_B + k] = 1.0;                             \
                rho_r[k] = 1.0;                                                     \
                rho_i[k] = 0.0;                                                     \
            } else {                                                                \
                ar[k] = 1.0; ai[k] = 0.0; g[k] = 0.0; rho_r[k] = 1.0; rho_i[k] = 0.0; \
            }                                                                       \
        } while (0)

    /* Finish the task in slot k: copy x out with its true residual. */
    #define STORE_SLOT(k, res)                                                      \
        do {                                                                        \
            const int32_t t_ = task[k];                                             \
            double* xo = X_out + 2 * (int64_t)t_ * n;                               \
            for (int64_t i_ = 0; i_ < n; ++i_) {                                    \
                xo[2 * i_] = Xr[i_ * KRY_B + k];                                    \
                xo[2 * i_ + 1] = Xi[i_ * KRY_B + k];                                \
            }                                                                       \
            iters_out[t_] = it[k];                                                  \
            relres_out[t_] = (res);                                                 \
        } while (0)

    for (int k = 0; k < KRY_B; ++k) {
        int32_t t = next < n_tasks ? next++ : -1;
        LOAD_SLOT(k, t);
    }
    double pq_r[KRY_B], pq_i[KRY_B];
    static double part[KRY_MAX_THREADS][3][KRY_B];
    for (;;) {
        int active = 0;
        for (int k = 0; k < KRY_B; ++k) active += task[k] >= 0;
        if (!active) break;
        block_apply(&m, ar, ai, g, Pr, Pi, Qr, Qi, pq_r, pq_i, nt);
        double a_r[KRY_B], a_i[KRY_B];
        for (int k = 0; k < KRY_B; ++k) {
            const double den = pq_r[k] * pq_r[k] + pq_i[k] * pq_i[k];
            if (task[k] < 0 || den == 0.0) {
                a_r[k] = a_i[k] = 0.0;       /* idle slot, or breakdown: restarted below */
                continue;
            }
            a_r[k] = (rho_r[k] * pq_r[k] + rho_i[k] * pq_i[k]) / den;
            a_i[k] = (rho_i[k] * pq_r[k] - rho_r[k] * pq_i[k]) / den;
        }
        /* x += a p; r -= a q; rho' = r^T r; |r|^2 */
        #pragma omp parallel num_threads(nt)
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            double s_r[KRY_B], s_i[KRY_B], s_n[KRY_B];
            for (int k = 0; k < KRY_B; ++k) s_r[k] = s_i[k] = s_n[k] = 0.0;
            #pragma omp for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                for (int k = 0; k < KRY_B; ++k) {
                    const int64_t o = i * KRY_B + k;
                    Xr[o] += a_r[k] * Pr[o] - a_i[k] * Pi[o];
                    Xi[o] += a_r[k] * Pi[o] + a_i[k] * Pr[o];
                    const double rr = Rr[o] - (a_r[k] * Qr[o] - a_i[k] * Qi[o]);
                    const double ri = Ri[o] - (a_r[k] * Qi[o] + a_i[k] * Qr[o]);
                    Rr[o] = rr;
                    Ri[o] = ri;
                    s_r[k] += rr * rr - ri * ri;
                    s_i[k] += 2.0 * rr * ri;
                    s_n[k] += rr * rr + ri * ri;
                }
            }
            for (int k = 0; k < KRY_B; ++k) {
                part[tid][0][k] = s_r[k];
                part[tid][1][k] = s_i[k];
                part[tid][2][k] = s_n[k];
            }
        }
        double b_r[KRY_B], b_i[KRY_B], rn[KRY_B];
        for (int k = 0; k < KRY_B; ++k) {
            double nr = 0.0, ni = 0.0, nn = 0.0;
            for (int t = 0; t < nt; ++t) {
                nr += part[t][0][k];
                ni += part[t][1][k];
                nn += part[t][2][k];
            }
            rn[k] = sqrt(nn);
            const double den = rho_r[k] * rho_r[k] + rho_i[k] * rho_i[k];
            b_r[k] = den > 0.0 ? (nr * rho_r[k] + ni * rho_i[k]) / den : 0.0;
            b_i[k] = den > 0.0 ? (ni * rho_r[k] - nr * rho_i[k]) / den : 0.0;
            rho_r[k] = nr;
            rho_i[k] = ni;
            if (task[k] >= 0) ++it[k];
        }
        /* p = r + b p */
        #pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            for (int k = 0; k < KRY_B; ++k) {
                const int64_t o = i * KRY_B + k;
                const double pr = Pr[o], pi = Pi[o];
                Pr[o] = Rr[o] + b_r[k] * pr - b_i[k] * pi;
                Pi[o] = Ri[o] + b_r[k] * pi + b_i[k] * pr;
            }
        }
        /* convergence, restarts and slot refills */
        for (int k = 0; k < KRY_B; ++k) {
            if (task[k] < 0) continue;
            const int breakdown = (pq_r[k] == 0.0 && pq_i[k] == 0.0) ||
                                  (rho_r[k] == 0.0 && rho_i[k] == 0.0);
            if (!(rn[k] <= tol) && !breakdown && it[k] < max_iter) continue;
            const int64_t j = cols[task[k]];
            const double tr = true_residual(&m, ar[k], ai[k], g[k], j, Xr, Xi, Rr, Ri, k, 1, nt);
            if (tr <= tol || it[k] >= max_iter) {
                if (!(tr <= tol)) ++failed;
                STORE_SLOT(k, tr);
                int32_t t = next < n_tasks ? next++ : -1;
                LOAD_SLOT(k, t);
                continue;
            }
            /* restart from x with its true residual (already in R): p = r, rho = r^T r */
            double nr = 0.0, ni = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                const int64_t o = i * KRY_B + k;
                Pr[o] = Rr[o];
                Pi[o] = Ri[o];
                nr += Rr[o] * Rr[o] - Ri[o] * Ri[o];
                ni += 2.0 * Rr[o] * Ri[o];
            }
            rho_r[k] = nr;
            rho_i[k] = ni;
        }
    }
    #undef LOAD_SLOT
    #undef STORE_SLOT
    free(buf);
    return failed;
}

/* Number of OpenMP threads the solver uses (1 without OpenMP). */
int krylov_threads(void) { return n_threads_used(); }
