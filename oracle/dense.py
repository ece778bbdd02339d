"""Plain dense FP64 references for rho, G and N_e (Eqs. 2, 5, 6, 8, 40).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Route 1 (definition): solve H c = eps S c (Eq. 2) with S-orthonormal c, then
    rho = 2 sum_nu f(beta (eps_nu - mu)) c_nu c_nu^T                      (Eq. 5, spin factor 2)
with f either the exact Fermi function or the M-pole truncation of Eq. (7).
Route 2 (Eq. 8, dense): rho = M0 + sum_p w_p Re G(alpha_p), G(Z) = (Z S - H)^{-1} (Eq. 6),
alpha_p = mu + i z_p/beta, w_p = -4 R_p/beta, M0 = S^{-1} (the zeroth moment; the paper
evaluates it as i R G(iR) with large R, whose real part tends to S^{-1}).
N_e = Tr(rho S) (Eq. 40) = sum over the pattern of rho_ij S_ij.
Energy density matrix (Eq. 10): e = 2 sum_nu eps_nu f c_nu c_nu^T by definition, or from G with
the zeroth and first moments M0 = S^{-1}, M1 = S^{-1} H S^{-1}.
Density of states from the retarded Green function (Eq. 41): D(E) = -(2/pi) Im Tr(G(E + i eta) S),
by dense inverses, or as the sum of Lorentzians (2/pi) eta / ((E - eps_nu)^2 + eta^2) over the
generalised eigenvalues (Tr(G(z) S) = sum_nu 1/(z - eps_nu) since c^T S c = I).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from .poles import cf_poles, fermi_from_poles, fermi_exact


def generalized_eig(Hd, Sd):
    """Eigenpairs of H c = eps S c with c^T S c = I (LAPACK sygvd via scipy)."""
    return scipy.linalg.eigh(Hd, Sd)


def occupation(eps, mu, kT, M=None):
    """2 f(beta(eps - mu)); f = M-pole truncated Fermi function, or exact if M is None."""
    x = (np.asarray(eps) - mu) / kT
    if M is None:
        return 2.0 * fermi_exact(x)
    z, R = cf_poles(M)
    return 2.0 * fermi_from_poles(x, z, R)


def density_eig(eps, C, mu, kT, M=None):
    """Dense rho = C diag(2 f) C^T (route 1)."""
    occ = occupation(eps, mu, kT, M)
    return (C * occ[None, :]) @ C.T


def electron_count_eig(eps, mu, kT, M=None):
    """Tr(rho S) = sum_nu 2 f(beta(eps_nu - mu)) because c^T S c = 1."""
    return float(np.sum(occupation(eps, mu, kT, M)))


def green_dense(Hd, Sd, Z):
    """G(Z) = (Z S - H)^{-1} by dense LU (Eq. 6)."""
    return np.linalg.inv(Z * Sd - Hd)


def density_inv(Hd, Sd, mu, kT, M):
    """Dense rho by Eq. (8): S^{-1} + sum_p w_p Re (alpha_p S - H)^{-1} (route 2, tiny inputs)."""
    beta = 1.0 / kT
    z, R = cf_poles(M)
    rho = np.linalg.inv(Sd)
    for zp, Rp in zip(z, R):
        alpha = mu + 1j * zp / beta
        rho = rho + (-4.0 * Rp / beta) * np.real(green_dense(Hd, Sd, alpha))
    return rho


def density_inv_terms(Hd, Sd, mu, kT, M):
    """The M + 1 terms of Eq. (8) one by one (tiny inputs): [S^{-1}, w_1 Re G(alpha_1), ...,
    w_M Re G(alpha_M)]; their sum is `density_inv`.  Poles are independent (Sec. III.D), so any
    partition of these terms among processes sums to the same rho."""
    beta = 1.0 / kT
    z, R = cf_poles(M)
    terms = [np.linalg.inv(Sd)]
    for zp, Rp in zip(z, R):
        terms.append((-4.0 * Rp / beta) * np.real(green_dense(Hd, Sd, mu + 1j * zp / beta)))
    return terms


def energy_density_eig(eps, C, mu, kT, M=None):
    """Energy density matrix by definition: e = sum_nu eps_nu 2 f(beta(eps_nu - mu)) c c^T."""
    w = np.asarray(eps) * occupation(eps, mu, kT, M)
    return (C * w[None, :]) @ C.T


def energy_density_inv(Hd, Sd, mu, kT, M):
    """Energy density matrix by Eq. (10) with exact moments (tiny inputs):
    e = M1 + kappa M0 - (4/beta) sum_p R_p Re(alpha_p G(alpha_p)), kappa = (4/beta) sum_p R_p,
    M0 = S^{-1} and M1 = S^{-1} H S^{-1} (the zeroth and first moments of G)."""
    beta = 1.0 / kT
    z, R = cf_poles(M)
    Si = np.linalg.inv(Sd)
    e = Si @ Hd @ Si + (4.0 / beta) * float(np.sum(R)) * Si
    for zp, Rp in zip(z, R):
        alpha = mu + 1j * zp / beta
        e = e - (4.0 / beta) * Rp * np.real(alpha * green_dense(Hd, Sd, alpha))
    return e


def on_pattern(A, system):
    """Values of a dense matrix on the CSR pattern of the system (original order)."""
    return A[system.rows(), system.col]


def electron_count_pattern(rho_pat, system):
    """Tr(rho S) from pattern values: sum_ij rho_ij S_ij (S vanishes off the pattern)."""
    return float(np.dot(rho_pat, system.S))


def find_mu_eig(eps, kT, n_electrons, M=None, tol=1e-13, max_iter=200):
    """Bisection for mu with sum_nu 2 f_M(beta(eps_nu - mu)) = N_e (Eq. 40 on route 1)."""
    lo = float(np.min(eps)) - 50.0 * kT - 1.0
    hi = float(np.max(eps)) + 50.0 * kT + 1.0
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if electron_count_eig(eps, mid, kT, M) < n_electrons:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def sparse_matrices(system):
    """H and S as scipy CSR matrices."""
    H = scipy.sparse.csr_matrix((system.H, system.col, system.rowptr), shape=(system.n, system.n))
    S = scipy.sparse.csr_matrix((system.S, system.col, system.rowptr), shape=(system.n, system.n))
    return H, S


def green_columns(system, Z, cols):
    """Columns G(Z)[:, cols] by a sparse direct solve of (Z S - H) x = e_j (SuperLU)."""
    H, S = sparse_matrices(system)
    X = (Z * S - H).tocsc().astype(np.complex128)
    lu = scipy.sparse.linalg.splu(X)
    rhs = np.zeros((system.n, len(cols)), dtype=np.complex128)
    rhs[np.asarray(cols), np.arange(len(cols))] = 1.0
    return lu.solve(rhs)


def density_columns(system, mu, kT, M, cols):
    """Columns rho[:, cols] by Eq. (8) with sparse solves per pole (sampled-column route)."""
    beta = 1.0 / kT
    z, R = cf_poles(M)
    H, S = sparse_matrices(system)
    lu = scipy.sparse.linalg.splu(S.tocsc())
    rhs = np.zeros((system.n, len(cols)))
    rhs[np.asarray(cols), np.arange(len(cols))] = 1.0
    rho = lu.solve(rhs)
    for zp, Rp in zip(z, R):
        g = green_columns(system, mu + 1j * zp / beta, cols)
        rho = rho + (-4.0 * Rp / beta) * np.real(g)
    return rho


def energy_density_columns(system, mu, kT, M, cols):
    """Columns e[:, cols] by Eq. (10) with sparse solves per pole; M1 e_j = S^{-1} H S^{-1} e_j."""
    beta = 1.0 / kT
    z, R = cf_poles(M)
    H, S = sparse_matrices(system)
    lu = scipy.sparse.linalg.splu(S.tocsc())
    rhs = np.zeros((system.n, len(cols)))
    rhs[np.asarray(cols), np.arange(len(cols))] = 1.0
    m0 = lu.solve(rhs)
    e = lu.solve(H @ m0) + (4.0 / beta) * float(np.sum(R)) * m0
    for zp, Rp in zip(z, R):
        alpha = mu + 1j * zp / beta
        e = e - (4.0 / beta) * Rp * np.real(alpha * green_columns(system, alpha, cols))
    return e


def dos_eig(eps, E, eta):
    """Spin-summed Lorentzian-broadened density of states at energies E (route 1)."""
    E = np.atleast_1d(np.asarray(E, dtype=np.float64))
    d = E[:, None] - np.asarray(eps)[None, :]
    return (2.0 / np.pi) * np.sum(eta / (d * d + eta * eta), axis=1)


def dos_inv(Hd, Sd, E, eta):
    """Eq. (41) as written: -(2/pi) Im Tr(G(E + i eta) S) with G by dense LU (route 2)."""
    E = np.atleast_1d(np.asarray(E, dtype=np.float64))
    out = np.empty(E.size)
    for k, e in enumerate(E):
        G = green_dense(Hd, Sd, e + 1j * eta)
        out[k] = -(2.0 / np.pi) * np.imag(np.trace(G @ Sd))
    return out
