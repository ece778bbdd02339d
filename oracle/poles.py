"""Poles z_p and residues R_p of the continued-fraction Fermi expansion (Eq. 7, Sec. II.B).

TEST INFRASTRUCTURE ONLY: this package is the slow, plain CPU reference that the CUDA path
is checked against.  Only tests, the package smoke check and the bench's CPU-baseline leg may
import it.

Eq. (7) writes 1/(1+e^x) = 1/2 - (x/4) / (1 + (x/2)^2/(3 + (x/2)^2/(5 + ...))), i.e.
1/2 - (x/4) T(x/2) with T(w) = tanh(w)/w = 1/(1 + w^2/(3 + w^2/(5 + ...))).  The paper
defers the pole construction to its Ref. [CF] ("an eigenvalue problem").  Our reading,
derived here from the fraction itself:

  T(w) = 1/(d_1 + w^2/(d_2 + ...)), d_k = 2k-1.  An equivalence transform gives
  T = 1/(1 + e_1 w^2/(1 + e_2 w^2/(1 + ...))) with e_k = 1/(d_k d_{k+1}).  With
  u = i w and lambda = 1/u, h = u T obeys h = 1/(lambda - e_1/(lambda - e_2/(lambda - ...))),
  the (1,1) resolvent element of the symmetric tridiagonal matrix A with zero diagonal and
  off-diagonal sqrt(e_k) = 1/sqrt((2k-1)(2k+1)).  With eigenpairs (lambda_j, v_j) of the
  K x K truncation, h = sum_j v_{1j}^2/(lambda - lambda_j).  Eigenvalues come in +/- pairs;
  substituting w = x/2 and pairing +lambda_j with -lambda_j yields
      1/(1+e^x) ~= 1/2 + sum_p [R_p/(x - i z_p) + R_p/(x + i z_p)],
      z_p = 2/lambda_p,  R_p = -v_{1p}^2 / lambda_p^2   (lambda_p > 0).
  Truncating the fraction after the denominator 4M-1 (K = 2M) gives exactly M pole pairs.

Pinned by: the backward-recurrence evaluation of the printed fraction (cf_fermi_truncated),
the Matsubara limit (z_1 -> pi, R_1 -> -1) and the exact Fermi function.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def cf_poles(M: int):
    """M pole pairs of the continued fraction truncated at depth 2M.

    Returns (z, R): float64 arrays of length M, z ascending (z_1 ~ pi), R < 0.
    """
    M = int(M)
    if M < 1:
        raise ValueError("M >= 1")
    K = 2 * M
    k = np.arange(1, K, dtype=np.float64)
    off = 1.0 / np.sqrt((2.0 * k - 1.0) * (2.0 * k + 1.0))
    lam, V = scipy.linalg.eigh_tridiagonal(np.zeros(K), off)
    pos = lam > 0
    lam_p = lam[pos]
    v1 = V[0, pos]
    z = 2.0 / lam_p
    R = -(v1 ** 2) / lam_p ** 2
    order = np.argsort(z)
    return z[order], R[order]


def fermi_from_poles(x, z, R):
    """1/2 + sum_p 2 R_p x / (x^2 + z_p^2): the pole form of Eq. (7) (second line)."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 + np.sum(2.0 * R[None, :] * x[..., None] / (x[..., None] ** 2 + z[None, :] ** 2),
                        axis=-1)


def cf_fermi_truncated(x, depth: int):
    """Backward evaluation of the printed fraction of Eq. (7), denominators 1, 3, ..., 2*depth-1.

    1/2 - (x/4) / (1 + y/(3 + y/(5 + ... + y/(2*depth-1)))), y = (x/2)^2.
    """
    x = np.asarray(x, dtype=np.float64)
    y = (0.5 * x) ** 2
    t = np.full_like(x, 2.0 * depth - 1.0)
    for k in range(depth - 1, 0, -1):
        t = (2.0 * k - 1.0) + y / t
    return 0.5 - 0.25 * x / t


def fermi_exact(x):
    """1/(1+e^x), evaluated without overflow."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x >= 0
    e = np.exp(-x[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def pole_weights(mu: float, kT: float, M: int):
    """Complex shifts alpha_p = mu + i z_p / beta and real weights w_p = -4 R_p / beta (Eq. 8).

    rho = M0 + sum_p w_p Re G(alpha_p), since Im(-4i/beta R_p G) = -4 R_p/beta Re G for
    real R_p (Eq. 8 with Im(-i g) = -Re g).
    """
    beta = 1.0 / kT
    z, R = cf_poles(M)
    alpha = mu + 1j * z / beta
    w = -4.0 * R / beta
    return alpha, w
