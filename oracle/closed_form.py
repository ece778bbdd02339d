"""Closed-form spectrum of the open s-valent nearest-neighbour chain (a pin for the oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

H = a I + b T and S = I + s T with T the adjacency matrix of an open chain of N sites share
the eigenvectors v_k(j) = sin(j theta_k), theta_k = k pi/(N+1), k = 1..N, with T v = 2 cos(theta)
v.  Hence eps_k = (a + 2 b cos theta_k)/(1 + 2 s cos theta_k) (|2s| < 1), and
v_k^T S v_k = (N+1)/2 (1 + 2 s cos theta_k) normalises c_k for Eq. (2).
"""
from __future__ import annotations

import numpy as np


def chain_spectrum(N, a, b, s):
    """(eps, C): eigenvalues (ascending) and S-orthonormal eigenvectors as columns."""
    k = np.arange(1, N + 1)
    th = k * np.pi / (N + 1)
    ct = np.cos(th)
    eps = (a + 2.0 * b * ct) / (1.0 + 2.0 * s * ct)
    j = np.arange(1, N + 1)
    V = np.sin(np.outer(j, th))
    norm = np.sqrt(0.5 * (N + 1) * (1.0 + 2.0 * s * ct))
    C = V / norm[None, :]
    order = np.argsort(eps)
    return eps[order], C[:, order]


def chain_density(N, a, b, s, mu, kT, occupation):
    """rho = sum_k occ(eps_k) c_k c_k^T with a caller-given occupation function."""
    eps, C = chain_spectrum(N, a, b, s)
    occ = occupation(eps, mu, kT)
    return (C * occ[None, :]) @ C.T, eps


def chain_energy_density(N, a, b, s, mu, kT, occupation):
    """e = sum_k eps_k occ(eps_k) c_k c_k^T (the energy density matrix of the chain)."""
    eps, C = chain_spectrum(N, a, b, s)
    w = eps * occupation(eps, mu, kT)
    return (C * w[None, :]) @ C.T, eps
