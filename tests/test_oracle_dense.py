"""Pins for the dense rho / G / N_e oracle (Eqs. 2, 5, 6, 8, 40)."""
import numpy as np
import pytest

from synth import chain_nntb, lattice_system
from oracle.closed_form import chain_spectrum, chain_density
from oracle.dense import (generalized_eig, density_eig, density_inv, occupation,
                          electron_count_eig, find_mu_eig, on_pattern, electron_count_pattern,
                          green_dense, green_columns, density_columns)


def _occ_exact(eps, mu, kT):
    return occupation(eps, mu, kT, None)


@pytest.mark.parametrize("M", [None, 40])
def test_eig_route_matches_chain_closed_form(M):
    N, a, b, s = 40, 0.1, -0.8, 0.15
    sysm = chain_nntb(N, a, b, s)
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    eps_cf, C_cf = chain_spectrum(N, a, b, s)
    assert np.max(np.abs(eps - eps_cf)) < 1e-13
    mu, kT = 0.05, 0.02
    rho = density_eig(eps, C, mu, kT, M)
    rho_cf, _ = chain_density(N, a, b, s, mu, kT, lambda e, m, t: occupation(e, m, t, M))
    assert np.max(np.abs(rho - rho_cf)) < 1e-12


def test_spin_factor_full_band():
    # Eq. (5) carries the spin factor 2: with mu far above the spectrum every state holds
    # two electrons, so Tr(rho S) = 2N (closed form count, independent of LAPACK).
    N = 30
    eps, C = chain_spectrum(N, 0.0, -0.5, 0.1)
    assert abs(electron_count_eig(eps, 5.0, 0.05, None) - 2 * N) < 1e-12
    sysm = chain_nntb(N, 0.0, -0.5, 0.1)
    Hd, Sd = sysm.dense()
    rho = density_eig(*generalized_eig(Hd, Sd), 5.0, 0.05, None)
    assert abs(np.trace(rho @ Sd) - 2 * N) < 1e-10
    assert np.max(np.abs(rho - 2 * np.linalg.inv(Sd))) < 1e-10   # full band: rho = 2 S^{-1}


def _small_system(seed=7, shape=(4, 3, 1), o=2, nb="2d"):
    return lattice_system(shape, o, nb, seed)


def test_two_routes_agree():
    # Route 1 (eigenvectors + the same truncated f_M) and route 2 (Eq. 8 by dense inverses)
    # are independent computations of rho; they agree to rounding.
    sysm = _small_system()
    Hd, Sd = sysm.dense()
    mu, kT, M = -0.1, 0.03, 40
    eps, C = generalized_eig(Hd, Sd)
    r1 = density_eig(eps, C, mu, kT, M)
    r2 = density_inv(Hd, Sd, mu, kT, M)
    assert np.max(np.abs(r1 - r2)) < 1e-11
    assert np.max(np.abs(r2 - r2.T)) < 1e-13          # rho is real symmetric


def test_planted_mistakes_are_caught():
    # Dropping the zeroth moment or flipping the residue sign breaks route agreement.
    sysm = _small_system()
    Hd, Sd = sysm.dense()
    mu, kT, M = -0.1, 0.03, 20
    eps, C = generalized_eig(Hd, Sd)
    r1 = density_eig(eps, C, mu, kT, M)
    r2 = density_inv(Hd, Sd, mu, kT, M)
    assert np.max(np.abs(r1 - (r2 - np.linalg.inv(Sd)))) > 1e-2
    assert np.max(np.abs(r1 - (2 * np.linalg.inv(Sd) - r2))) > 1e-2


def test_trace_and_mu_bisection():
    sysm = _small_system(seed=11, shape=(5, 4, 1), o=2)
    Hd, Sd = sysm.dense()
    kT, M = 0.02, 40
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    rho = density_eig(eps, C, mu, kT, M)
    # Eq. (40): Tr(rho S) over the pattern equals the electron count at the converged mu
    ne = electron_count_pattern(on_pattern(rho, sysm), sysm)
    assert abs(ne - sysm.n_electrons) < 1e-9
    assert abs(np.trace(rho @ Sd) - ne) < 1e-10


def test_pole_convergence():
    # Sec. II.B: rho_M converges to the exact-Fermi rho as M grows.
    sysm = _small_system(seed=3)
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu, kT = 0.0, 0.01
    exact = density_eig(eps, C, mu, kT, None)
    errs = [np.max(np.abs(density_eig(eps, C, mu, kT, M) - exact)) for M in (5, 10, 20, 40)]
    assert errs[0] > errs[1] > errs[2] >= 0
    assert errs[-1] < 1e-13


def test_sampled_columns_match_dense():
    sysm = _small_system(seed=5)
    Hd, Sd = sysm.dense()
    mu, kT, M = 0.05, 0.03, 20
    cols = [0, 3, sysm.n - 1]
    r_cols = density_columns(sysm, mu, kT, M, cols)
    r2 = density_inv(Hd, Sd, mu, kT, M)
    assert np.max(np.abs(r_cols - r2[:, cols])) < 1e-12
    Z = 0.3 + 0.2j
    g = green_columns(sysm, Z, cols)
    assert np.max(np.abs(g - green_dense(Hd, Sd, Z)[:, cols])) < 1e-12


@pytest.mark.parametrize("M", [8, 40, 160])
def test_particle_hole_symmetry_at_half_filling(M):
    # A bipartite lattice (nearest-neighbour square lattice, zero on-site energy, S = I) has a
    # spectrum symmetric about 0, and the pole-truncated Fermi function of Eq. 7 keeps
    # f_M(x) + f_M(-x) = 1 (the continued fraction of tanh is odd).  So at mu = 0 and any M:
    # rho = I - tanh_M(H / 2kT) with tanh_M odd in H, i.e. every diagonal element is exactly 1
    # (spin factor 2 x 1/2) and rho vanishes between distinct sites of the same sublattice (odd
    # powers of H connect opposite sublattices only).  Both routes: eigendecomposition (Eq. 5)
    # and the contour sum of dense inverses with the M0 term (Eq. 8).
    nx, ny = 6, 5
    n = nx * ny
    H = np.zeros((n, n))
    for y in range(ny):
        for x in range(nx):
            i = x + nx * y
            if x + 1 < nx:
                H[i, i + 1] = H[i + 1, i] = -1.0
            if y + 1 < ny:
                H[i, i + nx] = H[i + nx, i] = -0.7
    S = np.eye(n)
    kT = 0.05
    eps, C = generalized_eig(H, S)
    parity = np.array([(i % nx + i // nx) % 2 for i in range(n)])
    same = (parity[:, None] == parity[None, :]) & ~np.eye(n, dtype=bool)
    for rho in (density_eig(eps, C, 0.0, kT, M), density_inv(H, S, 0.0, kT, M)):
        assert np.max(np.abs(np.diag(rho) - 1.0)) < 1e-12
        assert np.max(np.abs(rho[same])) < 1e-12
        assert abs(np.trace(rho @ S) - n) < 1e-10                 # half filling: N_e = N
    # away from mu = 0 the symmetry maps mu -> -mu: rho(mu) + P rho(-mu) P = 2 I with
    # P = diag(+-1) on the sublattices (P H P = -H)
    P = np.diag(np.where(parity == 0, 1.0, -1.0))
    r1 = density_inv(H, S, 0.13, kT, M)
    r2 = density_inv(H, S, -0.13, kT, M)
    assert np.max(np.abs(r1 + P @ r2 @ P - 2.0 * np.eye(n))) < 1e-11
