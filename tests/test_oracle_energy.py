"""Pins for the oracle's energy density matrix (Eq. 10).

e = 2 sum_nu eps_nu f(beta(eps_nu - mu)) c_nu c_nu^T.  Three independent routes: the definition
on LAPACK eigenpairs, the open-chain closed form, and Eq. (10) with dense inverses and exact
moments M0 = S^{-1}, M1 = S^{-1} H S^{-1}; plus the band-energy trace identity and sampled columns.
"""
import numpy as np
import pytest

from synth import chain_nntb, lattice_system
from oracle.closed_form import chain_energy_density
from oracle.dense import (generalized_eig, occupation, energy_density_eig, energy_density_inv,
                          energy_density_columns, density_eig)


@pytest.mark.parametrize("M", [None, 40])
def test_energy_density_matches_chain_closed_form(M):
    N, a, b, s = 36, 0.1, -0.8, 0.15
    sysm = chain_nntb(N, a, b, s)
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu, kT = 0.05, 0.02
    e = energy_density_eig(eps, C, mu, kT, M)
    e_cf, _ = chain_energy_density(N, a, b, s, mu, kT, lambda x, m, t: occupation(x, m, t, M))
    assert np.max(np.abs(e - e_cf)) < 1e-12


def test_energy_density_routes_agree():
    # the definition and Eq. (10) (poles with weights -4 R_p alpha_p / beta, kappa M0, M1) are
    # different computations of the same matrix for the same M-pole Fermi function
    sysm = lattice_system((4, 3, 1), 2, "2d", 17)
    Hd, Sd = sysm.dense()
    mu, kT, M = -0.05, 0.03, 40
    eps, C = generalized_eig(Hd, Sd)
    e1 = energy_density_eig(eps, C, mu, kT, M)
    e2 = energy_density_inv(Hd, Sd, mu, kT, M)
    assert np.max(np.abs(e1 - e2)) < 1e-11
    assert np.max(np.abs(e2 - e2.T)) < 1e-12


def test_band_energy_trace():
    # Tr(e S) = sum_nu eps_nu 2 f_nu (the band energy), and Tr(e S) = Tr(rho H)
    sysm = lattice_system((5, 2, 1), 2, "2d", 18)
    Hd, Sd = sysm.dense()
    mu, kT, M = 0.1, 0.02, 40
    eps, C = generalized_eig(Hd, Sd)
    e = energy_density_eig(eps, C, mu, kT, M)
    band = float(np.sum(eps * occupation(eps, mu, kT, M)))
    assert abs(np.trace(e @ Sd) - band) < 1e-11
    rho = density_eig(eps, C, mu, kT, M)
    assert abs(np.trace(rho @ Hd) - band) < 1e-11


def test_planted_mistake_in_moments_is_caught():
    # dropping the first moment or the kappa M0 term breaks agreement with the definition
    sysm = lattice_system((4, 3, 1), 2, "2d", 19)
    Hd, Sd = sysm.dense()
    mu, kT, M = 0.0, 0.03, 40
    eps, C = generalized_eig(Hd, Sd)
    e1 = energy_density_eig(eps, C, mu, kT, M)
    e2 = energy_density_inv(Hd, Sd, mu, kT, M)
    Si = np.linalg.inv(Sd)
    assert np.max(np.abs((e2 - Si @ Hd @ Si) - e1)) > 1e-3
    from oracle.poles import cf_poles
    kappa = 4.0 * kT * float(np.sum(cf_poles(M)[1]))
    assert np.max(np.abs((e2 - kappa * Si) - e1)) > 1e-3


def test_energy_density_sampled_columns():
    sysm = lattice_system((5, 4, 1), 2, "2d", 20)
    Hd, Sd = sysm.dense()
    mu, kT, M = -0.1, 0.02, 30
    cols = [0, 7, 33]
    ec = energy_density_columns(sysm, mu, kT, M, cols)
    e = energy_density_inv(Hd, Sd, mu, kT, M)
    assert np.max(np.abs(ec - e[:, cols])) < 1e-11
