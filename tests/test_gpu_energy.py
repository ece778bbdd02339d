"""GPU energy density matrix (Eq. 10) against the oracle's definition route.

ndsi_density_energy shares the poles and the M0 point with ndsi_density and adds three points for
the first moment; rho must be unchanged bit for bit, e must match the oracle within the
tolerance of each precision form.
"""
import numpy as np
import pytest

from synth import lattice_system, config_system
from oracle.dense import (generalized_eig, density_eig, energy_density_eig, find_mu_eig, on_pattern,
                          occupation)
from tests.libtools import lib

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(sysm, mu, kT, M, precision=0, host=False, **opts):
    torch = _torch()
    nd = lib()
    plan = nd.analyze_system(sysm, precision=precision, **opts)
    if host:
        rho, e, ne = np.zeros(sysm.nnz), np.zeros(sysm.nnz), np.zeros(1)
        nd.ndsi_density_energy(plan, sysm.H.copy(), sysm.S.copy(), mu, kT, M, rho, e, ne)
        return rho, e, float(ne[0]), None
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    rho = torch.zeros(sysm.nnz, dtype=torch.float64, device="cuda")
    e = torch.zeros_like(rho)
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density_energy(plan, H, S, mu, kT, M, rho, e, ne)
    rho2 = torch.zeros_like(rho)
    nd.ndsi_density(plan, H, S, mu, kT, M, rho2, ne)
    torch.cuda.synchronize()
    return rho.cpu().numpy(), e.cpu().numpy(), float(ne.cpu()[0]), rho2.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-9)])
@pytest.mark.parametrize("shape,o,nb,M", [((40, 1, 1), 3, "1d", 40), ((9, 8, 1), 2, "2d", 40),
                                         ((5, 5, 4), 2, "3d", 60)])
def test_energy_density_matches_oracle(precision, tol, shape, o, nb, M):
    sysm = lattice_system(shape, o, nb, 61)
    Hd, Sd = sysm.dense()
    kT = 0.01
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    e_ref = on_pattern(energy_density_eig(eps, C, mu, kT, M), sysm)
    rho_ref = on_pattern(density_eig(eps, C, mu, kT, M), sysm)
    rho, e, ne, rho_plain = _run(sysm, mu, kT, M, precision)
    print(f"e err {np.max(np.abs(e - e_ref)):.2e} (precision {precision}, {shape})")
    assert np.max(np.abs(e - e_ref)) < tol
    assert np.max(np.abs(rho - rho_ref)) < tol
    assert np.array_equal(rho, rho_plain)             # the extra points carry zero rho weight
    # band energy: Tr(e S) = sum_nu eps_nu 2 f_nu
    band = float(np.sum(eps * occupation(eps, mu, kT, M)))
    assert abs(float(np.dot(e, sysm.S)) - band) < 1e2 * tol


def test_energy_density_host_buffers_and_replay():
    sysm = lattice_system((7, 6, 1), 2, "2d", 62)
    r_d, e_d, n_d, _ = _run(sysm, -0.1, 0.02, 30)
    r_h, e_h, n_h, _ = _run(sysm, -0.1, 0.02, 30, host=True)
    assert np.array_equal(e_d, e_h) and np.array_equal(r_d, r_h) and n_d == n_h


def test_energy_density_C1():
    sysm = config_system("C1")
    kT, M = sysm.meta["kT"], sysm.meta["poles"]
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    e_ref = on_pattern(energy_density_eig(eps, C, mu, kT, M), sysm)
    rho, e, ne, _ = _run(sysm, mu, kT, M)
    assert np.max(np.abs(e - e_ref)) < 1e-10


def test_energy_density_periodic_lattice():
    # a periodic cell (separators wrapping around it) changes nothing in Eq. 10's evaluation
    sysm = lattice_system((9, 8, 1), 2, "2d", 62, periodic=(True, True, False))
    Hd, Sd = sysm.dense()
    kT, M = 0.01, 40
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    e_ref = on_pattern(energy_density_eig(eps, C, mu, kT, M), sysm)
    rho, e, ne, rho_plain = _run(sysm, mu, kT, M, 0, cell=sysm.meta["cell"])
    assert np.max(np.abs(e - e_ref)) < 1e-10
    assert np.array_equal(rho, rho_plain)
