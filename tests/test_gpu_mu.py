"""GPU chemical-potential search (Eq. 40) against the oracle's bisection on the eigenvalues."""
import numpy as np
import pytest

from synth import config_system, lattice_system
from oracle.dense import generalized_eig, find_mu_eig, electron_count_eig, on_pattern, density_eig
from tests.libtools import lib

pytestmark = pytest.mark.gpu


def _setup(sysm, **opts):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nd = lib()
    plan = nd.analyze_system(sysm, **opts)
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    rho = torch.zeros(sysm.nnz, dtype=torch.float64, device="cuda")
    return nd, plan, H, S, rho


@pytest.mark.parametrize("precision", [0, 1])
def test_find_mu_C1(precision):
    sysm = config_system("C1")
    kT, M = sysm.meta["kT"], sysm.meta["poles"]
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu_ref = find_mu_eig(eps, kT, sysm.n_electrons, M)
    nd, plan, H, S, rho = _setup(sysm, precision=precision)
    mu, ne, iters = nd.ndsi_find_mu(plan, H, S, kT, M, sysm.n_electrons, rho, tol_electrons=1e-8)
    print(f"find_mu C1 prec={precision}: mu={mu:.12f} ref={mu_ref:.12f} iters={iters}")
    assert abs(ne - sysm.n_electrons) < 1e-8
    # the root in mu is as sharp as N'(mu) allows: compare through the exact electron count
    assert abs(electron_count_eig(eps, mu, kT, M) - sysm.n_electrons) < 1e-7
    assert iters <= 40
    ref = on_pattern(density_eig(eps, C, mu, kT, M), sysm)
    assert np.max(np.abs(rho.cpu().numpy() - ref)) < 1e-9


def test_find_mu_seeded_bracket_saves_evaluations():
    sysm = lattice_system((10, 10, 1), 3, "2d", 808)
    kT, M = 0.01, 40
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    mu_ref = find_mu_eig(eps, kT, sysm.n_electrons, M)
    nd, plan, H, S, rho = _setup(sysm)
    mu0, ne0, it0 = nd.ndsi_find_mu(plan, H, S, kT, M, sysm.n_electrons, rho)
    mu1, ne1, it1 = nd.ndsi_find_mu(plan, H, S, kT, M, sysm.n_electrons, rho,
                                    mu_lo=mu_ref - 0.02, mu_hi=mu_ref + 0.03)
    print(f"find_mu unseeded {it0} evaluations, seeded {it1}")
    assert abs(ne0 - sysm.n_electrons) < 1e-8 and abs(ne1 - sysm.n_electrons) < 1e-8
    assert it1 < it0
    # a wrong seed (bracket entirely above the root) is widened, not trusted
    mu2, ne2, it2 = nd.ndsi_find_mu(plan, H, S, kT, M, sysm.n_electrons, rho,
                                    mu_lo=mu_ref + 0.2, mu_hi=mu_ref + 0.3)
    assert abs(ne2 - sysm.n_electrons) < 1e-8


def test_find_mu_rejects_bad_arguments():
    sysm = lattice_system((4, 4, 1), 2, "2d", 3)
    nd, plan, H, S, rho = _setup(sysm)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_find_mu(plan, H, S, -0.01, 20, sysm.n_electrons, rho)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_find_mu(plan, H, S, 0.01, 20, 3.0 * sysm.n, rho)   # more electrons than states
