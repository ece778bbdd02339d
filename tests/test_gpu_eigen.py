"""Selected eigenstates near an energy (App. B) against the oracle's definition."""
import numpy as np
import pytest

from synth import lattice_system, chain_nntb
from oracle.closed_form import chain_spectrum
from oracle.eigen import eigenstates_near
from tests.libtools import lib

pytestmark = pytest.mark.gpu


def _setup(sysm, **opts):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nd = lib()
    plan = nd.analyze_system(sysm, **opts)
    return nd, plan, torch.as_tensor(sysm.H, device="cuda"), torch.as_tensor(sysm.S, device="cuda")


def _check(eps, C, res, eps_ref, C_ref, Sd, tol_e, tol_p):
    assert np.max(np.abs(eps - eps_ref)) < tol_e
    # same invariant subspace (S-projectors), S-orthonormal columns
    Pg = C.T @ C @ Sd
    Pr = C_ref @ C_ref.T @ Sd
    assert np.max(np.abs(Pg - Pr)) < tol_p
    assert np.max(np.abs(C @ Sd @ C.T - np.eye(len(eps)))) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_eigenstates_match_definition(precision):
    sysm = lattice_system((9, 8, 1), 4, "2d", seed=81)
    Hd, Sd = sysm.dense()
    xi, n = -0.2, 5
    eps_ref, C_ref = eigenstates_near(Hd, Sd, xi, n)
    nd, plan, H, S = _setup(sysm, precision=precision)
    eps, C, res, it = nd.ndsi_eigenstates(plan, H, S, xi, n, eta=1e-3, block=9, tol=1e-10)
    print(f"eigenstates prec={precision}: {it} iterations, residuals {res.max():.2e}")
    assert np.all(res < 1e-10)
    _check(eps, C, res, eps_ref, C_ref, Sd, 1e-11, 1e-8)
    # the convention of the output: largest-magnitude component positive
    for j in range(n):
        assert C[j, np.argmax(np.abs(C[j]))] > 0


def test_eigenstates_chain_closed_form_and_device_output():
    import torch
    N, a, b, s = 300, 0.1, -0.8, 0.15
    sysm = chain_nntb(N, a, b, s)
    eps_cf, C_cf = chain_spectrum(N, a, b, s)
    xi, n = 0.37, 3
    pick = np.sort(np.argsort(np.abs(eps_cf - xi))[:n])
    nd, plan, H, S = _setup(sysm)
    Cd = torch.zeros((n, sysm.n), dtype=torch.float64, device="cuda")
    eps, C, res, it = nd.ndsi_eigenstates(plan, H, S, xi, n, block=6, C_out=Cd)
    Sd = sysm.dense()[1]
    _check(eps, Cd.cpu().numpy(), res, eps_cf[pick], C_cf[:, pick], Sd, 1e-11, 1e-8)


def test_eigenstates_errors():
    sysm = lattice_system((4, 4, 1), 2, "2d", seed=82)
    nd, plan, H, S = _setup(sysm)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_eigenstates(plan, H, S, 0.0, 4, block=2)          # block < n_states
    with pytest.raises(nd.NdsiError):
        nd.ndsi_eigenstates(plan, H, S, 0.0, 2, eta=0.0)
    with pytest.raises(nd.NdsiError) as e:
        nd.ndsi_eigenstates(plan, H, S, 0.0, 3, max_iter=1, tol=1e-14)
    assert e.value.code == 5                                       # not converged: NDSI_ERR_TIMEOUT


def test_eigenstates_periodic_lattice_host_inputs():
    # periodic cell, host H and S (staged inside the call), host output
    sysm = lattice_system((8, 9, 1), 2, "2d", seed=83, periodic=(True, True, False))
    Hd, Sd = sysm.dense()
    xi, n = 0.1, 4
    eps_ref, C_ref = eigenstates_near(Hd, Sd, xi, n)
    nd = lib()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    plan = nd.analyze_system(sysm, cell=sysm.meta["cell"])
    eps, C, res, it = nd.ndsi_eigenstates(plan, sysm.H.copy(), sysm.S.copy(), xi, n, block=8)
    _check(eps, C, res, eps_ref, C_ref, Sd, 1e-11, 1e-8)
