"""GPU density of states from the retarded Green function (Eq. 41) and the chemical-potential
search that starts from it (procedure (2), Eqs. 41-43), against the oracle."""
import numpy as np
import pytest

from synth import lattice_system, chain_nntb
from oracle.dense import generalized_eig, dos_eig, find_mu_eig, electron_count_eig
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
    return nd, plan, H, S


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-8)])
def test_dos_matches_lorentzian_sum(precision, tol):
    sysm = lattice_system((9, 8, 1), 4, "2d", seed=51)      # several fronts, ragged blocks
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    E = np.concatenate([np.linspace(eps[0] - 0.5, eps[-1] + 0.5, 37), [eps[0], eps[len(eps) // 2]]])
    nd, plan, H, S = _setup(sysm, precision=precision)
    for eta in (0.02, 0.3):
        d = nd.ndsi_dos(plan, H, S, E, eta)
        ref = dos_eig(eps, E, eta)
        assert np.max(np.abs(d - ref)) < tol * np.max(ref), (eta, np.max(np.abs(d - ref)))


def test_dos_chunked_and_host_inputs():
    sysm = chain_nntb(200, 0.1, -0.8, 0.15)
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    E = np.linspace(-2.0, 2.0, 7)
    nd, plan, H, S = _setup(sysm)
    whole = nd.ndsi_dos(plan, H, S, E, 0.05)
    info = nd.ndsi_plan_info(plan)
    small = nd.analyze_system(sysm, max_workspace_bytes=int(info["front_elems"] * 16 * 3))
    chunked = nd.ndsi_dos(small, sysm.H, sysm.S, E, 0.05)        # host H, S; points in chunks
    ref = dos_eig(eps, E, 0.05)
    assert np.max(np.abs(whole - ref)) < 1e-10 * np.max(ref)
    assert np.max(np.abs(chunked - whole)) < 1e-12 * np.max(ref)


def test_dos_rejects_bad_arguments():
    sysm = lattice_system((4, 4, 1), 2, "2d", 3)
    nd, plan, H, S = _setup(sysm)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_dos(plan, H, S, [0.0], 0.0)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_dos(plan, H, S, [], 0.1)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_dos(plan, H, S, [np.nan], 0.1)
    batched = nd.analyze_batched([sysm, sysm])
    import torch
    H2 = torch.cat([H, H]); S2 = torch.cat([S, S])
    with pytest.raises(nd.NdsiError):
        nd.ndsi_dos(batched, H2, S2, [0.0], 0.1)


@pytest.mark.parametrize("seed", [810, 811])
def test_find_mu_procedure_2_start(seed):
    # unbracketed search: DeltaN at the middle of the bounds, the DOS trial mu, DeltaN there; it
    # must converge to the oracle's root and in fewer sweeps than a bracket spanning the spectrum
    import torch
    sysm = lattice_system((10, 10, 1), 3, "2d", seed)
    kT, M = 0.01, 40
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    nd, plan, H, S = _setup(sysm)
    rho = torch.zeros(sysm.nnz, dtype=torch.float64, device="cuda")
    mu0, ne0, it0 = nd.ndsi_find_mu(plan, H, S, kT, M, sysm.n_electrons, rho)
    mu1, ne1, it1 = nd.ndsi_find_mu(plan, H, S, kT, M, sysm.n_electrons, rho,
                                    mu_lo=eps[0] - 1.0, mu_hi=eps[-1] + 1.0)
    print(f"find_mu procedure (2) start: {it0} sweeps; spectrum-wide bracket: {it1}")
    assert abs(ne0 - sysm.n_electrons) < 1e-8 and abs(ne1 - sysm.n_electrons) < 1e-8
    assert abs(electron_count_eig(eps, mu0, kT, M) - sysm.n_electrons) < 1e-7
    assert it0 < it1 and it0 <= 10
