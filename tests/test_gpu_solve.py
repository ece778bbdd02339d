"""Solves with the nested-dissection factors (App. B, Eqs. B8-B15) against dense solves."""
import numpy as np
import pytest

from synth import lattice_system
from tests.libtools import lib

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("shape,orb,kind,precision,tol", [
    ((9, 8, 1), 4, "2d", 0, 1e-11),
    ((5, 4, 4), 2, "3d", 0, 1e-11),
    ((9, 8, 1), 4, "2d", 1, 1e-8),
    ((40, 1, 1), 3, "1d", 0, 1e-11),
])
def test_factors_solve_matches_dense(shape, orb, kind, precision, tol):
    torch = _torch()
    nd = lib()
    sysm = lattice_system(shape, orb, kind, seed=71)
    Hd, Sd = sysm.dense()
    z = np.array([0.1 + 0.05j, -0.7 + 0.3j, 2.0 + 1e-3j])
    plan = nd.analyze_system(sysm, precision=precision)
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    f = nd.ndsi_factor_poles(plan, H, S, z)
    rng = np.random.default_rng(5)
    for k in (1, 11):                       # one and two right-hand-side groups (ragged)
        Y = rng.normal(size=(sysm.n, k)) + 1j * rng.normal(size=(sysm.n, k))
        for p, zp in enumerate(z):
            X = np.zeros_like(Y)
            nd.ndsi_factors_solve(f, p, Y, X)
            ref = np.linalg.solve(zp * Sd - Hd, Y)
            err = np.max(np.abs(X - ref)) / np.max(np.abs(ref))
            assert err < tol, (p, k, err)
    # device buffers give the same result
    Yd = torch.as_tensor(Y, device="cuda")
    Xd = torch.zeros_like(Yd)
    nd.ndsi_factors_solve(f, 1, Yd, Xd)
    ref = np.linalg.solve(z[1] * Sd - Hd, Y)
    assert np.max(np.abs(Xd.cpu().numpy() - ref)) / np.max(np.abs(ref)) < tol
    assert np.array_equal(Yd.cpu().numpy(), Y)          # input untouched


def test_solve_after_selinv_is_rejected():
    torch = _torch()
    nd = lib()
    sysm = lattice_system((4, 4, 1), 2, "2d", seed=72)
    plan = nd.analyze_system(sysm)
    f = nd.ndsi_factor_poles(plan, sysm.H, sysm.S, np.array([0.1 + 0.1j]))
    Y = np.ones((sysm.n, 1), dtype=np.complex128)
    X = np.zeros_like(Y)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_factors_solve(f, 1, Y, X)                 # pole out of range
    nd.ndsi_selinv(f)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_factors_solve(f, 0, Y, X)
