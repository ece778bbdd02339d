"""Pins of the oracle's Krylov column route (oracle/krylov.py), on the CPU.

The route computes rho e_j = S^{-1} e_j + sum_p w_p Re[(alpha_p S - H)^{-1} e_j] (Eq. 8) with
COCG solves, for systems too large for dense or sparse-direct solves.  It is pinned here against
what does not depend on it: the closed-form spectrum of the s-valent chain, dense inverses, and
its own a-posteriori error bound (|A^{-1}| <= 1 / (Im(alpha) lambda_min(S))), which must hold
against the exact columns; planted mistakes must show.
"""
import numpy as np
import pytest

from synth import chain_nntb, lattice_system
from oracle.closed_form import chain_density
from oracle.dense import density_inv, green_dense
from oracle.krylov import (density_columns_krylov, green_columns_krylov, overlap_lower_bound,
                           solve_columns)
from oracle.poles import fermi_from_poles, cf_poles


def _occ(M):
    z, R = cf_poles(M)
    return lambda eps, mu, kT: 2.0 * fermi_from_poles((eps - mu) / kT, z, R)


@pytest.mark.parametrize("M", [20, 60])
def test_chain_columns_match_closed_form(M):
    N, a, b, s, mu, kT = 60, 0.1, -1.0, 0.2, -0.3, 0.02
    sysm = chain_nntb(N, a, b, s)
    cols = [0, 17, N - 1]
    got, info = density_columns_krylov(sysm, mu, kT, M, cols)
    ref, _ = chain_density(N, a, b, s, mu, kT, _occ(M))
    err = np.max(np.abs(got - ref[:, cols]))
    assert err < 1e-12
    assert err <= info["bound"]


def test_lattice_columns_match_dense_route_and_bound():
    sysm = lattice_system((5, 4, 3), 3, "3d", 1201)
    mu, kT, M = -0.12, 0.01, 40
    cols = [0, 77, 150, sysm.n - 1]
    got, info = density_columns_krylov(sysm, mu, kT, M, cols)
    Hd, Sd = sysm.dense()
    ref = density_inv(Hd, Sd, mu, kT, M)[:, cols]
    err = np.max(np.abs(got - ref))
    assert err < 1e-12
    assert err <= info["bound"] < 1e-10
    assert info["max_residual"] <= 1e-13


def test_loose_tolerance_stays_inside_its_bound():
    # a loose residual target leaves a visible error, and the bound still covers it
    sysm = lattice_system((5, 4, 3), 3, "3d", 1201)
    mu, kT, M = -0.12, 0.01, 20
    got, info = density_columns_krylov(sysm, mu, kT, M, [5, 99], tol=1e-5)
    Hd, Sd = sysm.dense()
    err = np.max(np.abs(got - density_inv(Hd, Sd, mu, kT, M)[:, [5, 99]]))
    assert 1e-12 < err <= info["bound"]


@pytest.mark.parametrize("Z", [0.3 + 0.05j, -0.2 - 0.01j, 1e3j])
def test_green_columns_match_dense_inverse(Z):
    sysm = lattice_system((6, 5, 1), 2, "2d", 33)
    Hd, Sd = sysm.dense()
    cols = [1, 30, 59]
    got = green_columns_krylov(sysm, Z, cols)
    ref = green_dense(Hd, Sd, Z)[:, cols]
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref)) / min(1.0, abs(Z.imag))


def test_overlap_solve_is_plain_cg():
    sysm = lattice_system((6, 5, 1), 2, "2d", 34)
    _, Sd = sysm.dense()
    X, it, res = solve_columns(sysm, [1.0, 1.0], [0.0, 0.0], [3, 40])
    ref = np.linalg.inv(Sd)[:, [3, 40]]
    assert np.max(np.abs(X.T - ref)) < 1e-13
    assert np.all(np.abs(X.imag) == 0.0)
    assert overlap_lower_bound(sysm) >= 0.25 - 1e-12


def test_planted_sign_of_h_is_detected():
    # solving (alpha S + H) instead of (alpha S - H): the dense comparison must fail clearly
    sysm = lattice_system((6, 5, 1), 2, "2d", 35)
    Hd, Sd = sysm.dense()
    Z = 0.2 + 0.05j
    X, _, _ = solve_columns(sysm, [Z], [-1.0], [7])
    assert np.max(np.abs(X[0] - green_dense(Hd, Sd, Z)[:, 7])) > 1e-3


def test_residual_target_is_enforced():
    sysm = lattice_system((6, 5, 1), 2, "2d", 36)
    with pytest.raises(RuntimeError):
        solve_columns(sysm, [0.1 + 0.001j], [1.0], [3], max_iter=3)
    with pytest.raises(ValueError):
        solve_columns(sysm, [0.1 + 0.01j], [1.0], [sysm.n])
