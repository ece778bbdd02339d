"""Pins for the App. B oracle: selected eigenstates near xi and the three-step solve.

Eigenpairs: the open-chain closed form; every pair satisfies H c = eps S c and c^T S c = I.
Three-step solve (B8-B15): dense solves on App. A's matrix and on random perfect-tree
matrices (real and complex shifted), plus a planted mistake (steps applied in place, so later
steps read modified values) that must fail.  The block iteration (B2-B3) converges to the
definition.
"""
import numpy as np
import pytest

from synth import chain_nntb, lattice_system
from oracle.closed_form import chain_spectrum
from oracle.eigen import eigenstates_near, three_step_solve, block_shift_invert
from oracle.recurrence import perfect_layout, recurrence_selected_inverse
from tests.conftest import golden_path


def test_eigenstates_near_chain_closed_form():
    N, a, b, s = 40, 0.1, -0.8, 0.15
    Hd, Sd = chain_nntb(N, a, b, s).dense()
    eps_cf, C_cf = chain_spectrum(N, a, b, s)
    xi = 0.23
    eps, C = eigenstates_near(Hd, Sd, xi, 5)
    pick = np.sort(np.argsort(np.abs(eps_cf - xi))[:5])
    assert np.max(np.abs(eps - eps_cf[pick])) < 1e-13
    # eigenvectors equal up to sign (the chain spectrum is simple)
    for i, k in enumerate(pick):
        sgn = np.sign(C[:, i] @ Sd @ C_cf[:, k])
        assert np.max(np.abs(C[:, i] - sgn * C_cf[:, k])) < 1e-12
    assert np.max(np.abs(C.T @ Sd @ C - np.eye(5))) < 1e-13


def _random_structured(P, rng, complex_shift=None):
    leaf = list(rng.integers(1, 4, 2 ** (P + 1)))
    seps = {p: list(rng.integers(1, 3, 2 ** (P - p))) for p in range(P + 1)}
    dom, sep = perfect_layout(P, leaf, seps)
    n = len(dom[P + 1][0])
    # couplings only along the tree: block ij nonzero when one set contains the other's separator path
    H = np.zeros((n, n))
    def fill(r, c):
        H[np.ix_(r, c)] = rng.normal(0, 0.3, (len(r), len(c)))
    for p in range(P + 1):
        for q in range(2 ** (P + 1 - p)):
            fill(sep[p][q // 2], dom[p][q])
    H = np.tril(H, -1)
    H = H + H.T + np.diag(rng.uniform(-1, 1, n))
    S = np.eye(n) + 0.05 * (np.abs(H) > 0) * (1 - np.eye(n))
    X = H - (complex_shift if complex_shift is not None else 0.3) * S
    return X, P, dom, sep


@pytest.mark.parametrize("P,shift", [(1, None), (2, None), (2, 0.1 + 0.05j), (3, -0.4 + 0.2j)])
def test_three_step_solve_matches_dense(P, shift):
    rng = np.random.default_rng(7 + P)
    X, P, dom, sep = _random_structured(P, rng, shift)
    y = rng.normal(size=(X.shape[0], 3))
    x = three_step_solve(X, P, dom, sep, y)
    ref = np.linalg.solve(X, y)
    assert np.max(np.abs(x - ref)) < 1e-10 * np.max(np.abs(ref))


def test_three_step_solve_appA():
    X = np.loadtxt(golden_path("appA_structured_X.txt"))
    dom, sep = perfect_layout(1, [1, 1, 1, 1], {0: [1, 1], 1: [1]})
    for k in range(7):
        e = np.zeros(7)
        e[k] = 1.0
        assert np.max(np.abs(three_step_solve(X, 1, dom, sep, e)[:, 0] - np.linalg.solve(X, e))) < 1e-12


def test_planted_in_place_forward_step_is_caught():
    # applying (B8) in place (reading separators already changed by lower levels) is wrong
    rng = np.random.default_rng(3)
    X, P, dom, sep = _random_structured(2, rng)
    rec = {}
    recurrence_selected_inverse(X, P, dom, sep, rec)
    L = {(k[1], k[2]): v for k, v in rec.items() if k[0] == "L"}
    y = rng.normal(size=(X.shape[0], 1))
    y_bad = y.copy()
    for p in range(P + 1):
        for n in range(2 ** (P - p)):
            c = sep[p][n]
            y_bad[c] = y_bad[c] - L[(p, 2 * n)] @ y_bad[dom[p][2 * n]] - L[(p, 2 * n + 1)] @ y_bad[dom[p][2 * n + 1]]
    y_good = y.copy()
    for p in range(P + 1):
        for n in range(2 ** (P - p)):
            c = sep[p][n]
            y_good[c] = y[c] - L[(p, 2 * n)] @ y[dom[p][2 * n]] - L[(p, 2 * n + 1)] @ y[dom[p][2 * n + 1]]
    assert np.max(np.abs(y_bad - y_good)) > 1e-3


def test_block_iteration_converges_to_definition():
    sysm = lattice_system((6, 5, 1), 2, "2d", 61)
    Hd, Sd = sysm.dense()
    xi = -0.1
    eps_ref, C_ref = eigenstates_near(Hd, Sd, xi, 4)
    C0 = np.random.default_rng(1).normal(size=(sysm.n, 8))
    eps, C = block_shift_invert(Hd, Sd, xi, C0, 30)
    pick = np.sort(np.argsort(np.abs(eps - xi))[:4])
    assert np.max(np.abs(eps[pick] - eps_ref)) < 1e-11
    # same eigenspace: S-projectors agree
    Pg = C[:, pick] @ C[:, pick].T @ Sd
    Pr = C_ref @ C_ref.T @ Sd
    assert np.max(np.abs(Pg - Pr)) < 1e-8
