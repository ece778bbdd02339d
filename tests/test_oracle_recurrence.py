"""Pins for the recurrence oracle (Eqs. 28-32, 38-39) against App. A and dense inverses."""
import numpy as np
import pytest

from oracle.recurrence import perfect_layout, recurrence_selected_inverse
from tests.conftest import golden_lines, golden_path


def _appA():
    X = np.loadtxt(golden_path("appA_structured_X.txt"))
    dom, sep = perfect_layout(1, [1, 1, 1, 1], {0: [1, 1], 1: [1]})
    return X, dom, sep


def test_appA_intermediates():
    X, dom, sep = _appA()
    rec = {}
    recurrence_selected_inverse(X, 1, dom, sep, rec)
    for line in golden_lines("appA_intermediates.txt"):
        key, vals = line.split(":")
        parts = key.split()
        k = (parts[0],) + tuple(int(v) for v in parts[1:])
        want = np.array([float(v) for v in vals.split()])
        assert np.allclose(rec[k].ravel(), want, atol=0), k


def test_appA_selected_inverse():
    X, dom, sep = _appA()
    G = recurrence_selected_inverse(X, 1, dom, sep)
    rows = [ln.split() for ln in golden_lines("appA_selected_inverse.txt")]
    for i in range(7):
        for j in range(7):
            if rows[i][j] != "*":
                assert G[i, j] == float(rows[i][j]), (i, j)


def test_appA_as_printed_is_inconsistent():
    # The matrix as printed (root coupled to positions 2 and 5) cannot produce the printed
    # inverse: eight printed elements disagree with its exact inverse.
    X, _, _ = _appA()
    Xp = X.copy()
    Xp[3, 6] = Xp[6, 3] = 0
    Xp[4, 6] = Xp[6, 4] = 1
    rows = [ln.split() for ln in golden_lines("appA_selected_inverse.txt")]
    Gp = np.linalg.inv(Xp)
    bad = sum(abs(Gp[i, j] - float(rows[i][j])) > 1e-12
              for i in range(7) for j in range(7) if rows[i][j] != "*")
    assert bad == 8


@pytest.mark.parametrize("P,leaf,sepsz", [(1, 3, 2), (2, 2, 1), (2, 4, 3)])
def test_recurrence_equals_dense_inverse(P, leaf, sepsz):
    # A random complex-symmetric chain-like structured matrix: the computed blocks of
    # Eq. (38) equal the dense inverse (brute force).
    rng = np.random.default_rng(P * 100 + leaf)
    leaf_sizes = [leaf] * 2 ** (P + 1)
    sep_sizes = {p: [sepsz] * 2 ** (P - p) for p in range(P + 1)}
    dom, sep = perfect_layout(P, leaf_sizes, sep_sizes)
    n = len(dom[P + 1][0])
    # couple each separator to its two domains (dense random blocks), plus diagonal blocks
    X = np.zeros((n, n), dtype=complex)
    for n0, idx in dom[0].items():
        X[np.ix_(idx, idx)] = rng.normal(size=(leaf, leaf))
    for p in range(P + 1):
        for k, s in sep[p].items():
            X[np.ix_(s, s)] = rng.normal(size=(sepsz, sepsz))
            for d in (dom[p][2 * k], dom[p][2 * k + 1]):
                X[np.ix_(s, d)] = rng.normal(size=(sepsz, len(d))) * (rng.random((sepsz, len(d))) < 0.5)
    X = X + X.T + (0.7 + 0.9j) * np.eye(n)
    G = recurrence_selected_inverse(X, P, dom, sep)
    ref = np.linalg.inv(X)
    m = ~np.isnan(G.real)
    assert m.sum() > n
    assert np.max(np.abs(G[m] - ref[m])) < 1e-10 * max(1.0, np.max(np.abs(ref)))
