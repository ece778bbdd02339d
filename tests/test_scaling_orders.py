"""Computational order of the path from the host analysis (flops per pole of factor + selected
inversion) on the periodic s-valent NNTB lattices of Fig. 4 (leaf domains of 20 atoms).

The paper's recurrence (Eqs. 28-32, Table II) costs O(N (log2 N)^2), O(N^2) and O(N^{7/3}) for
1D, 2D and 3D lattices (fitted from timings: N^0.90 (log2 N)^2, N^1.90, N^2.35, Fig. 4).  The
multifrontal form built here keeps every dense block on struct(J) only, and reaches the orders of
nested-dissection factorisation instead: N, N^{3/2} and N^2.
"""
import numpy as np
import pytest

from synth import lattice_system
from tests.libtools import lib


def _order(shapes, nb, periodic):
    nd = lib()
    N, F = [], []
    for sh in shapes:
        s = lattice_system(sh, 1, nb, 1, periodic=periodic)
        N.append(s.n)
        F.append(nd.ndsi_plan_info(nd.analyze_system(s, cell=s.meta["cell"]))["flops_per_pole"])
    return np.polyfit(np.log(N), np.log(F), 1)[0]


@pytest.mark.parametrize("label,shapes,nb,periodic,lo,hi,paper", [
    ("1D", [(n, 1, 1) for n in (512, 1024, 2048, 4096, 8192)], "1d", (True, False, False), 0.95, 1.10, None),
    ("2D", [(L, L, 1) for L in (24, 32, 48, 64, 96)], "2dnn", (True, True, False), 1.45, 1.65, 1.90),
    ("3D", [(L, L, L) for L in (10, 12, 16, 20, 24)], "3d", (True, True, True), 1.95, 2.20, 2.35)])
def test_flop_orders(label, shapes, nb, periodic, lo, hi, paper):
    p = _order(shapes, nb, periodic)
    print(f"{label}: flops per pole ~ N^{p:.3f}")
    assert lo < p < hi
    if paper is not None:
        assert p < paper
