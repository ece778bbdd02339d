"""The seeded input generators: structure and the guarantees the recipe states (no method
arithmetic here; these are the inputs both the oracle and the library consume)."""
import numpy as np
import pytest

from synth import lattice_system, config_system, chain_nntb


@pytest.mark.parametrize("shape,nb,periodic,neigh", [
    ((6, 5, 1), "2dnn", (True, True, False), 4), ((7, 1, 1), "1d", (True, False, False), 2),
    ((4, 3, 5), "3d", (True, True, True), 26), ((6, 6, 1), "2d", (True, True, False), 8)])
def test_periodic_lattices_have_full_neighbour_shells(shape, nb, periodic, neigh):
    s = lattice_system(shape, 2, nb, 3, periodic=periodic)
    aob = s.atom_of_basis
    rows = s.rows()
    pairs = {(int(a), int(b)) for a, b in zip(aob[rows], aob[s.col]) if a != b}
    deg = np.bincount([a for a, _ in pairs], minlength=s.n_atoms)
    assert np.all(deg == neigh)
    assert s.meta["cell"] == tuple(float(n) if p else 0.0 for n, p in zip(shape, periodic))


@pytest.mark.parametrize("system", [
    lattice_system((6, 5, 1), 3, "2d", 4), lattice_system((5, 4, 4), 2, "3d", 5, periodic=(True, True, True)),
    chain_nntb(30, 0.1, -0.8, 0.15)])
def test_matrices_symmetric_and_overlap_positive(system):
    Hd, Sd = system.dense()
    assert np.array_equal(Hd, Hd.T) and np.array_equal(Sd, Sd.T)
    assert np.linalg.eigvalsh(Sd).min() >= 0.25 - 1e-12


def test_periodic_axis_needs_three_atoms():
    with pytest.raises(ValueError):
        lattice_system((2, 5, 1), 1, "2d", 1, periodic=(True, False, False))


def test_seeds_reproduce():
    a, b = config_system("C1"), config_system("C1")
    assert np.array_equal(a.H, b.H) and np.array_equal(a.S, b.S) and np.array_equal(a.col, b.col)
