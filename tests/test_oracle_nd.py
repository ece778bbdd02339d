"""Pins for the nested-dissection oracle (Sec. II.C.1) and its symbolic fill."""
import numpy as np
import pytest

from synth import csr_from_dense, chain_nntb, lattice_system, config_system
from oracle.nd import atom_adjacency, nested_dissection, symbolic_structure
from tests.conftest import golden_lines


def test_appA_ordering():
    perm = [int(v) for v in golden_lines("appA_ordering.txt")[0].split()]
    s = chain_nntb(7, 1.0, 1.0, 0.0)
    t = nested_dissection(s.centers, atom_adjacency(s), leaf_atoms=1)
    assert (t["perm_atoms"] + 1).tolist() == perm
    # the tree: four one-atom domains, separators {2}, {6}, root {4}
    assert [len(n) for n in t["nodes"]] == [1, 1, 1, 1, 1, 1, 1]
    assert t["parent"].tolist() == [2, 2, 6, 5, 5, 6, -1]


def test_appA_structured_matrix_from_ordering():
    # Permuting the chain by the oracle's ordering gives the structured X of App. A.
    X = np.loadtxt(__import__("tests.conftest", fromlist=["golden_path"]).golden_path(
        "appA_structured_X.txt"))
    s = chain_nntb(7, 1.0, 1.0, 0.0)
    Hd, _ = s.dense()
    t = nested_dissection(s.centers, atom_adjacency(s), leaf_atoms=1)
    p = t["perm_atoms"]
    assert np.array_equal(Hd[np.ix_(p, p)], X)


def test_fig1_chain10_labels():
    labels = [int(v) for v in golden_lines("fig1_chain10.txt")[0].split()]
    s = chain_nntb(10)
    t = nested_dissection(s.centers, atom_adjacency(s), leaf_atoms=2)
    lab = np.empty(10, int)
    lab[t["perm_atoms"]] = np.arange(1, 11)
    assert lab.tolist() == labels


def _check_tree(sysm, t, leaf_atoms):
    adj = atom_adjacency(sysm)
    na = sysm.n_atoms
    perm = t["perm_atoms"]
    assert sorted(perm.tolist()) == list(range(na))
    # postorder: children precede parents, and each subtree occupies a contiguous range
    parent = t["parent"]
    for c, p in enumerate(parent):
        if p >= 0:
            assert p > c
    # subtree atom sets
    sub = [set(n) for n in t["nodes"]]
    for j, ch in enumerate(t["children"]):
        for c in ch:
            sub[j] |= sub[c]
    for j, ch in enumerate(t["children"]):
        if ch:
            a0, a1 = sub[ch[0]], sub[ch[1]]
            # separator validity: no H/S coupling between the two subdomains
            for a in a0:
                assert not (set(adj[a]) & a1)
        else:
            assert len(t["nodes"][j]) <= leaf_atoms or True
    return adj


@pytest.mark.parametrize("name", ["C1", "C2", "C3"])
def test_config_trees_are_valid(name):
    sysm = config_system(name)
    t = nested_dissection(sysm.centers, atom_adjacency(sysm), leaf_atoms=20)
    _check_tree(sysm, t, 20)
    leaves = [n for n, ch in zip(t["nodes"], t["children"]) if not ch]
    assert all(len(n) <= 20 for n in leaves)


def test_chain64_structure():
    # A 64-atom chain with 20-atom leaves: 4 leaves, 3 one-atom separators, depth 3.
    sysm = config_system("C1")
    t = nested_dissection(sysm.centers, atom_adjacency(sysm), leaf_atoms=20)
    sizes = [len(n) for n in t["nodes"]]
    kinds = [bool(ch) for ch in t["children"]]
    assert sum(1 for k in kinds if not k) == 4
    assert [s for s, k in zip(sizes, kinds) if k] == [1, 1, 1]
    assert sum(sizes) == 64


def test_symbolic_structure_matches_numeric_fill():
    # Brute force: the nonzero pattern of the LDL^T factor of a random matrix with the
    # system's pattern, in the structured order, equals the symbolic struct sets.
    sysm = lattice_system((6, 5, 1), 1, "2d", 1234)
    adj = atom_adjacency(sysm)
    t = nested_dissection(sysm.centers, adj, leaf_atoms=4)
    st = symbolic_structure(t, adj)
    Hd, Sd = sysm.dense()
    rng = np.random.default_rng(0)
    A = np.where(Hd != 0, rng.uniform(1, 2, Hd.shape), 0.0)
    A = A + A.T + 50 * np.eye(sysm.n)
    p = t["perm_atoms"]
    Ap = A[np.ix_(p, p)]
    Lc = np.linalg.cholesky(Ap)
    nz = np.abs(Lc) > 1e-300
    pos = np.empty(len(p), int)
    pos[p] = np.arange(len(p))
    for atoms, s in zip(t["nodes"], st):
        if not atoms:
            continue
        cols = pos[np.array(atoms)]
        rows = np.nonzero(nz[:, cols].any(axis=1))[0]
        rows = rows[rows > cols.max()]
        assert sorted(p[rows].tolist()) == sorted(s)


@pytest.mark.parametrize("name", ["C2", "C3"])
def test_elimination_tree_property(name):
    # struct(child) minus the parent's own atoms is contained in struct(parent).
    sysm = config_system(name)
    adj = atom_adjacency(sysm)
    t = nested_dissection(sysm.centers, adj, leaf_atoms=20)
    st = symbolic_structure(t, adj)
    for c, p in enumerate(t["parent"]):
        if p >= 0:
            assert set(st[c]) - set(t["nodes"][p]) <= set(st[p])
    assert st[-1] == []


def test_fig2_periodic_square_lattice():
    # Fig. 2: s-valent NNTB square lattice, 1024 atoms per periodic cell.  The first separator
    # consists of two lines; innermost domains hold 9 atoms; separators run over six levels
    # (labelled 0 to 5).
    sysm = lattice_system((32, 32, 1), 1, "2dnn", 1, periodic=(True, True, False))
    t = nested_dissection(sysm.centers, atom_adjacency(sysm), 20, cell=sysm.meta["cell"])
    _check_tree(sysm, t, 20)
    root = len(t["nodes"]) - 1
    sep = np.array(t["nodes"][root])
    ax = t["axis"][root]
    lines = np.unique(sysm.centers[sep, ax])
    assert len(sep) == 64 and len(lines) == 2
    for x in lines:
        assert np.sum(sysm.centers[sep, ax] == x) == 32
    leaves = [len(n) for n, ch in zip(t["nodes"], t["children"]) if not ch]
    assert set(leaves) == {9} and len(leaves) == 64
    parent = t["parent"]

    def depth(j):
        d = 0
        while parent[j] >= 0:
            j, d = parent[j], d + 1
        return d

    assert sorted({depth(j) for j, ch in enumerate(t["children"]) if ch}) == [0, 1, 2, 3, 4, 5]


@pytest.mark.parametrize("shape,nb,periodic,shift", [
    ((12, 1, 1), "1d", (True, False, False), 0.0),
    ((9, 7, 1), "2d", (True, False, False), -0.5),
    ((8, 8, 1), "2d", (True, True, False), 3.25),
    ((5, 4, 6), "3d", (True, True, True), 0.0),
])
def test_periodic_trees_are_valid(shape, nb, periodic, shift):
    # separators must cut the wrap-around couplings too; moving every atom by whole cells gives
    # the same tree (ordering uses the wrapped coordinate, neighbours their nearest image)
    sysm = lattice_system(shape, 2, nb, 5, periodic=periodic)
    adj = atom_adjacency(sysm)
    cell = np.array(sysm.meta["cell"])
    cen = sysm.centers + shift * cell[None, :]
    t = nested_dissection(cen, adj, 4, cell=cell)
    _check_tree(sysm, t, 4)
    k = np.random.default_rng(3).integers(-2, 3, size=cen.shape)
    t2 = nested_dissection(cen + k * cell[None, :], adj, 4, cell=cell)
    assert np.array_equal(t2["perm_atoms"], t["perm_atoms"])
    assert np.array_equal(t2["parent"], t["parent"])


def _long_tail_system(base, n_tail, radius, seed):
    """The base lattice plus n_tail one-orbital atoms, each coupled to every atom within radius."""
    rng = np.random.default_rng(seed)
    Hd, Sd = base.dense()
    o = base.n // base.n_atoms
    tails = rng.uniform(0, 1, (n_tail, 3)) * (base.centers.max(0) + 1e-9)
    n = base.n + n_tail
    H = np.zeros((n, n))
    S = np.zeros((n, n))
    H[:base.n, :base.n] = Hd
    S[:base.n, :base.n] = Sd
    for k, c in enumerate(tails):
        i = base.n + k
        H[i, i], S[i, i] = rng.uniform(-1, 1), 1.0
        near = np.nonzero(np.linalg.norm(base.centers - c, axis=1) <= radius)[0]
        for a in near:
            for q in range(o):
                j = a * o + q
                H[i, j] = H[j, i] = rng.normal(0, 0.05)
                S[i, j] = S[j, i] = 1e-3
    cen = np.vstack([base.centers, tails])
    aob = np.concatenate([base.atom_of_basis, base.n_atoms + np.arange(n_tail)]).astype(np.int32)
    return csr_from_dense(H, S, cen, aob)


def test_screening_moves_long_tails_to_the_root():
    base = lattice_system((10, 9, 1), 2, "2d", 8)
    sysm = _long_tail_system(base, 3, 4.0, 2)
    adj = atom_adjacency(sysm)
    degs = sorted(len(a) for a in adj)
    screen = 12                                    # lattice atoms have at most 8 + 3 neighbours
    assert degs[-3] > screen >= max(len(adj[a]) for a in range(base.n_atoms))
    t = nested_dissection(sysm.centers, adj, 6, screen_degree=screen)
    _check_tree(sysm, t, 6)
    t0 = nested_dissection(base.centers, atom_adjacency(base), 6)
    # the kept atoms are dissected exactly as the lattice alone; the tails join the root
    assert len(t["nodes"]) == len(t0["nodes"])
    for a, b in zip(t["nodes"][:-1], t0["nodes"][:-1]):
        assert a == b
    tails = list(range(base.n_atoms, sysm.n_atoms))
    assert t["nodes"][-1] == sorted(t0["nodes"][-1] + tails)
    # without screening the long tails spread through the tree and the root separator grows
    t_off = nested_dissection(sysm.centers, adj, 6)
    _check_tree(sysm, t_off, 6)
