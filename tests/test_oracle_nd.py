"""Pins for the nested-dissection oracle (Sec. II.C.1) and its symbolic fill."""
import numpy as np
import pytest

from synth import chain_nntb, lattice_system, config_system
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
