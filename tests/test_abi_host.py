"""Host-side checks of the C-ABI library: symbols, pole generator, bit-exact structure analysis.

No GPU compute is called here (ndsi_analyze, ndsi_plan_* and ndsi_poles are host code)."""
import ctypes

import numpy as np
import pytest

from synth import chain_nntb, config_system, lattice_system, csr_from_dense
from oracle.nd import atom_adjacency, nested_dissection, symbolic_structure
from oracle.poles import cf_poles
from tests.libtools import lib, header_functions
from tests.conftest import golden_lines


def test_library_exports_every_declared_symbol():
    nd = lib()
    declared = header_functions()
    assert len(declared) >= 11
    for name in declared:
        assert hasattr(nd.load(), name), name
    assert set(nd.EXPORTED_SYMBOLS) <= set(declared)


@pytest.mark.parametrize("M", [1, 3, 40, 80, 160])
def test_poles_match_oracle(M):
    nd = lib()
    z, R = nd.ndsi_poles(M)
    z0, R0 = cf_poles(M)
    assert np.max(np.abs(z - z0) / z0) < 1e-13
    assert np.max(np.abs(R - R0) / np.abs(R0)) < 1e-11


def _compare_structure(system, leaf, cell=None, screen_degree=0):
    nd = lib()
    opts = {} if cell is None else {"cell": cell}
    plan = nd.analyze_system(system, leaf_atoms=leaf, screen_degree=screen_degree, **opts)
    adj = atom_adjacency(system)
    tr = nested_dissection(system.centers, adj, leaf, cell=cell, screen_degree=screen_degree)
    st = symbolic_structure(tr, adj)
    assert np.array_equal(nd.ndsi_plan_export(plan, "perm_atoms"), tr["perm_atoms"])
    assert np.array_equal(nd.ndsi_plan_export(plan, "parent"), tr["parent"])
    na = nd.ndsi_plan_export(plan, "node_atoms")
    assert [na[j + 1] - na[j] for j in range(len(tr["nodes"]))] == [len(x) for x in tr["nodes"]]
    sp = nd.ndsi_plan_export(plan, "struct_ptr")
    sa = nd.ndsi_plan_export(plan, "struct_atoms")
    for j, s in enumerate(st):
        assert sa[sp[j]:sp[j + 1]].tolist() == s
    # basis permutation keeps every atom's orbitals together, in ascending order
    pb = nd.ndsi_plan_export(plan, "perm_basis")
    aob = system.atom_of_basis
    assert sorted(pb.tolist()) == list(range(system.n))
    assert np.array_equal(aob[pb], np.repeat(tr["perm_atoms"], np.bincount(aob)[tr["perm_atoms"]]))
    return plan


def test_appA_ordering_bit_exact():
    s = chain_nntb(7, 1.0, 1.0, 0.0)
    plan = _compare_structure(s, 1)
    nd = lib()
    perm = [int(v) for v in golden_lines("appA_ordering.txt")[0].split()]
    assert (nd.ndsi_plan_export(plan, "perm_atoms") + 1).tolist() == perm


@pytest.mark.parametrize("name", ["C1", "C2", "C3"])
def test_config_structure_bit_exact(name):
    _compare_structure(config_system(name), 20)


@pytest.mark.parametrize("seed,shape,o,nb,leaf", [
    (1, (9, 1, 1), 3, "1d", 2), (2, (7, 5, 1), 2, "2d", 3), (3, (4, 5, 3), 1, "3d", 4),
    (4, (13, 11, 1), 1, "2d", 5), (5, (5, 5, 5), 2, "3d", 7)])
def test_random_structure_bit_exact(seed, shape, o, nb, leaf):
    _compare_structure(lattice_system(shape, o, nb, seed), leaf)


@pytest.mark.parametrize("shape,o,nb,periodic,leaf", [
    ((32, 32, 1), 1, "2dnn", (True, True, False), 20), ((12, 1, 1), 3, "1d", (True, False, False), 2),
    ((9, 7, 1), 2, "2d", (True, False, False), 4), ((5, 4, 6), 1, "3d", (True, True, True), 5),
    ((6, 6, 6), 2, "3d", (False, True, False), 8)])
def test_periodic_structure_bit_exact(shape, o, nb, periodic, leaf):
    s = lattice_system(shape, o, nb, 11, periodic=periodic)
    _compare_structure(s, leaf, cell=s.meta["cell"])
    # coordinates moved by -0.4 cells (wrapping differs from the unshifted lattice)
    cell = np.array(s.meta["cell"])
    s.centers = s.centers - 0.4 * cell[None, :]
    _compare_structure(s, leaf, cell=s.meta["cell"])


def test_screened_structure_bit_exact():
    from tests.test_oracle_nd import _long_tail_system
    s = _long_tail_system(lattice_system((10, 9, 1), 2, "2d", 8), 3, 4.0, 2)
    _compare_structure(s, 6, screen_degree=12)
    _compare_structure(s, 6)


def test_shuffled_atoms_bit_exact():
    # Atom numbering unrelated to geometry (ties in coordinates resolved by atom index).
    rng = np.random.default_rng(9)
    s = lattice_system((6, 6, 1), 2, "2d", 21)
    perm = rng.permutation(s.n_atoms)
    cen = s.centers[perm]
    Hd, Sd = s.dense()
    o = 2
    bperm = (perm[:, None] * o + np.arange(o)[None]).ravel()
    s2 = csr_from_dense(Hd[np.ix_(bperm, bperm)], Sd[np.ix_(bperm, bperm)], cen,
                        np.repeat(np.arange(s.n_atoms), o))
    _compare_structure(s2, 4)


def test_plan_info_counts():
    nd = lib()
    s = config_system("C2")
    info = nd.ndsi_plan_info(nd.analyze_system(s))
    assert info["n"] == 4096 and info["nnz"] == s.nnz and info["n_atoms"] == 1024
    assert info["n_levels"] >= 6 and info["flops_per_pole"] > 1e8


def _raw_analyze(n, rowptr, col, n_atoms, centers, aob):
    nd = lib()
    with pytest.raises(nd.NdsiError) as ei:
        nd.ndsi_analyze(n, rowptr, col, n_atoms, centers, aob)
    return ei.value.code


def test_invalid_patterns_rejected():
    nd = lib()
    cen = np.zeros((3, 3))
    cen[:, 0] = np.arange(3)
    aob = np.arange(3)
    # missing diagonal in row 1
    assert _raw_analyze(3, [0, 2, 3, 5], [0, 1, 0, 1, 2], 3, cen, aob) == nd.ndsi.NDSI_ERR_INVALID
    # asymmetric: (0,2) without (2,0)
    assert _raw_analyze(3, [0, 2, 3, 4], [0, 2, 1, 2], 3, cen, aob) == nd.ndsi.NDSI_ERR_INVALID
    # unsorted columns
    assert _raw_analyze(3, [0, 2, 4, 5], [1, 0, 0, 1, 2], 3, cen, aob) == nd.ndsi.NDSI_ERR_INVALID
    # atom without basis functions
    assert _raw_analyze(3, [0, 1, 2, 3], [0, 1, 2], 4, np.zeros((4, 3)), aob) == nd.ndsi.NDSI_ERR_INVALID
    with pytest.raises(nd.NdsiError):
        nd.ndsi_poles(0)


def test_invalid_options_rejected():
    nd = lib()
    sysm = lattice_system((4, 4, 1), 2, "2d", 3)
    for opts in (dict(block=24), dict(outer_block=40), dict(outer_block=48, block=32),
                 dict(precision=1, split_slices=3), dict(cell=(-1.0, 0.0, 0.0)),
                 dict(cell=(float("nan"), 0.0, 0.0)), dict(screen_degree=-1)):
        with pytest.raises(nd.NdsiError) as ei:
            nd.analyze_system(sysm, **opts)
        assert ei.value.code == nd.ndsi.NDSI_ERR_INVALID


def test_two_level_schedule():
    # diagonal blocks of outer_block columns: exactly ceil(s / outer) - 1 outer panel steps for
    # the widest node of a level, and the pivot-level GEMMs never leave the diagonal blocks
    nd = lib()
    sysm = lattice_system((6, 6, 5), 3, "3d", 5)
    for outer in (32, 64, 128):
        p = nd.analyze_system(sysm, leaf_atoms=12, outer_block=outer)
        sch = nd.ndsi_plan_export(p, "schedule")
        na = nd.ndsi_plan_export(p, "node_atoms")
        lv = nd.ndsi_plan_export(p, "level")
        s = np.diff(na) * 3
        for L in range(lv.max() + 1):
            smax = s[lv == L].max()
            n_outer = sum(1 for k, l, t, c in sch if k == 3 and l == L and t == 16)  # opanel
            assert n_outer == -(-smax // outer) - 1, (outer, L, smax, n_outer)


def test_batched_plan_merges_levels():
    # Three uneven systems in one plan: one schedule, levels aligned, fewer launches than
    # the three plans run one after another.
    nd = lib()
    systems = [lattice_system((30, 1, 1), 3, "1d", 1), lattice_system((7, 6, 1), 2, "2d", 2),
               lattice_system((4, 4, 3), 2, "3d", 3)]
    singles = [nd.ndsi_plan_info(nd.analyze_system(s)) for s in systems]
    info = nd.ndsi_plan_info(nd.analyze_batched(systems))
    assert info["n_systems"] == 3
    assert info["n"] == sum(s.n for s in systems) and info["nnz"] == sum(s.nnz for s in systems)
    assert info["n_nodes"] == sum(i["n_nodes"] for i in singles)
    assert info["n_levels"] == max(i["n_levels"] for i in singles)
    assert info["front_elems"] == sum(i["front_elems"] for i in singles)
    assert info["n_launches"] < sum(i["n_launches"] for i in singles)
    assert abs(info["flops_per_pole"] - sum(i["flops_per_pole"] for i in singles)) < 1e-6 * info["flops_per_pole"]
