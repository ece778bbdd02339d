"""GPU parity of the split-precision (emulated FP64 on BF16 tensor cores) path.

Tolerance: 1e-9 max-abs on rho for the split form (the FP64 form keeps 1e-10).  G is compared
to the dense inverse relative to max|G|.
"""
import numpy as np
import pytest

from synth import config_system, lattice_system
from oracle.dense import (generalized_eig, density_eig, find_mu_eig, on_pattern,
                          electron_count_pattern, green_dense)
from tests.libtools import lib
from tests.test_gpu_parity import _selinv, _density

pytestmark = pytest.mark.gpu

RHO_TOL_SPLIT = 1e-9


@pytest.mark.parametrize("shape,o,nb,leaf", [
    ((40, 1, 1), 3, "1d", 6), ((9, 7, 1), 2, "2d", 5), ((5, 4, 4), 2, "3d", 6),
    ((11, 10, 1), 4, "2d", 20), ((6, 6, 5), 3, "3d", 20)])
def test_split_selected_inverse_matches_dense(shape, o, nb, leaf):
    sysm = lattice_system(shape, o, nb, 77)
    Hd, Sd = sysm.dense()
    Z = [0.1 + 0.0314j, -0.7 + 2.5j, 1e7j]
    g = _selinv(sysm, Z, leaf_atoms=leaf, precision=lib().NDSI_PREC_SPLIT)
    for q, z in enumerate(Z):
        ref = on_pattern(green_dense(Hd, Sd, z), sysm)
        rel = np.max(np.abs(g[q] - ref)) / np.max(np.abs(ref))
        print(f"split G rel err {shape} z={z}: {rel:.2e}")
        assert rel < 1e-9


@pytest.mark.parametrize("outer", [32, 64])
def test_split_outer_blocks(outer):
    # outer panel, trailing update and inverse-assembly GEMMs on the tensor cores between FP64
    # diagonal blocks of `outer` columns
    sysm = lattice_system((6, 6, 5), 3, "3d", 5)
    Hd, Sd = sysm.dense()
    Z = [-0.2 + 0.05j, 0.3 + 1.5j]
    g = _selinv(sysm, Z, leaf_atoms=12, outer_block=outer, precision=lib().NDSI_PREC_SPLIT)
    for q, z in enumerate(Z):
        ref = on_pattern(green_dense(Hd, Sd, z), sysm)
        rel = np.max(np.abs(g[q] - ref)) / np.max(np.abs(ref))
        assert rel < 1e-9


def _rho_split(sysm, kT, M, leaf=20, slices=6):
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    ref = on_pattern(density_eig(eps, C, mu, kT, M), sysm)
    rho, ne = _density(sysm, mu, kT, M, leaf_atoms=leaf, precision=lib().NDSI_PREC_SPLIT,
                       split_slices=slices)
    return rho, ne, ref


def test_split_density_C1():
    sysm = config_system("C1")
    rho, ne, ref = _rho_split(sysm, sysm.meta["kT"], sysm.meta["poles"])
    err = np.max(np.abs(rho - ref))
    print(f"split C1 rho err {err:.2e}")
    assert err < RHO_TOL_SPLIT
    assert abs(ne - sysm.n_electrons) < 1e-7


@pytest.mark.parametrize("shape,o,nb,leaf,M", [
    ((12, 12, 1), 2, "2d", 20, 40), ((6, 6, 6), 2, "3d", 20, 40), ((7, 5, 3), 3, "3d", 8, 60)])
def test_split_density_lattices(shape, o, nb, leaf, M):
    rho, ne, ref = _rho_split(lattice_system(shape, o, nb, 123), 0.01, M, leaf)
    err = np.max(np.abs(rho - ref))
    print(f"split rho err {shape}: {err:.2e}")
    assert err < RHO_TOL_SPLIT


def test_split_error_falls_with_slices():
    sysm = lattice_system((10, 10, 1), 3, "2d", 99)
    errs = {}
    for S in (4, 5, 6, 7):
        rho, ne, ref = _rho_split(sysm, 0.01, 30, slices=S)
        errs[S] = np.max(np.abs(rho - ref))
    print("split rho err by slices", errs)
    assert errs[4] > errs[6]
    assert errs[6] < RHO_TOL_SPLIT and errs[7] < RHO_TOL_SPLIT


def test_split_matches_fp64_path_C2():
    sysm = config_system("C2")
    kT, M, mu = sysm.meta["kT"], sysm.meta["poles"], -0.12
    r64, n64 = _density(sysm, mu, kT, M)
    rs, ns = _density(sysm, mu, kT, M, precision=lib().NDSI_PREC_SPLIT)
    err = np.max(np.abs(rs - r64))
    print(f"split vs fp64 C2: rho {err:.2e}, N_e {abs(ns - n64):.2e}")
    assert err < RHO_TOL_SPLIT


def test_autotune_keeps_accuracy():
    # the autotuner moves each GEMM step to whichever of the tensor-core and FP64 paths is faster;
    # the density must stay within the split tolerance and the graph path must keep working
    import torch
    nd = lib()
    sysm = lattice_system((6, 6, 6), 2, "3d", 123)
    kT, M = 0.01, 40
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    ref = on_pattern(density_eig(eps, C, mu, kT, M), sysm)
    plan = nd.analyze_system(sysm, precision=nd.NDSI_PREC_SPLIT)
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    f_old = nd.ndsi_factor_poles(plan, H, S, np.array([mu + 0.05j]))
    n_split, n_fp64 = nd.ndsi_autotune(plan, H, S, mu, kT, M)
    sched = nd.ndsi_plan_export(plan, "schedule")
    assert n_split + n_fp64 == sum(1 for k, l, t, c in sched if k == 3 and t not in (3, 4, 6, 7))
    # every tensor-core step keeps one of the two tile shapes it was timed with
    shapes = nd.ndsi_plan_export(plan, "tile_shapes")
    assert set(shapes[shapes > 0].tolist()) <= {40, 48}
    assert int((shapes > 0).sum()) == n_split
    assert all(shapes[i] == -1 for i, (k, l, t, c) in enumerate(sched) if k != 3)
    # factors made before the retuning are refused by the selected inversion
    with pytest.raises(nd.NdsiError):
        nd.ndsi_selinv(f_old, None)
    rho = torch.zeros(sysm.nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        nd.ndsi_density(plan, H, S, mu, kT, M, rho, ne)
    torch.cuda.synchronize()
    assert nd.ndsi_graph_info(plan) > 0
    assert np.max(np.abs(rho.cpu().numpy() - ref)) < RHO_TOL_SPLIT


def test_accumulators_per_scale_are_most_accurate():
    # One accumulator per slice-product scale (the default, bands = 0) keeps every scale exact;
    # five bands keep t+u = 2..5 exact and mix the rest in a tail; four leave t+u = 5 in the tail
    # too, where the tensor core drops low bits of the smaller products.
    nd = lib()
    sysm = lattice_system((6, 6, 5), 3, "3d", 5)
    Hd, Sd = sysm.dense()
    Z = [-0.2 + 0.004j, 0.3 + 0.02j]
    refs = [on_pattern(green_dense(Hd, Sd, z), sysm) for z in Z]
    errs = {}
    for bands in (0, 4, 5):
        g = _selinv(sysm, Z, leaf_atoms=12, precision=nd.NDSI_PREC_SPLIT, split_bands=bands)
        errs[bands] = max(np.max(np.abs(g[q] - refs[q])) / np.max(np.abs(refs[q])) for q in range(len(Z)))
    print(f"split G rel err: per scale {errs[0]:.2e}, 4 bands {errs[4]:.2e}, 5 bands {errs[5]:.2e}")
    # Im z = 0.004 is closer to the real axis than any pole of the configs (pi kT >= 0.0063):
    # four bands lose ~4e-9 here, five and one per scale stay well inside the tolerance
    assert errs[5] < 1e-9 and errs[0] < 1e-9
    assert errs[5] < errs[4] / 4
    assert errs[0] <= 2 * errs[5]
    plan = nd.analyze_system(sysm, leaf_atoms=12, precision=nd.NDSI_PREC_SPLIT)
    info = nd.ndsi_plan_info(plan)
    assert info["split_bands"] == info["split_slices"] == 6


@pytest.mark.parametrize("bands", [0, 4, 5])
def test_split_density_bands(bands):
    rho, ne, ref = _rho_split_bands(lattice_system((6, 6, 6), 2, "3d", 123), 0.01, 40, bands)
    assert np.max(np.abs(rho - ref)) < RHO_TOL_SPLIT


def _rho_split_bands(sysm, kT, M, bands):
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    ref = on_pattern(density_eig(eps, C, mu, kT, M), sysm)
    rho, ne = _density(sysm, mu, kT, M, precision=lib().NDSI_PREC_SPLIT, split_bands=bands)
    return rho, ne, ref
