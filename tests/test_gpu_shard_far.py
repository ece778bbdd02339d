"""GPU checks of the pole-sharded density, the far-pole slice relaxation of split plans and the
FP64 throughput probe.

* ndsi_density_poles: the shares ndsi_pole_shard assigns to 1, 2, 3 and 5 ranks sum to
  ndsi_density's rho and Tr(rho S) (FP64 and split plans); an empty share writes zeros; the
  batched form sums to ndsi_density_batched for every system.
* split_far_ratio: with the relaxation (default) and without it the density stays within the
  split tolerance of the oracle; it changes nothing on FP64 plans and nothing in ndsi_selinv.
* ndsi_fp64_peak: a plausible DFMA rate.
"""
import numpy as np
import pytest

from synth import lattice_system
from oracle.dense import generalized_eig, density_eig, on_pattern, green_dense
from tests.libtools import lib
from tests.test_gpu_parity import _density, _selinv

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision", [0, 1])
def test_pole_shares_sum_to_density(precision):
    torch = _torch()
    nd = lib()
    s = lattice_system((7, 6, 3), 2, "3d", 515)
    mu, kT, M = -0.05, 0.01, 40
    plan = nd.analyze_system(s, precision=precision)
    H = torch.as_tensor(s.H, device="cuda")
    S = torch.as_tensor(s.S, device="cuda")
    rho = torch.zeros(s.nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density(plan, H, S, mu, kT, M, rho, ne)
    ref, ne_ref = rho.cpu().numpy(), float(ne.cpu()[0])
    for world in (1, 2, 3, 5):
        tot = np.zeros(s.nnz)
        tot_ne = 0.0
        for r in range(world):
            b, e, m0 = nd.ndsi_pole_shard(M, r, world)
            part = torch.full((s.nnz,), float("nan"), dtype=torch.float64, device="cuda")
            pne = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            nd.ndsi_density_poles(plan, H, S, mu, kT, M, b, e, m0, part, pne)
            tot += part.cpu().numpy()
            tot_ne += float(pne.cpu()[0])
        assert np.max(np.abs(tot - ref)) < 1e-13, world
        assert abs(tot_ne - ne_ref) < 1e-10, world
    # an empty share (no poles, no M0) writes zeros; host outputs work as for ndsi_density
    part = np.full(s.nnz, np.nan)
    pne = np.full(1, np.nan)
    nd.ndsi_density_poles(plan, s.H.copy(), s.S.copy(), mu, kT, M, 7, 7, False, part, pne)
    assert np.all(part == 0.0) and pne[0] == 0.0
    with pytest.raises(nd.NdsiError):
        nd.ndsi_density_poles(plan, H, S, mu, kT, M, 5, 41, True, rho, ne)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_pole_shares_sum_to_batched_density(precision):
    torch = _torch()
    nd = lib()
    systems = [lattice_system((9, 1, 1), 3, "1d", 701), lattice_system((5, 4, 1), 2, "2d", 702),
               lattice_system((4, 3, 3), 2, "3d", 703)]
    plan = nd.analyze_batched(systems, precision=precision)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device="cuda")
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device="cuda")
    nnz = int(H.shape[0])
    mus, kts, M = np.array([-0.1, 0.0, 0.05]), np.array([0.01, 0.02, 0.015]), 30
    rho = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(3, dtype=torch.float64, device="cuda")
    nd.ndsi_density_batched(plan, H, S, mus, kts, M, rho, ne)
    ref, ne_ref = rho.cpu().numpy(), ne.cpu().numpy()
    for world in (2, 4):
        tot, tot_ne = np.zeros(nnz), np.zeros(3)
        for r in range(world):
            b, e, m0 = nd.ndsi_pole_shard(M, r, world)
            part = torch.full((nnz,), float("nan"), dtype=torch.float64, device="cuda")
            pne = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            nd.ndsi_density_batched_poles(plan, H, S, mus, kts, M, b, e, m0, part, pne)
            tot += part.cpu().numpy()
            tot_ne += pne.cpu().numpy()
        assert np.max(np.abs(tot - ref)) < 1e-13, world
        assert np.max(np.abs(tot_ne - ne_ref)) < 1e-10, world


def test_far_pole_relaxation_keeps_split_tolerance():
    s = lattice_system((7, 6, 5), 3, "3d", 616)
    kT, M = 0.004, 80
    Hd, Sd = s.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu = -0.1
    ref = on_pattern(density_eig(eps, C, mu, kT, M), s)
    errs = {}
    for ratio in (-1.0, 0.0, 8.0):
        rho, ne = _density(s, mu, kT, M, precision=1, split_far_ratio=ratio)
        errs[ratio] = float(np.max(np.abs(rho - ref)))
    print("split rho err by far ratio", errs)
    assert max(errs.values()) < 1e-9
    # the FP64 path ignores the option
    r0, _ = _density(s, mu, kT, M, precision=0)
    r1, _ = _density(s, mu, kT, M, precision=0, split_far_ratio=4.0)
    assert np.array_equal(r0, r1)


def test_far_pole_relaxation_leaves_selinv_alone():
    s = lattice_system((5, 5, 4), 2, "3d", 617)
    Hd, Sd = s.dense()
    Z = [0.1 + 0.02j, -0.3 + 3.0j]
    g1 = _selinv(s, Z, precision=1, split_far_ratio=2.0)
    g2 = _selinv(s, Z, precision=1, split_far_ratio=-1.0)
    assert np.array_equal(g1, g2)
    ref = on_pattern(green_dense(Hd, Sd, Z[1]), s)
    assert np.max(np.abs(g1[1] - ref)) < 1e-10 * np.max(np.abs(ref))


def test_bad_far_ratio_rejected():
    nd = lib()
    s = lattice_system((3, 3, 1), 2, "2d", 618)
    with pytest.raises(nd.NdsiError):
        nd.analyze_system(s, precision=1, split_far_ratio=0.5)


def test_fp64_peak_probe():
    _torch()
    nd = lib()
    t = nd.ndsi_fp64_peak()
    print(f"measured FP64 rate {t:.3f} TFLOP/s")
    assert 0.3 < t < 3.0
