"""Batched plans: several uneven systems (own mu and kT) in one launch per tree level."""
import numpy as np
import pytest

from synth import lattice_system
from oracle.dense import generalized_eig, density_eig, on_pattern, electron_count_pattern
from tests.libtools import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-9)])
def test_batched_density_matches_single_and_oracle(precision, tol):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nd = lib()
    systems = [lattice_system((60, 1, 1), 3, "1d", 11), lattice_system((9, 8, 1), 2, "2d", 12),
               lattice_system((5, 4, 4), 2, "3d", 13)]
    mus = [-0.2, 0.05, 0.1]
    kTs = [0.01, 0.02, 0.015]
    M = 40
    plan = nd.analyze_batched(systems, precision=precision)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device="cuda")
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device="cuda")
    nnz = sum(s.nnz for s in systems)
    rho = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(3, dtype=torch.float64, device="cuda")
    nd.ndsi_density_batched(plan, H, S, mus, kTs, M, rho, ne)
    torch.cuda.synchronize()
    rho = rho.cpu().numpy()
    ne = ne.cpu().numpy()
    off = 0
    for i, sy in enumerate(systems):
        r_b = rho[off:off + sy.nnz]
        off += sy.nnz
        p1 = nd.analyze_system(sy, precision=precision)
        r1 = torch.zeros(sy.nnz, dtype=torch.float64, device="cuda")
        n1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        nd.ndsi_density(p1, torch.as_tensor(sy.H, device="cuda"), torch.as_tensor(sy.S, device="cuda"),
                        mus[i], kTs[i], M, r1, n1)
        assert np.max(np.abs(r_b - r1.cpu().numpy())) < 1e-13
        Hd, Sd = sy.dense()
        eps, C = generalized_eig(Hd, Sd)
        ref = on_pattern(density_eig(eps, C, mus[i], kTs[i], M), sy)
        assert np.max(np.abs(r_b - ref)) < tol
        assert abs(ne[i] - electron_count_pattern(r_b, sy)) < 1e-9


def test_find_mu_batched_lockstep():
    # every system's mu from one lockstep search over the batched plan (Eq. 40 per system)
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.dense import generalized_eig, find_mu_eig, electron_count_eig
    nd = lib()
    systems = [lattice_system((8, 7, 1), 2, "2d", seed=61), lattice_system((30, 1, 1), 3, "1d", seed=62),
               lattice_system((4, 4, 3), 2, "3d", seed=63)]
    kT = np.array([0.01, 0.02, 0.01])
    ne = np.array([s.n_electrons * f for s, f in zip(systems, (1.0, 0.8, 1.2))])
    M = 40
    plan = nd.analyze_batched(systems)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device="cuda")
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device="cuda")
    rho = torch.zeros(H.numel(), dtype=torch.float64, device="cuda")
    mu, n_e, rounds = nd.ndsi_find_mu_batched(plan, H, S, kT, M, ne, rho)
    singles = []
    for i, s in enumerate(systems):
        eps, _ = generalized_eig(*s.dense())
        assert abs(n_e[i] - ne[i]) < 1e-8
        assert abs(electron_count_eig(eps, mu[i], kT[i], M) - ne[i]) < 1e-7
        p1 = nd.analyze_system(s)
        r1 = torch.zeros(s.nnz, dtype=torch.float64, device="cuda")
        _, _, it = nd.ndsi_find_mu(p1, torch.as_tensor(s.H, device="cuda"), torch.as_tensor(s.S, device="cuda"),
                                   kT[i], M, ne[i], r1)
        singles.append(it)
    print(f"find_mu_batched: {rounds} batched sweeps; single searches {singles}")
    assert rounds <= max(singles) + 2 and rounds < sum(singles)
    # rho_out is the batched density at the returned chemical potentials
    rho2 = torch.zeros_like(rho)
    ne2 = torch.zeros(len(systems), dtype=torch.float64, device="cuda")
    nd.ndsi_density_batched(plan, H, S, mu, kT, M, rho2, ne2)
    torch.cuda.synchronize()
    assert torch.equal(rho, rho2)


def test_find_mu_batched_with_brackets_and_host_rho():
    # brackets per system (one of them wrong, so that system widens it) and a host rho buffer
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle.dense import generalized_eig, find_mu_eig, electron_count_eig
    nd = lib()
    systems = [lattice_system((7, 6, 1), 2, "2d", seed=64), lattice_system((24, 1, 1), 2, "1d", seed=65)]
    kT = np.array([0.01, 0.01])
    ne = np.array([s.n_electrons for s in systems])
    M = 40
    eps = [generalized_eig(*s.dense())[0] for s in systems]
    ref = [find_mu_eig(e, k, n, M) for e, k, n in zip(eps, kT, ne)]
    lo = np.array([ref[0] - 0.05, ref[1] + 0.2])
    hi = np.array([ref[0] + 0.05, ref[1] + 0.3])
    plan = nd.analyze_batched(systems)
    H = np.concatenate([s.H for s in systems])
    S = np.concatenate([s.S for s in systems])
    rho = np.zeros(H.size)
    mu, n_e, rounds = nd.ndsi_find_mu_batched(plan, H, S, kT, M, ne, rho, mu_lo=lo, mu_hi=hi)
    assert np.all(np.abs(n_e - ne) < 1e-8)
    for e, m, k, n in zip(eps, mu, kT, ne):
        assert abs(electron_count_eig(e, m, k, M) - n) < 1e-7
    rho2 = np.zeros_like(rho)
    nd.ndsi_density_batched(plan, H, S, mu, kT, M, rho2)
    assert np.array_equal(rho, rho2)


def test_batched_workload_electron_counts_match_oracle():
    # Tr(rho S) (Eq. 40) of the batched workload's systems (split path, 120 poles) against the
    # oracle's eigenvalue counts stored by tests/golden/make_c4_electron_counts.py
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth import batched_systems
    from tests.conftest import golden_lines
    nd = lib()
    systems = batched_systems()
    ref = {int(l.split()[0]): float(l.split()[2]) for l in golden_lines("c4_electron_counts.txt")}
    plan = nd.analyze_batched(systems, precision=1)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device="cuda")
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device="cuda")
    rho = torch.zeros(H.numel(), dtype=torch.float64, device="cuda")
    ne = torch.zeros(len(systems), dtype=torch.float64, device="cuda")
    nd.ndsi_density_batched(plan, H, S, np.full(len(systems), -0.12), np.full(len(systems), 0.01), 120, rho, ne)
    torch.cuda.synchronize()
    got = ne.cpu().numpy()
    for i, v in ref.items():
        assert abs(got[i] - v) < 1e-9, (i, got[i], v)
