"""CUDA-graph replay of the density sweep: identical results to direct launches.

The captured graph must reproduce the eager launch sequence bit for bit, must be replayed (not
recaptured) when only mu changes, must be recaptured when an output buffer moves, and must stay
out of the way while profiling is on.  Both precision forms and a batched plan are covered.
"""
import numpy as np
import pytest

from synth import lattice_system, batched_systems
from tests.libtools import lib

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(nd, torch, plan, H, S, mu, kT, M, nnz):
    rho = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density(plan, H, S, mu, kT, M, rho, ne)
    torch.cuda.synchronize()
    return rho.cpu().numpy(), float(ne.cpu()[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_matches_direct_launches(precision):
    torch = _torch()
    nd = lib()
    sysm = lattice_system((9, 7, 1), 4, "2d", seed=31)
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    plan_g = nd.analyze_system(sysm, precision=precision)
    plan_d = nd.analyze_system(sysm, precision=precision)
    nd.ndsi_graph_enable(plan_d, False)
    for mu in (-0.2, 0.15):
        rg, ng = _run(nd, torch, plan_g, H, S, mu, 0.01, 24, sysm.nnz)
        rd, ndd = _run(nd, torch, plan_d, H, S, mu, 0.01, 24, sysm.nnz)
        assert np.array_equal(rg, rd) and ng == ndd
    assert nd.ndsi_graph_info(plan_g) > 0
    assert nd.ndsi_graph_info(plan_d) == 0


def test_graph_replays_and_recaptures():
    torch = _torch()
    nd = lib()
    sysm = lattice_system((6, 6, 1), 4, "2d", seed=32)
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    plan = nd.analyze_system(sysm)
    rho = torch.zeros(sysm.nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density(plan, H, S, 0.0, 0.01, 16, rho, ne)
    n0 = nd.ndsi_graph_info(plan)
    first = rho.clone()
    nd.ndsi_density(plan, H, S, 0.3, 0.01, 16, rho, ne)      # new mu: replay
    assert nd.ndsi_graph_info(plan) == n0
    assert not torch.equal(first, rho)
    rho2 = torch.zeros_like(rho)
    nd.ndsi_density(plan, H, S, 0.0, 0.01, 16, rho2, ne)     # new output buffer: recapture
    torch.cuda.synchronize()
    assert torch.equal(first, rho2)
    # profiling forces direct launches (per-kernel events) and still gives the same result
    nd.ndsi_profile_enable(plan, True)
    rho3 = torch.zeros_like(rho)
    nd.ndsi_density(plan, H, S, 0.0, 0.01, 16, rho3, ne)
    torch.cuda.synchronize()
    prof = nd.ndsi_profile_read(plan)
    nd.ndsi_profile_enable(plan, False)
    assert torch.equal(first, rho3)
    assert sum(v["launches"] for v in prof.values()) > 0


def test_graph_batched_plan():
    torch = _torch()
    nd = lib()
    systems = [lattice_system((10, 1, 1), 4, "1d", seed=40), lattice_system((5, 4, 1), 4, "2d", seed=41)]
    plans = []
    for graphs in (True, False):
        p = nd.analyze_batched(systems)
        nd.ndsi_graph_enable(p, graphs)
        plans.append(p)
    H = torch.as_tensor(np.concatenate([s.H for s in systems]), device="cuda")
    S = torch.as_tensor(np.concatenate([s.S for s in systems]), device="cuda")
    mu = np.array([-0.1, 0.05])
    kT = np.array([0.01, 0.02])
    out = []
    for p in plans:
        rho = torch.zeros(H.numel(), dtype=torch.float64, device="cuda")
        ne = torch.zeros(2, dtype=torch.float64, device="cuda")
        nd.ndsi_density_batched(p, H, S, mu, kT, 20, rho, ne)
        torch.cuda.synchronize()
        out.append((rho.cpu().numpy(), ne.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
