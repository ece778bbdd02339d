"""The allocation-free residue sum (ndsi_residue_sum_static) against ndsi_density.

ndsi_residue_sum_static serves callers that cannot allocate device memory (a host framework
owning the whole device budget, or a latency-critical path that must not call cudaMalloc or
cudaFree).  It keeps its partial traces in a fixed file-scope device array; this test feeds it
G from ndsi_selinv and checks rho and Tr(rho S) against the allocating path (ndsi_density),
on two calls in a row, so a wrong symbol address or stale array contents would show.
This file is collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from synth import lattice_system
from tests.libtools import lib

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_static_residue_sum_matches_density():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nd = lib()
    sysm = lattice_system((12, 11, 1), 3, "2d", 4242)
    mu, kT, M = -0.08, 0.01, 40
    plan = nd.analyze_system(sysm)
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    # reference: the allocating path
    rho_ref = torch.zeros(sysm.nnz, dtype=torch.float64, device="cuda")
    ne_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density(plan, H, S, mu, kT, M, rho_ref, ne_ref)
    # the same points and weights: alpha_p = mu + i z_p kT, w_p = -4 R_p kT, and iR with weight iR
    z, R = nd.ndsi_poles(M)
    Rm0 = nd.ndsi_default_options().m0_radius
    pts = np.concatenate([mu + 1j * z * kT, [1j * Rm0]])
    wts = np.concatenate([-4.0 * R * kT + 0j, [1j * Rm0]])
    f = nd.ndsi_factor_poles(plan, H, S, pts)
    G = torch.zeros((len(pts), sysm.nnz, 2), dtype=torch.float64, device="cuda")
    nd.ndsi_selinv(f, G)
    c = torch.as_tensor(np.ascontiguousarray(wts.view(np.float64)), device="cuda")
    ref = rho_ref.cpu().numpy()
    for _ in range(2):
        rho = torch.full((sysm.nnz,), float("nan"), dtype=torch.float64, device="cuda")
        ne = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        nd.ndsi_residue_sum_static(G, c, len(pts), S, sysm.nnz, rho, ne)
        torch.cuda.synchronize()
        assert np.max(np.abs(rho.cpu().numpy() - ref)) < TOL
        assert abs(float(ne.cpu()[0]) - float(ne_ref.cpu()[0])) < TOL * sysm.n
    # without the trace (the reduction launch is skipped), on a caller stream
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        rho = torch.full((sysm.nnz,), float("nan"), dtype=torch.float64, device="cuda")
    nd.ndsi_residue_sum_static(G, c, len(pts), S, sysm.nnz, rho, None, stream=st)
    st.synchronize()
    assert np.max(np.abs(rho.cpu().numpy() - ref)) < TOL


def test_static_residue_sum_rejects_oversize_and_host():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nd = lib()
    G = torch.zeros(4, dtype=torch.float64, device="cuda")
    c = torch.zeros(2, dtype=torch.float64, device="cuda")
    S = torch.zeros(2, dtype=torch.float64, device="cuda")
    rho = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(nd.NdsiError) as ei:
        nd.ndsi_residue_sum_static(G, c, 1, S, 8_388_609, rho)
    assert ei.value.code == nd.ndsi.NDSI_ERR_INVALID and "static scratch limit" in str(ei.value)
    with pytest.raises(nd.NdsiError):
        nd.ndsi_residue_sum_static(G.cpu(), c, 1, S, 2, rho)
    # G and c are read as 16-byte complex pairs: a view one double in is refused before any launch
    Gw = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(nd.NdsiError) as ei:
        nd.ndsi_residue_sum_static(Gw[1:5], c, 1, S, 2, rho)
    assert ei.value.code == nd.ndsi.NDSI_ERR_INVALID and "aligned" in str(ei.value)
    cw = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(nd.NdsiError):
        nd.ndsi_residue_sum_static(G, cw[1:3], 1, S, 2, rho)
