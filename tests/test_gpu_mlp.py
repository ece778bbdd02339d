"""GPU kernels of the learned mu seed against the FP64 oracle, and what the seed gains."""
import numpy as np
import pytest

from synth import lattice_system, mu_training_systems
from oracle import mlp as omlp
from oracle.dense import generalized_eig
from tests.libtools import lib

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_mlp_forward_and_gradient_match_oracle():
    torch = _torch()
    nd = lib()
    P = torch.zeros(nd.NDSI_MLP_PARAMS, dtype=torch.float32, device="cuda")
    nd.ndsi_mlp_init(P, 3)
    rng = np.random.default_rng(4)
    n = 150
    X = rng.normal(0, 1, (n, 32)).astype(np.float32)
    T = rng.normal(0, 0.5, n).astype(np.float32)
    Xd = torch.as_tensor(X, device="cuda")
    Td = torch.as_tensor(T, device="cuda")
    Y = torch.zeros(n, dtype=torch.float32, device="cuda")
    nd.ndsi_mlp_forward(P, Xd, n, Y)
    G = torch.zeros(nd.NDSI_MLP_PARAMS, dtype=torch.float32, device="cuda")
    L = torch.zeros(1, dtype=torch.float32, device="cuda")
    nd.ndsi_mlp_grad(P, Xd, Td, n, G, L)
    theta = P.cpu().numpy().astype(np.float64)
    y_ref, _ = omlp.forward(theta, X.astype(np.float64))
    g_ref = omlp.grad(theta, X.astype(np.float64), T.astype(np.float64))
    assert np.max(np.abs(Y.cpu().numpy() - y_ref)) < 1e-5 * max(1.0, np.max(np.abs(y_ref)))
    g = G.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) < 1e-5 * np.linalg.norm(g_ref)
    # element by element: each gradient entry is a sum over the samples, so its FP32 rounding
    # scales with the sum of the per-sample magnitudes (a small entry that is a cancellation of
    # large per-sample terms may differ by more than 1e-5 of itself, but not of that sum)
    scale = np.zeros_like(g_ref)
    for s_ in range(n):
        scale += np.abs(omlp.grad(theta, X[s_:s_ + 1].astype(np.float64), T[s_:s_ + 1].astype(np.float64))) / n
    bad = np.abs(g - g_ref) > 1e-5 * (np.abs(g_ref) + scale) + 1e-12
    assert not bad.any(), (np.nonzero(bad)[0][:10], g[bad][:5], g_ref[bad][:5])
    # every block of the parameter vector (including b3 and the W3 row) is exercised
    off = 0
    for name, shape in omlp.SIZES:
        k = int(np.prod(shape))
        assert np.max(np.abs(g_ref[off:off + k])) > 0, name
        off += k
    assert abs(float(L.cpu()[0]) - omlp.loss(theta, X, T)) < 1e-5 * omlp.loss(theta, X, T)


def test_features_match_exact_moments():
    torch = _torch()
    nd = lib()
    sysm = lattice_system((6, 6, 2), 4, "3d", 17)
    plan = nd.analyze_system(sysm)
    H = torch.as_tensor(sysm.H, device="cuda")
    S = torch.as_tensor(sysm.S, device="cuda")
    R = 64
    f = np.zeros(32, dtype=np.float32)
    nd.ndsi_mu_features(plan, H, S, sysm.n_electrons, 0.01, f, n_vectors=R, seed=99)
    Hd, Sd = sysm.dense()
    lh = np.linalg.eigvalsh(Hd) / 4.0
    ls = (np.linalg.eigvalsh(Sd) - 1.0) / 0.75
    exact_h = [np.mean(np.cos(k * np.arccos(np.clip(lh, -1, 1)))) for k in range(1, 25)]
    exact_s = [np.mean(np.cos(k * np.arccos(np.clip(ls, -1, 1)))) for k in range(1, 7)]
    bound = 6.0 * np.sqrt(2.0 / (R * sysm.n))   # stochastic-trace standard error x 6
    assert np.max(np.abs(f[:24] - exact_h)) < bound
    assert np.max(np.abs(f[24:30] - exact_s)) < bound
    assert abs(f[30] - sysm.n_electrons / (2 * sysm.n)) < 1e-6 and abs(f[31] - 0.1) < 1e-6


def test_seed_saves_mu_search_evaluations():
    torch = _torch()
    from paper_1005_0088_gb300.mu_seed import MuSeed, build_dataset, features
    nd = lib()
    train = mu_training_systems(240, 1)
    test = mu_training_systems(16, 2)
    X, T = build_dataset(train)
    model = MuSeed(seed=5)
    loss = model.train(X, T, steps=3000, lr=3e-3)
    it_plain, it_seed = [], []
    for sysm, kT in test:
        plan = nd.analyze_system(sysm)
        H = torch.as_tensor(sysm.H, device="cuda")
        S = torch.as_tensor(sysm.S, device="cuda")
        rho = torch.zeros(sysm.nnz, dtype=torch.float64, device="cuda")
        mu0, ne0, i0 = nd.ndsi_find_mu(plan, H, S, kT, 80, sysm.n_electrons, rho)
        lo, hi = model.bracket(features(plan, H, S, sysm.n_electrons, kT))
        mu1, ne1, i1 = nd.ndsi_find_mu(plan, H, S, kT, 80, sysm.n_electrons, rho, mu_lo=lo, mu_hi=hi)
        assert abs(ne0 - sysm.n_electrons) < 1e-8 and abs(ne1 - sysm.n_electrons) < 1e-8
        it_plain.append(i0)
        it_seed.append(i1)
    print(f"mu seed: train rmse {model.rmse:.3e}; evaluations plain {np.mean(it_plain):.1f}, "
          f"seeded {np.mean(it_seed):.1f}")
    assert np.mean(it_seed) < np.mean(it_plain)
