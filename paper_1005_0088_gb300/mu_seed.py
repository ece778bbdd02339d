"""Learned seed for the chemical-potential search (ndsi_find_mu).

The paper finds mu by iterating exact contour evaluations (Sec. II.C.3).  This module trains the
library's small network (ndsi_mlp_*) on mu values produced by that exact search, then uses its
prediction only to propose the starting bracket; ndsi_find_mu still verifies and widens it, so a
poor prediction costs evaluations but never accuracy.  Every step runs in libndsi.so; torch
holds the device buffers.
"""
from __future__ import annotations

import numpy as np

from . import ndsi as _nd


def _torch():
    import torch
    return torch


def features(plan, H, S, n_electrons, kT, n_vectors=16, seed=12345):
    """The 32 input features of a system (see ndsi_mu_features), as a host float32 array."""
    out = np.zeros(_nd.NDSI_MLP_INPUTS, dtype=np.float32)
    _nd.ndsi_mu_features(plan, H, S, n_electrons, kT, out, n_vectors=n_vectors, seed=seed)
    return out


def exact_mu(system, kT, n_poles=80, tol=1e-8, device="cuda", precision=_nd.NDSI_PREC_FP64):
    """(features, mu, evaluations) of one system, mu from the exact contour search."""
    torch = _torch()
    plan = _nd.analyze_system(system, precision=precision)
    H = torch.as_tensor(system.H, device=device)
    S = torch.as_tensor(system.S, device=device)
    rho = torch.zeros(system.nnz, dtype=torch.float64, device=device)
    f = features(plan, H, S, system.n_electrons, kT)
    mu, _, it = _nd.ndsi_find_mu(plan, H, S, kT, n_poles, system.n_electrons, rho,
                                 tol_electrons=tol)
    return f, mu, it


def build_dataset(pairs, n_poles=80):
    """Features X (n x 32) and exact mu T (n) for (System, kT) pairs."""
    X = np.zeros((len(pairs), _nd.NDSI_MLP_INPUTS), dtype=np.float32)
    T = np.zeros(len(pairs), dtype=np.float32)
    for i, (sysm, kT) in enumerate(pairs):
        X[i], T[i], _ = exact_mu(sysm, kT, n_poles)
    return X, T


class MuSeed:
    """The trained network on one device."""

    def __init__(self, seed=7, device="cuda"):
        torch = _torch()
        self.device = device
        self.params = torch.zeros(_nd.NDSI_MLP_PARAMS, dtype=torch.float32, device=device)
        _nd.ndsi_mlp_init(self.params, seed)
        self.rmse = None

    def train(self, X, T, steps=3000, lr=3e-3):
        torch = _torch()
        Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device=self.device)
        Td = torch.as_tensor(np.ascontiguousarray(T, dtype=np.float32), device=self.device)
        loss = _nd.ndsi_mlp_train(self.params, Xd, Td, len(T), steps, lr)
        self.rmse = float(np.sqrt(max(loss, 0.0)))
        return loss

    def predict(self, X):
        torch = _torch()
        X = np.atleast_2d(np.asarray(X, dtype=np.float32))
        Xd = torch.as_tensor(np.ascontiguousarray(X), device=self.device)
        Y = torch.zeros(X.shape[0], dtype=torch.float32, device=self.device)
        _nd.ndsi_mlp_forward(self.params, Xd, X.shape[0], Y)
        torch.cuda.synchronize()
        return Y.cpu().numpy().astype(np.float64)

    def bracket(self, feat, width=None):
        """(mu_lo, mu_hi) around the prediction; half-width = 3 x training RMSE by default."""
        mu = float(self.predict(feat)[0])
        w = width if width is not None else 3.0 * max(self.rmse or 0.05, 1e-3)
        return mu - w, mu + w
