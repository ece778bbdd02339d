"""The eigensolver's host Rayleigh-Ritz step (Eq. B3 in the span of the block) against SciPy's
generalised symmetric eigensolver, including a search space with a repeated direction."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    csrc = os.path.join(ROOT, "paper_1005_0088_gb300", "csrc")
    out = str(tmp_path_factory.mktemp("smalleig") / "small_eig_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I" + csrc, os.path.join(ROOT, "tests", "small_eig_check.cpp"),
                    os.path.join(csrc, "small_eig.cpp"), "-o", out], check=True, capture_output=True)
    return out


def _run(exe, Hs, Ss):
    m = Hs.shape[0]
    text = f"{m}\n" + " ".join(f"{v:.17g}" for v in Hs.ravel()) + "\n" + " ".join(f"{v:.17g}" for v in Ss.ravel())
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()
    r = int(out[0])
    e = np.array([float(v) for v in out[1:1 + r]])
    Y = np.array([float(v) for v in out[1 + r:1 + r + m * r]]).reshape(m, r)
    return e, Y


def _projected(rng, n, m, repeat=False):
    A = rng.normal(size=(n, n))
    H = 0.5 * (A + A.T)
    B = rng.normal(size=(n, n))
    S = B @ B.T / n + np.eye(n)
    V = rng.normal(size=(n, m))
    if repeat:
        V[:, -1] = 2.0 * V[:, 0]
    return V, H, S, V.T @ H @ V, V.T @ S @ V


@pytest.mark.parametrize("m", [2, 7, 24, 48])
def test_ritz_pairs_match_scipy(exe, m):
    rng = np.random.default_rng(m)
    V, H, S, Hs, Ss = _projected(rng, 80, m)
    e, Y = _run(exe, Hs, Ss)
    ref = scipy.linalg.eigh(Hs, Ss, eigvals_only=True)
    assert len(e) == m
    assert np.max(np.abs(np.sort(e) - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(Y.T @ Ss @ Y - np.eye(m))) < 1e-9
    assert np.max(np.abs(Hs @ Y - Ss @ Y * e[None, :])) < 1e-8 * np.max(np.abs(Hs))


def test_repeated_direction_is_dropped(exe):
    rng = np.random.default_rng(5)
    V, H, S, Hs, Ss = _projected(rng, 60, 10, repeat=True)
    e, Y = _run(exe, Hs, Ss)
    assert len(e) == 9
    Q, _ = np.linalg.qr(V[:, :-1])
    ref = scipy.linalg.eigh(Q.T @ H @ Q, Q.T @ S @ Q, eigvals_only=True)
    assert np.max(np.abs(np.sort(e) - ref)) < 1e-8 * np.max(np.abs(ref))
    assert np.max(np.abs(Y.T @ Ss @ Y - np.eye(9))) < 1e-8
