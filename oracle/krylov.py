"""Sampled columns of rho (Eq. 8) and G (Eq. 6) by Krylov solves, for systems too large for the
dense routes and for a sparse direct factorisation on the host.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For a column j, Eq. (8) gives
    rho e_j = S^{-1} e_j + sum_p w_p Re[(alpha_p S - H)^{-1} e_j],
    alpha_p = mu + i z_p kT,  w_p = -4 R_p kT,
so every sampled column needs one solve with S and one with alpha_p S - H per pole.  Each solve
is done by COCG (conjugate gradients with the bilinear form x^T y, for the complex symmetric
matrix alpha S - H; plain CG for S) in `krylov.c`, to a true relative residual below `tol`.

Error bound (no reference needed).  For Im(alpha) = y > 0 and S symmetric positive definite,
Im(x^H (alpha S - H) x) = y x^H S x >= y lambda_min(S) |x|^2, hence |(alpha S - H)^{-1}|_2 <=
1 / (y lambda_min(S)); for S alone |S^{-1}|_2 = 1 / lambda_min(S).  A solve with true residual r
is therefore within |r| / (y lambda_min(S)) of the exact column in the 2-norm (and so in every
entry), and the error of the assembled column of rho is at most
    (|r_0| + sum_p |w_p| |r_p| / y_p) / lambda_min(S).
lambda_min(S) is bounded below by Gershgorin's theorem: min_i (S_ii - sum_{j != i} |S_ij|).
`density_columns_krylov` returns this bound beside the columns.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

from .poles import cf_poles

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "krylov.c")
_BUILD = os.path.join(_HERE, "_build", platform.machine())
_LIB = os.path.join(_BUILD, "libkrylov.so")
_lib = None


def build_krylov(force: bool = False) -> str:
    """Compile krylov.c (gcc, OpenMP) into the oracle's build folder; returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        # on x86-64 the vector units of every host in use (AVX2 + FMA) are named explicitly;
        # elsewhere the compiler's baseline vector set is used
        isa = ["-mavx2", "-mfma"] if platform.machine() in ("x86_64", "AMD64") else []
        cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c99"] + isa + [_SRC, "-o", tmp, "-lm"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("building the Krylov oracle failed:\n" + " ".join(cmd) + "\n" + res.stderr)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_krylov())
        P = ctypes.c_void_p
        lib.krylov_columns.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int32, P, P, P,
                                       ctypes.c_double, ctypes.c_int64, P, P, P]
        lib.krylov_columns.restype = ctypes.c_int
        lib.krylov_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def krylov_threads() -> int:
    """OpenMP threads the solver runs on."""
    return int(_load().krylov_threads())


def solve_columns(system, alphas, gammas, cols, tol=1e-13, max_iter=200000, require_converged=True):
    """x_t = (alphas[t] S - gammas[t] H)^{-1} e_{cols[t]} for every t.

    Returns (X complex [n_tasks, n], iterations int64 [n_tasks], true relative residuals
    [n_tasks]).  Raises if a solve misses `tol` within max_iter iterations, unless
    require_converged is False (then the iterates reached are returned as they are)."""
    lib = _load()
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.complex128))
    gammas = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64))
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
    t = alphas.shape[0]
    if gammas.shape != (t,) or cols.shape != (t,):
        raise ValueError("alphas, gammas and cols must have one entry per task")
    rowptr = np.ascontiguousarray(system.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(system.col, dtype=np.int32)
    H = np.ascontiguousarray(system.H, dtype=np.float64)
    S = np.ascontiguousarray(system.S, dtype=np.float64)
    X = np.zeros((t, system.n), dtype=np.complex128)
    iters = np.zeros(t, dtype=np.int64)
    res = np.zeros(t, dtype=np.float64)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.krylov_columns(system.n, ptr(rowptr), ptr(col), ptr(H), ptr(S), t, ptr(alphas),
                            ptr(gammas), ptr(cols), float(tol), int(max_iter), ptr(X), ptr(iters),
                            ptr(res))
    if rc < 0:
        raise ValueError("krylov_columns: invalid arguments or out of memory")
    if rc > 0 and require_converged:
        raise RuntimeError(f"krylov_columns: {rc} solves missed the residual target {tol:g} "
                           f"(worst {res.max():.3e})")
    return X, iters, res


def overlap_lower_bound(system) -> float:
    """Gershgorin lower bound of lambda_min(S): min_i (S_ii - sum_{j != i} |S_ij|)."""
    rows = system.rows()
    diag = rows == system.col
    off = np.zeros(system.n)
    np.add.at(off, rows[~diag], np.abs(system.S[~diag]))
    d = np.zeros(system.n)
    d[rows[diag]] = system.S[diag]
    return float(np.min(d - off))


def density_columns_krylov(system, mu, kT, M, cols, tol=1e-13):
    """Columns rho[:, cols] by Eq. (8) with Krylov solves (M0 = S^{-1} e_j and one solve per pole).

    All (point, column) solves go to the solver in one call, hardest first (smallest Im alpha),
    so the slow poles near the real axis start at once and the fast ones fill the other slots.
    Returns (rho_cols [n, len(cols)], info) with info = {"bound": a-posteriori bound of the
    max-abs error of every returned entry, "iterations": total iterations, "max_residual":
    largest true relative residual, "lambda_min_S_lower": the Gershgorin bound used}."""
    z, R = cf_poles(M)
    lam = overlap_lower_bound(system)
    if not lam > 0:
        raise ValueError("the Gershgorin bound does not show S positive definite")
    w = -4.0 * R * kT
    nc = len(cols)
    # task (p, c): p = 0..M-1 the poles in ascending z_p (hardest first), p = M the S solve
    alphas = np.concatenate([np.repeat(mu + 1j * z * kT, nc), np.full(nc, 1.0 + 0.0j)])
    gammas = np.concatenate([np.ones(M * nc), np.zeros(nc)])
    tcols = np.tile(np.asarray(cols, dtype=np.int32), M + 1)
    X, it, res = solve_columns(system, alphas, gammas, tcols, tol=tol)
    X = X.reshape(M + 1, nc, system.n)
    res = res.reshape(M + 1, nc)
    out = X[M].real.T + np.einsum("p,pcn->nc", w, X[:M].real)
    bound = np.max((res[M] + np.sum((np.abs(w) / (z * kT))[:, None] * res[:M], axis=0)) / lam)
    return out, {"bound": float(bound), "iterations": int(it.sum()), "max_residual": float(res.max()),
                 "lambda_min_S_lower": lam}


def green_columns_krylov(system, Z, cols, tol=1e-13):
    """Columns G(Z)[:, cols] = (Z S - H)^{-1} e_j (Eq. 6) by COCG, Im Z != 0."""
    X, _, _ = solve_columns(system, np.full(len(cols), Z, dtype=np.complex128),
                            np.ones(len(cols)), cols, tol=tol)
    return X.T
