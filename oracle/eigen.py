"""Selected eigenstates near an energy xi, and the three-step solve they need (App. B).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definition: the eigenpairs (eps_nu, c_nu) of H c = eps S c (Eq. 2) with the n smallest
|eps_nu - xi|, c S-orthonormal, by LAPACK on dense matrices (`eigenstates_near`).

The paper's route (App. B): block shift-invert iteration
    b_l = (H - xi S)^{-1} S c_l                                                    (B2)
    <b_l|H|b_l> c_{l+1} = <b_l|S|b_l> c_{l+1} eps_{l+1}                          (B3)
where the product with (H - xi S)^{-1} uses the factorisation X = L_P ... L_0 D L_0^T ... L_P^T
of the recurrence (Eqs. 28-32) in three steps: y' = L_0^{-1} ... L_P^{-1} y (B8, B9),
y'' = D^{-1} y' (B10, B11) and x = (L_P^T)^{-1} ... (L_0^T)^{-1} y'' (B12-B15).  Each L_p^{-1}
is I minus the off-diagonal blocks L_{p,q}, so every step reads only values that earlier steps
have not changed (`three_step_solve`, on the perfect-tree structured matrices of
`oracle.recurrence`).  `block_shift_invert` runs (B2)-(B3) with any solve; (B3) is solved in the
span of the block's vectors by a dense generalised eigensolver.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .recurrence import recurrence_selected_inverse


def eigenstates_near(Hd, Sd, xi, n):
    """(eps, C): the n eigenpairs of H c = eps S c nearest xi, ascending in eps, c^T S c = I."""
    eps, C = scipy.linalg.eigh(Hd, Sd)
    pick = np.sort(np.argsort(np.abs(eps - xi), kind="stable")[:n])
    return eps[pick], C[:, pick]


def three_step_solve(X, P, dom, sep, y):
    """X^{-1} y by (B8)-(B15) with the factors of Eqs. (28)-(32) (y: vector or columns)."""
    rec = {}
    recurrence_selected_inverse(X, P, dom, sep, rec)
    y = np.asarray(y)
    dt = np.result_type(X.dtype, y.dtype, np.float64)
    y = y.astype(dt).reshape(y.shape[0], -1)
    L = {(k[1], k[2]): v for k, v in rec.items() if k[0] == "L"}
    S = {(k[1], k[2]): v for k, v in rec.items() if k[0] == "S"}
    # (i) (B8), (B9): separator rows minus L_{p,2n} y[X_{p,2n}] + L_{p,2n+1} y[X_{p,2n+1}], all
    # read from the unmodified y
    y1 = y.copy()
    for p in range(P + 1):
        for n in range(2 ** (P - p)):
            c = sep[p][n]
            y1[c] = (y[c] - L[(p, 2 * n)] @ y[dom[p][2 * n]] - L[(p, 2 * n + 1)] @ y[dom[p][2 * n + 1]])
    # (ii) (B10), (B11): block-diagonal solves with S_{p,n} and A_{0,n}
    y2 = np.empty_like(y1)
    for p in range(P + 1):
        for n in range(2 ** (P - p)):
            c = sep[p][n]
            y2[c] = np.linalg.solve(S[(p, n)], y1[c])
    for n in dom[0]:
        a = dom[0][n]
        y2[a] = np.linalg.solve(X[np.ix_(a, a)], y1[a])
    # (iii) (B12)-(B14): level by level from the innermost separators up, domain rows minus
    # L_{p,q}^T x[C_{p,q//2}]
    x = y2
    for p in range(P + 1):
        xn = x.copy()
        for q in range(2 ** (P + 1 - p)):
            d, c = dom[p][q], sep[p][q // 2]
            xn[d] = x[d] - L[(p, q)].T @ x[c]
        x = xn
    return x                                                                     # (B15)


def block_shift_invert(Hd, Sd, xi, C0, n_iter, solve=None):
    """(B2)-(B3) from the starting block C0 (N x m); returns (eps, C) after n_iter steps.

    solve(y) must return (H - xi S)^{-1} y; dense LU by default."""
    if solve is None:
        lu = scipy.linalg.lu_factor(Hd - xi * Sd)
        solve = lambda y: scipy.linalg.lu_solve(lu, y)  # noqa: E731
    C = np.array(C0, dtype=np.float64)
    eps = None
    for _ in range(n_iter):
        b = solve(Sd @ C)                                                        # (B2)
        Hb, Sb = b.T @ Hd @ b, b.T @ Sd @ b
        eps, W = scipy.linalg.eigh(0.5 * (Hb + Hb.T), 0.5 * (Sb + Sb.T))         # (B3)
        C = b @ W
    return eps, C
