"""The paper's recurrence formulas for selected inversion on a structured matrix.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. II.C.2 in its own notation, for a structured matrix whose dissection tree is a
perfect binary tree with P+1 separator levels and 2^{P+1} innermost domains:
  X_{0,n} = A_{0,n} (innermost domains), X_{p+1,n} = [X_{p,2n}, X_{p,2n+1}, C_{p,n}] (Eq. 22),
  B_{p,m} couples separator C_{p, m//2} to domain X_{p,m}; B_{p,q}[Y] is the part of B_{p,q}
  with the columns of block Y (the bra-ket notation of Eqs. 25-27).
Factor (Eqs. 28-32), p = 0..P, m = 0..p-1 (Eqs. 33-37):
  V^T_{p,0,n}   = A_{0,n}^{-1} (B_{p,q}[B_{0,n}])^T                                   (30)
  Q^T_{p,m+1,n} = S_{m,n}^{-1} (B_{m,2n} V^T_{p,m,2n} + B_{m,2n+1} V^T_{p,m,2n+1}
                                 - (B_{p,q}[C_{m,n}])^T)                              (28)
  V^T_{p,m+1,n} = [V^T_{p,m,2n}; V^T_{p,m,2n+1}; 0] + [L^T_{m,2n}; L^T_{m,2n+1}; -I] Q^T (29)
  L_{p,q} = V_{p,p,q}                                                                  (31)
  S_{p,n} = C_{p,n} - B_{p,2n} L^T_{p,2n} - B_{p,2n+1} L^T_{p,2n+1}                   (32)
Inverse (Eqs. 38-39): X^{-1}_{0,n} = A_{0,n}^{-1};
  X^{-1}_{p+1,n} = diag(X^{-1}_{p,2n}, X^{-1}_{p,2n+1}, 0)
                   + [[Y^T_{p,2n} L_{p,2n}, ., -Y^T_{p,2n}], [., Y^T_{p,2n+1} L_{p,2n+1}, -Y^T_{p,2n+1}],
                      [-Y_{p,2n}, -Y_{p,2n+1}, S^{-1}_{p,n}]],   Y^T_{p,m} = L^T_{p,m} S^{-1}_{p,m//2}.
Only these blocks are formed; the cross blocks between X_{p,2n} and X_{p,2n+1} are not
(they hold no selected element), and are returned as NaN.  S^{-1} is formed by dense LU.
"""
from __future__ import annotations

import numpy as np


def perfect_layout(P, leaf_sizes, sep_sizes):
    """Index sets of the structured order for a perfect tree.

    leaf_sizes: 2^{P+1} sizes of A_{0,n}; sep_sizes[p]: 2^{P-p} sizes of C_{p,n}.
    Returns (dom, sep): dom[p][n] index arrays of X_{p,n} (p = 0..P+1), sep[p][n] of C_{p,n}.
    """
    dom = {0: {}}
    sep = {}
    pos = 0

    def build(p, n):
        nonlocal pos
        if p == 0:
            idx = np.arange(pos, pos + leaf_sizes[n])
            pos += leaf_sizes[n]
            dom[0][n] = idx
            return idx
        left = build(p - 1, 2 * n)
        right = build(p - 1, 2 * n + 1)
        s = np.arange(pos, pos + sep_sizes[p - 1][n])
        pos += sep_sizes[p - 1][n]
        sep.setdefault(p - 1, {})[n] = s
        dom.setdefault(p, {})[n] = np.concatenate([left, right, s])
        return dom[p][n]

    build(P + 1, 0)
    return dom, sep


def recurrence_selected_inverse(X, P, dom, sep, record=None):
    """Run Eqs. (28)-(32) then (38)-(39); returns X^{-1}_{P+1,0} with unformed blocks NaN.

    record: optional dict that receives the intermediates keyed like the paper
    ('V', p, m, n), ('Q', p, m, n), ('L', p, n), ('S', p, n).
    """
    X = np.asarray(X)
    dt = np.result_type(X.dtype, np.float64)
    rec = {} if record is None else record

    def blk(r, c):
        return X[np.ix_(r, c)]

    Ainv = {n: np.linalg.inv(blk(dom[0][n], dom[0][n])) for n in dom[0]}
    L, S, Sinv = {}, {}, {}
    for p in range(P + 1):
        for q in range(2 ** (P + 1 - p)):
            rows_C = sep[p][q // 2]                 # separator coupled by B_{p,q}
            V = {}
            for n in range(q * 2 ** p, (q + 1) * 2 ** p):          # Eqs. (30), (36)
                V[n] = Ainv[n] @ blk(rows_C, dom[0][n]).T
                rec[("V", p, 0, n)] = V[n]
            for m in range(p):                                      # Eqs. (28), (29)
                Vn = {}
                for n in range(q * 2 ** (p - m - 1), (q + 1) * 2 ** (p - m - 1)):
                    Bl = blk(sep[m][n], dom[m][2 * n])
                    Br = blk(sep[m][n], dom[m][2 * n + 1])
                    Qt = Sinv[(m, n)] @ (Bl @ V[2 * n] + Br @ V[2 * n + 1]
                                         - blk(rows_C, sep[m][n]).T)
                    rec[("Q", p, m + 1, n)] = Qt
                    ncols = Qt.shape[1]
                    top = np.concatenate([V[2 * n], V[2 * n + 1],
                                          np.zeros((len(sep[m][n]), ncols), dtype=dt)])
                    coef = np.concatenate([L[(m, 2 * n)].T, L[(m, 2 * n + 1)].T,
                                           -np.eye(len(sep[m][n]), dtype=dt)])
                    Vn[n] = top + coef @ Qt
                    rec[("V", p, m + 1, n)] = Vn[n]
                V = Vn
            L[(p, q)] = V[q].T                                     # Eq. (31)
            rec[("L", p, q)] = L[(p, q)]
        for n in range(2 ** (P - p)):                               # Eq. (32)
            S[(p, n)] = (blk(sep[p][n], sep[p][n])
                         - blk(sep[p][n], dom[p][2 * n]) @ L[(p, 2 * n)].T
                         - blk(sep[p][n], dom[p][2 * n + 1]) @ L[(p, 2 * n + 1)].T)
            Sinv[(p, n)] = np.linalg.inv(S[(p, n)])
            rec[("S", p, n)] = S[(p, n)]
    # Eqs. (38), (39)
    Xinv = {(0, n): Ainv[n] for n in dom[0]}
    for p in range(P + 1):
        for n in range(2 ** (P - p)):
            dl, dr, s = dom[p][2 * n], dom[p][2 * n + 1], sep[p][n]
            size = len(dl) + len(dr) + len(s)
            out = np.full((size, size), np.nan, dtype=dt)
            a, b = len(dl), len(dl) + len(dr)
            YlT = L[(p, 2 * n)].T @ Sinv[(p, n)]
            YrT = L[(p, 2 * n + 1)].T @ Sinv[(p, n)]
            out[:a, :a] = Xinv[(p, 2 * n)] + YlT @ L[(p, 2 * n)]
            out[a:b, a:b] = Xinv[(p, 2 * n + 1)] + YrT @ L[(p, 2 * n + 1)]
            out[:a, b:] = -YlT
            out[a:b, b:] = -YrT
            out[b:, :a] = -YlT.T
            out[b:, a:b] = -YrT.T
            out[b:, b:] = Sinv[(p, n)]
            Xinv[(p + 1, n)] = out
    return Xinv[(P + 1, 0)]
