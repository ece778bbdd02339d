"""Geometric nested dissection of Sec. II.C.1, steps (i)-(v), and the symbolic fill.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  An independent, plain-Python statement
of the ordering rules, compared bit for bit with the library's host analysis.

Granularity is the atom (the orbitals of an atom stay together).  Two atoms are adjacent when
H or S has a nonzero block between them.  For a domain D of N_d atoms:
 (i)   for each axis a_i (i = 0, 1, 2) number the atoms 1..N_d by (coordinate_i, atom index);
 (ii)  long-tail screening (optional, screen_degree > 0): atoms adjacent to more than
       screen_degree atoms are taken out of the dissection and placed in the root separator
       (read from the paper's rule that long-tail basis functions join the separator before the
       domain is dissected; the pattern's degree stands for the tail length);
 (iii) the nucleus is the atom with the fewest adjacent atoms inside the domain, ties broken by
       the lowest ordering number (this reproduces App. A's intermediates and Fig. 1's text);
 (iv)  grow the subdomain [m_min, m_max] one atom per step, taking the end whose growth gives
       the smaller measure |N0 - N1| + Ns (ties: extend m_max); n_min/n_max are the lowest and
       highest ordering numbers among domain atoms adjacent to, or inside, the subdomain;
       N0 = m_max - m_min + 1, Ns = n_max - n_min + 1 - N0, N1 = N_d - N0 - Ns.  Every state
       with N1 >= 1 (the initial one included) is a candidate; the best has the smallest
       (measure, Ns), ties going to the later step (Fig. 1: a 10-atom chain splits 5 | 1 | 4);
 (v)   the axis with the smallest (measure, Ns) wins, ties to the lowest axis.  Subdomain 0 =
       ordering numbers [m_min, m_max], separator = [n_min, n_max] minus subdomain 0,
       subdomain 1 = the rest.  Domains of <= leaf_atoms atoms, or without a candidate, are
       leaves.  The structured order is [subdomain 0, subdomain 1, separator] recursively;
       atoms inside a leaf or a separator are listed by ascending atom index.
Periodic axes (cell length L > 0 along the axis): coordinates are wrapped into [0, L) for the
ordering, and a neighbour b of atom a is seen at its image nearest a, image shift
l = -floor((x_b - x_a)/L + 1/2) of the wrapped coordinates, with ordering number
ord(b) + l N_d (step (i)'s numbering of the periodic cells); n_min can then be below 1 and
n_max above N_d, and the separator is [n_min, n_max] minus subdomain 0 taken modulo N_d.
"""
from __future__ import annotations

import math

import numpy as np


def atom_adjacency(system):
    """Sorted neighbour-atom lists (self excluded) from the CSR pattern of H and S."""
    aob = system.atom_of_basis
    rows = system.rows()
    ai = aob[rows].astype(np.int64)
    aj = aob[system.col].astype(np.int64)
    na = system.n_atoms
    key = np.unique(ai * na + aj)
    a, b = key // na, key % na
    keep = a != b
    a, b = a[keep], b[keep]
    adj = [[] for _ in range(na)]
    for x, y in zip(a.tolist(), b.tolist()):
        adj[x].append(y)
    return adj


def _split(D, centers, adj, leaf_atoms, cell=(0.0, 0.0, 0.0)):
    Nd = len(D)
    if Nd <= leaf_atoms:
        return None
    best = None  # (measure, Ns, axis, m_min, m_max, n_min, n_max, order)
    for axis in range(3):
        L = cell[axis]
        if L > 0:
            x = {a: centers[a][axis] - L * math.floor(centers[a][axis] / L) for a in D}
        else:
            x = {a: centers[a][axis] for a in D}
        order = sorted(D, key=lambda a: (x[a], a))
        ordn = {a: i + 1 for i, a in enumerate(order)}
        nucleus = min(D, key=lambda a: (sum(1 for b in adj[a] if b in ordn), ordn[a]))
        q = ordn[nucleus]

        def span(atom, lo, hi):
            for b in adj[atom]:
                o = ordn.get(b)
                if o is not None:
                    if L > 0:
                        o += -math.floor((x[b] - x[atom]) / L + 0.5) * Nd
                    if o < lo:
                        lo = o
                    if o > hi:
                        hi = o
            return lo, hi

        m_min = m_max = q
        n_min, n_max = span(nucleus, q, q)
        axis_best = None

        def consider(m_min, m_max, n_min, n_max, axis_best):
            N0 = m_max - m_min + 1
            Ns = n_max - n_min + 1 - N0
            N1 = Nd - N0 - Ns
            if N1 >= 1:
                key = (abs(N0 - N1) + Ns, Ns)
                if axis_best is None or key <= axis_best[0]:
                    return (key, m_min, m_max, n_min, n_max)
            return axis_best

        axis_best = consider(m_min, m_max, n_min, n_max, axis_best)
        while m_max - m_min + 1 < Nd:
            up = down = None
            if m_max < Nd:
                lo, hi = span(order[m_max], min(n_min, m_max + 1), max(n_max, m_max + 1))
                N0 = m_max - m_min + 2
                Ns = hi - lo + 1 - N0
                up = (abs(N0 - (Nd - N0 - Ns)) + Ns, lo, hi)
            if m_min > 1:
                lo, hi = span(order[m_min - 2], min(n_min, m_min - 1), max(n_max, m_min - 1))
                N0 = m_max - m_min + 2
                Ns = hi - lo + 1 - N0
                down = (abs(N0 - (Nd - N0 - Ns)) + Ns, lo, hi)
            if up is not None and (down is None or up[0] <= down[0]):
                m_max += 1
                n_min, n_max = up[1], up[2]
            else:
                m_min -= 1
                n_min, n_max = down[1], down[2]
            axis_best = consider(m_min, m_max, n_min, n_max, axis_best)
        if axis_best is not None:
            key = axis_best[0]
            if best is None or key < best[0]:
                best = (key, axis, axis_best[1], axis_best[2], axis_best[3], axis_best[4], order)
    if best is None:
        return None
    _, axis, m_min, m_max, n_min, n_max, order = best
    in_sep = {(x - 1) % Nd for x in list(range(n_min, m_min)) + list(range(m_max + 1, n_max + 1))}
    sub0 = order[m_min - 1:m_max]
    sep = [order[i] for i in sorted(in_sep)]
    sub1 = [order[i] for i in range(Nd) if i not in in_sep and not (m_min - 1 <= i < m_max)]
    return sorted(sub0), sorted(sub1), sorted(sep), axis


def nested_dissection(centers, adj, leaf_atoms=20, cell=None, screen_degree=0):
    """Supernodal tree in postorder.

    Returns dict with
      nodes: list of atom lists (ascending atom index) in postorder,
      parent: int array (-1 for the root), children: list of child-id lists,
      perm_atoms: atom order (concatenation of the node lists), axis: split axis (-1 for leaves).
    """
    centers = np.asarray(centers, dtype=np.float64).tolist()
    cell = tuple(float(c) for c in (cell if cell is not None else (0.0, 0.0, 0.0)))
    nodes, children, axes = [], [], []
    screened = [a for a in range(len(adj)) if screen_degree > 0 and len(adj[a]) > screen_degree]

    def rec(D, extra=()):
        res = _split(D, centers, adj, leaf_atoms, cell)
        if res is None:
            nodes.append(sorted(list(D) + list(extra)))
            children.append([])
            axes.append(-1)
            return len(nodes) - 1
        sub0, sub1, sep, axis = res
        c0 = rec(sub0)
        c1 = rec(sub1)
        nodes.append(sorted(sep + list(extra)))
        children.append([c0, c1])
        axes.append(axis)
        return len(nodes) - 1

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        kept = set(screened)
        rec([a for a in range(len(adj)) if a not in kept], screened)
    finally:
        sys.setrecursionlimit(old)
    parent = np.full(len(nodes), -1, dtype=np.int64)
    for p, ch in enumerate(children):
        for c in ch:
            parent[c] = p
    perm = [a for nd in nodes for a in nd]
    return dict(nodes=nodes, parent=parent, children=children, perm_atoms=np.array(perm),
                axis=np.array(axes))


def symbolic_structure(tree, adj):
    """struct(J) for every supernode J, in atoms, from the filled graph of the ordered matrix.

    Symmetric elimination in the structured order adds an edge between every two later
    neighbours of an eliminated atom; struct(J) is the set of later atoms adjacent (after fill)
    to some atom of J, minus J.  Returned as lists of atom ids sorted by structured position.
    """
    perm = tree["perm_atoms"]
    na = len(perm)
    pos = np.empty(na, dtype=np.int64)
    pos[perm] = np.arange(na)
    M = np.zeros((na, na), dtype=bool)
    for a, nb in enumerate(adj):
        for b in nb:
            M[pos[a], pos[b]] = True
    for k in range(na):
        later = np.nonzero(M[k, k + 1:])[0] + k + 1
        if later.size > 1:
            M[np.ix_(later, later)] = True
    out = []
    for atoms in tree["nodes"]:
        if not atoms:
            out.append([])
            continue
        p = pos[np.array(atoms)]
        last = p.max()
        cols = np.nonzero(M[p].any(axis=0))[0]
        cols = cols[cols > last]
        out.append(perm[cols].tolist())
    return out
