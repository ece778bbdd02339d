"""Geometric nested dissection of Sec. II.C.1, steps (i)-(v), and the symbolic fill.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  An independent, plain-Python statement
of the ordering rules, compared bit for bit with the library's host analysis.

Granularity is the atom (the orbitals of an atom stay together).  Two atoms are adjacent when
H or S has a nonzero block between them.  For a domain D of N_d atoms:
 (i)   for each axis a_i (i = 0, 1, 2) number the atoms 1..N_d by (coordinate_i, atom index);
 (ii)  long-tail screening is not applied (uniform lattices need none);
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
"""
from __future__ import annotations

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


def _split(D, centers, adj, leaf_atoms):
    Nd = len(D)
    if Nd <= leaf_atoms:
        return None
    best = None  # (measure, Ns, axis, m_min, m_max, n_min, n_max, order)
    for axis in range(3):
        order = sorted(D, key=lambda a: (centers[a][axis], a))
        ordn = {a: i + 1 for i, a in enumerate(order)}
        nucleus = min(D, key=lambda a: (sum(1 for b in adj[a] if b in ordn), ordn[a]))
        q = ordn[nucleus]

        def span(atom, lo, hi):
            for b in adj[atom]:
                o = ordn.get(b)
                if o is not None:
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
    sub0 = order[m_min - 1:m_max]
    sep = order[n_min - 1:m_min - 1] + order[m_max:n_max]
    sub1 = order[:n_min - 1] + order[n_max:]
    return sorted(sub0), sorted(sub1), sorted(sep), axis


def nested_dissection(centers, adj, leaf_atoms=20):
    """Supernodal tree in postorder.

    Returns dict with
      nodes: list of atom lists (ascending atom index) in postorder,
      parent: int array (-1 for the root), children: list of child-id lists,
      perm_atoms: atom order (concatenation of the node lists), axis: split axis (-1 for leaves).
    """
    centers = np.asarray(centers, dtype=np.float64).tolist()
    nodes, children, axes = [], [], []

    def rec(D):
        res = _split(D, centers, adj, leaf_atoms)
        if res is None:
            nodes.append(sorted(D))
            children.append([])
            axes.append(-1)
            return len(nodes) - 1
        sub0, sub1, sep, axis = res
        c0 = rec(sub0)
        c1 = rec(sub1)
        nodes.append(sep)
        children.append([c0, c1])
        axes.append(axis)
        return len(nodes) - 1

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        rec(list(range(len(adj))))
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
