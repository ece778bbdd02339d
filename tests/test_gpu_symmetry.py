"""GPU density and selected inverse against exact symmetries, no oracle involved.

A bipartite system (S = I, hopping only between neighbouring sites of opposite sublattices, no
on-site terms) has P H P = -H with P = +-1 on the two sublattices, and the pole-truncated Fermi
function of Eq. 7 keeps f_M(x) + f_M(-x) = 1.  So rho(mu) + P rho(-mu) P = 2 I for every M:
rho_ii(mu) + rho_ii(-mu) = 2, rho_ii(0) = 1, and rho_ij(mu) = rho_ij(-mu) between neighbours.  A
wrong pole weight, a dropped or mis-scaled M0 term (Eq. 8) or a wrong spin factor breaks it.
"""
import numpy as np
import pytest

from synth import csr_from_dense
from tests.test_gpu_parity import _density

pytestmark = pytest.mark.gpu


def _bipartite_cubic(shape, seed):
    nx, ny, nz = shape
    o = 2
    na = nx * ny * nz
    rng = np.random.Generator(np.random.PCG64(seed))
    Hd = np.zeros((na * o, na * o))
    centers = np.zeros((na, 3))
    sub = np.zeros(na, dtype=int)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                a = x + nx * (y + ny * z)
                centers[a] = (x, y, z)
                sub[a] = (x + y + z) % 2
                for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    x2, y2, z2 = x + dx, y + dy, z + dz
                    if x2 < nx and y2 < ny and z2 < nz:
                        b = x2 + nx * (y2 + ny * z2)
                        blk = rng.normal(-0.5, 0.2, (o, o))
                        Hd[a * o:(a + 1) * o, b * o:(b + 1) * o] = blk
                        Hd[b * o:(b + 1) * o, a * o:(a + 1) * o] = blk.T
    aob = np.repeat(np.arange(na, dtype=np.int32), o)
    s = csr_from_dense(Hd, np.eye(na * o), centers=centers, atom_of_basis=aob)
    return s, sub[aob]


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-9)])
def test_density_particle_hole_symmetry(precision, tol):
    s, p = _bipartite_cubic((8, 7, 6), 41)
    rows = s.rows()
    diag = rows == s.col
    assert np.all(p[rows[~diag]] != p[s.col[~diag]])       # the pattern links opposite sublattices only
    kT, M = 0.02, 80
    r0, n0 = _density(s, 0.0, kT, M, precision=precision, leaf_atoms=12)
    assert np.max(np.abs(r0[diag] - 1.0)) < tol
    assert abs(n0 - s.n) < tol * s.n
    rp, _ = _density(s, 0.13, kT, M, precision=precision, leaf_atoms=12)
    rm, _ = _density(s, -0.13, kT, M, precision=precision, leaf_atoms=12)
    assert np.max(np.abs(rp[diag] + rm[diag] - 2.0)) < tol
    assert np.max(np.abs(rp[~diag] - rm[~diag])) < tol
    assert np.max(np.abs(rp[~diag])) > 1e-3                 # the off-diagonal entries are not trivially zero


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-9)])
def test_green_at_conjugate_points_is_conjugate(precision, tol):
    # real H and S: (z* S - H)^{-1} = conj((z S - H)^{-1}) on every selected element
    from synth import lattice_system
    from tests.test_gpu_parity import _selinv
    s = lattice_system((7, 6, 5), 2, "3d", 43)
    Z = np.array([-0.3 + 0.04j, 0.8 + 1.7j])
    g = _selinv(s, np.concatenate([Z, np.conj(Z)]), precision=precision, leaf_atoms=12)
    for q in range(len(Z)):
        scale = np.max(np.abs(g[q]))
        assert np.max(np.abs(g[len(Z) + q] - np.conj(g[q]))) < tol * scale


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-9)])
def test_density_is_invariant_under_affine_energy_change(precision, tol):
    # rho depends on the pencil only through (eps - mu) / kT: H -> a H + b S, mu -> a mu + b,
    # kT -> a kT leaves every element of rho unchanged (the points alpha_p = mu + i z_p kT, the
    # weights -4 R_p kT and M0 all follow)
    from synth import lattice_system
    s = lattice_system((7, 6, 5), 2, "3d", 44)
    a, b = 2.5, 0.3
    mu, kT, M = -0.12, 0.01, 80
    r1, n1 = _density(s, mu, kT, M, precision=precision, leaf_atoms=12)
    H0 = s.H.copy()
    s.H = a * H0 + b * s.S
    try:
        r2, n2 = _density(s, a * mu + b, a * kT, M, precision=precision, leaf_atoms=12)
    finally:
        s.H = H0
    assert np.max(np.abs(r2 - r1)) < tol
    assert abs(n2 - n1) < tol * s.n
