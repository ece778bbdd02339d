"""GPU parity of the FP64 path against the oracle (dense inverse, eigen route, sampled columns).

Every call goes through the C ABI (libndsi.so) via the ctypes binding; torch only allocates.
Tolerance: 1e-10 max-abs on rho (FP64 form); G is compared relative to max|G|.
"""
import numpy as np
import pytest

from synth import chain_nntb, config_system, lattice_system, csr_from_dense
from oracle.dense import (generalized_eig, density_eig, find_mu_eig, on_pattern,
                          electron_count_pattern, green_dense, density_columns)
from tests.conftest import golden_lines, golden_path
from tests.libtools import lib

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-10


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _selinv(system, Z, **opts):
    torch = _torch()
    nd = lib()
    plan = nd.analyze_system(system, **opts)
    H = _dev(torch, system.H)
    S = _dev(torch, system.S)
    f = nd.ndsi_factor_poles(plan, H, S, np.asarray(Z, dtype=complex))
    G = torch.zeros((len(Z), system.nnz, 2), dtype=torch.float64, device="cuda")
    nd.ndsi_selinv(f, G)
    torch.cuda.synchronize()
    g = G.cpu().numpy()
    return g[..., 0] + 1j * g[..., 1]


def _density(system, mu, kT, M, host=False, **opts):
    torch = _torch()
    nd = lib()
    plan = nd.analyze_system(system, **opts)
    if host:
        H, S = system.H.copy(), system.S.copy()
        rho = np.zeros(system.nnz)
        ne = np.zeros(1)
        nd.ndsi_density(plan, H, S, mu, kT, M, rho, ne)
        return rho, float(ne[0])
    H = _dev(torch, system.H)
    S = _dev(torch, system.S)
    rho = torch.zeros(system.nnz, dtype=torch.float64, device="cuda")
    ne = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd.ndsi_density(plan, H, S, mu, kT, M, rho, ne)
    torch.cuda.synchronize()
    return rho.cpu().numpy(), float(ne.cpu()[0])


def test_appA_selected_inverse_exact():
    # App. A: X is the structured all-ones chain; with H = -X, S = I and z = 0 the library
    # factors X itself (indefinite, nonsingular pivots 1, -1, 1) and must return the printed
    # selected inverse exactly.
    X = np.loadtxt(golden_path("appA_structured_X.txt"))
    perm = [int(v) - 1 for v in golden_lines("appA_ordering.txt")[0].split()]
    inv = np.empty(7, int)
    inv[perm] = np.arange(7)
    Xo = X[np.ix_(inv, inv)]                       # back to chain order
    sysm = csr_from_dense(-Xo, np.eye(7))
    g = _selinv(sysm, [0.0], leaf_atoms=1)[0]
    ref = np.linalg.inv(Xo)
    assert np.array_equal(g.real, on_pattern(ref, sysm)) and np.all(g.imag == 0)
    rows = [ln.split() for ln in golden_lines("appA_selected_inverse.txt")]
    G = np.full((7, 7), np.nan)
    G[sysm.rows(), sysm.col] = g.real
    Gs = G[np.ix_(perm, perm)]
    for i in range(7):
        for j in range(7):
            if rows[i][j] != "*" and not np.isnan(Gs[i, j]):
                assert Gs[i, j] == float(rows[i][j])


@pytest.mark.parametrize("shape,o,nb,leaf", [
    ((40, 1, 1), 3, "1d", 6), ((9, 7, 1), 2, "2d", 5), ((5, 4, 4), 2, "3d", 6),
    ((11, 10, 1), 4, "2d", 20), ((6, 6, 5), 3, "3d", 20)])
def test_selected_inverse_matches_dense(shape, o, nb, leaf):
    sysm = lattice_system(shape, o, nb, 77)
    Hd, Sd = sysm.dense()
    Z = [0.1 + 0.0314j, -0.7 + 2.5j, 1e7j, 0.3 - 0.05j]
    g = _selinv(sysm, Z, leaf_atoms=leaf)
    for q, z in enumerate(Z):
        ref = on_pattern(green_dense(Hd, Sd, z), sysm)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(g[q] - ref)) < 1e-12 * scale * max(1.0, np.sqrt(sysm.n) / 10), (shape, z)
        # complex symmetry: G_ij = G_ji on the pattern
        Gm = np.zeros((sysm.n, sysm.n), complex)
        Gm[sysm.rows(), sysm.col] = g[q]
        assert np.max(np.abs(Gm - Gm.T)) == 0.0


@pytest.mark.parametrize("block", [16, 32, 64])
def test_pivot_block_sizes(block):
    sysm = lattice_system((8, 7, 1), 5, "2d", 5)
    Hd, Sd = sysm.dense()
    z = -0.2 + 0.05j
    g = _selinv(sysm, [z], leaf_atoms=12, block=block)[0]
    ref = on_pattern(green_dense(Hd, Sd, z), sysm)
    assert np.max(np.abs(g - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("block,outer", [(32, 32), (16, 48), (32, 64), (16, 128)])
def test_outer_block_sizes(block, outer):
    # two-level factorisation of A_J: diagonal blocks of `outer` columns factored and inverted in
    # pivot blocks of `block`, outer panel / trailing update / inverse assembly between them;
    # the separators here (up to 108 columns) span several outer blocks
    sysm = lattice_system((6, 6, 5), 3, "3d", 5)
    Hd, Sd = sysm.dense()
    Z = [-0.2 + 0.05j, 0.3 + 1.5j]
    g = _selinv(sysm, Z, leaf_atoms=12, block=block, outer_block=outer)
    for q, z in enumerate(Z):
        ref = on_pattern(green_dense(Hd, Sd, z), sysm)
        assert np.max(np.abs(g[q] - ref)) < 1e-11 * np.max(np.abs(ref))


def _rho_check(sysm, kT, M, leaf=20, host=False, tol=RHO_TOL, **opts):
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    mu = find_mu_eig(eps, kT, sysm.n_electrons, M)
    rho_ref = on_pattern(density_eig(eps, C, mu, kT, M), sysm)
    rho, ne = _density(sysm, mu, kT, M, host=host, leaf_atoms=leaf, **opts)
    assert np.max(np.abs(rho - rho_ref)) < tol
    assert abs(ne - electron_count_pattern(rho, sysm)) < 1e-9
    assert abs(ne - sysm.n_electrons) < 1e-8
    return rho, ne


def test_density_C1_full():
    sysm = config_system("C1")
    _rho_check(sysm, sysm.meta["kT"], sysm.meta["poles"])


@pytest.mark.parametrize("shape,o,nb,leaf,M", [
    ((12, 12, 1), 2, "2d", 20, 40), ((6, 6, 6), 2, "3d", 20, 40), ((7, 5, 3), 3, "3d", 8, 60),
    ((200, 1, 1), 2, "1d", 9, 40)])
def test_density_small_lattices(shape, o, nb, leaf, M):
    _rho_check(lattice_system(shape, o, nb, 123), 0.01, M, leaf)


@pytest.mark.parametrize("shape,o,nb,periodic,leaf", [
    ((12, 10, 1), 2, "2d", (True, True, False), 12), ((5, 4, 6), 2, "3d", (True, True, True), 8),
    ((60, 1, 1), 3, "1d", (True, False, False), 4)])
@pytest.mark.parametrize("precision,tol", [(0, RHO_TOL), (1, 1e-9)])
def test_density_periodic_lattices(shape, o, nb, periodic, leaf, precision, tol):
    # periodic cells (Sec. II.C.1 step (i)): separators wrap around the cell
    sysm = lattice_system(shape, o, nb, 124, periodic=periodic)
    _rho_check(sysm, 0.01, 40, leaf, tol=tol, cell=sysm.meta["cell"], precision=precision)


def test_density_screened_long_tails():
    # long-tail atoms in the root separator (Sec. II.C.1 step (ii))
    from tests.test_oracle_nd import _long_tail_system
    sysm = _long_tail_system(lattice_system((10, 9, 1), 2, "2d", 8), 3, 4.0, 2)
    _rho_check(sysm, 0.01, 40, 6, screen_degree=12)


def test_density_host_buffers_match_device():
    sysm = lattice_system((10, 9, 1), 2, "2d", 31)
    r1, n1 = _density(sysm, -0.05, 0.01, 40)
    r2, n2 = _density(sysm, -0.05, 0.01, 40, host=True)
    assert np.array_equal(r1, r2) and n1 == n2


def test_density_chunked_poles_match():
    # A workspace cap that forces several pole chunks gives the same rho.
    torch = _torch()
    nd = lib()
    sysm = lattice_system((10, 8, 1), 3, "2d", 8)
    r1, n1 = _density(sysm, 0.0, 0.01, 30)
    plan = nd.analyze_system(sysm)
    info = nd.ndsi_plan_info(plan)
    r2, n2 = _density(sysm, 0.0, 0.01, 30, max_workspace_bytes=int(info["front_elems"] * 16 * 7))
    assert np.max(np.abs(r1 - r2)) < 1e-13 and abs(n1 - n2) < 1e-11


def test_density_C2_full_sampled_columns():
    # Full C2 (N = 4096, 80 poles) in the bench's launch configuration; sampled columns of rho
    # from the oracle's sparse solves, compared on their pattern entries.
    sysm = config_system("C2")
    kT, M = sysm.meta["kT"], sysm.meta["poles"]
    mu = -0.12
    rho, ne = _density(sysm, mu, kT, M)
    rng = np.random.default_rng(5)
    cols = sorted(rng.choice(sysm.n, 6, replace=False).tolist())
    ref = density_columns(sysm, mu, kT, M, cols)
    rows = sysm.rows()
    for t, j in enumerate(cols):
        sel = np.nonzero(sysm.col == j)[0]
        assert np.max(np.abs(rho[sel] - ref[rows[sel], t])) < RHO_TOL
    assert abs(ne - electron_count_pattern(rho, sysm)) < 1e-8
    # rho is symmetric on the pattern
    R = np.zeros((sysm.n, sysm.n))
    R[rows, sysm.col] = rho
    assert np.max(np.abs(R - R.T)) < 1e-13


def test_singular_pivot_reported():
    # z = 0 with H = 0 makes every pivot block zero: the kernel's pivot check reports it.
    nd = lib()
    sysm = lattice_system((4, 4, 1), 2, "2d", 3)
    sysm.H[:] = 0.0
    with pytest.raises(nd.NdsiError) as ei:
        _selinv(sysm, [0.0])
    assert ei.value.code == nd.ndsi.NDSI_ERR_SINGULAR


@pytest.mark.parametrize("precision", [0, 1])
def test_degenerate_systems(precision):
    # one atom with one orbital (a 1 x 1 front, no separator), one innermost domain holding the
    # whole system (no dissection step), and a 2-atom chain split into three one-atom nodes
    for sysm, leaf in ((lattice_system((1, 1, 1), 1, "1d", 41), 20),
                       (lattice_system((4, 3, 1), 3, "2d", 42), 20),
                       (lattice_system((3, 1, 1), 2, "1d", 43), 1)):
        Hd, Sd = sysm.dense()
        Z = [0.2 + 0.01j, -1.3 + 0.7j]
        g = _selinv(sysm, Z, leaf_atoms=leaf, precision=precision)
        for q, z in enumerate(Z):
            ref = on_pattern(green_dense(Hd, Sd, z), sysm)
            assert np.max(np.abs(g[q] - ref)) < 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,tol", [(0, RHO_TOL), (1, 1e-9)])
def test_density_empty_and_full_bands(precision, tol):
    # mu well below the spectrum: no electrons (rho ~ 0); well above: every state doubly
    # occupied, rho = 2 S^{-1} on the pattern and Tr(rho S) = 2N (the full-band closed form).
    # |eps - mu| / kT stays within 120..300, where the 40-pole fraction equals the Fermi
    # function to ~1e-14 and exp(-120) is negligible.
    sysm = lattice_system((6, 5, 1), 2, "2d", 44)
    Hd, Sd = sysm.dense()
    eps, _ = generalized_eig(Hd, Sd)
    assert eps.min() > -1.6 and eps.max() < 1.6
    rho_lo, ne_lo = _density(sysm, -4.0, 0.02, 40, precision=precision)
    assert np.max(np.abs(rho_lo)) < tol and abs(ne_lo) < 1e-8
    rho_hi, ne_hi = _density(sysm, 4.0, 0.02, 40, precision=precision)
    ref = on_pattern(2.0 * np.linalg.inv(Sd), sysm)
    assert np.max(np.abs(rho_hi - ref)) < tol
    assert abs(ne_hi - 2 * sysm.n) < 1e-7


def test_density_single_pole():
    # M = 1: one pole pair plus the M0 point, against the oracle's one-pole Fermi function
    sysm = lattice_system((5, 4, 1), 2, "2d", 45)
    Hd, Sd = sysm.dense()
    eps, C = generalized_eig(Hd, Sd)
    rho_ref = on_pattern(density_eig(eps, C, 0.05, 0.05, 1), sysm)
    rho, ne = _density(sysm, 0.05, 0.05, 1)
    assert np.max(np.abs(rho - rho_ref)) < RHO_TOL


@pytest.mark.parametrize("precision", [1, 0])
def test_density_C3_electron_count_matches_oracle(precision):
    # Tr(rho S) (Eq. 40) of the 3D cubic workload, N = 16384, 80 poles, against the oracle's
    # eigenvalue count stored by tests/golden/make_c3_electron_count.py
    ref = float(golden_lines("c3_electron_count.txt")[0])
    sysm = config_system("C3")
    _, ne = _density(sysm, -0.12, 0.01, 80, precision=precision)
    assert abs(ne - ref) < 1e-9, (ne, ref)
