"""Seeded tight-binding Hamiltonian/overlap pairs on 1D/2D/3D lattices (open, or periodic
along chosen axes).

Recipe (one draw order, fixed per seed; PCG64 via numpy.random.Generator):
  * atoms on the integer grid (lattice constant a = 1), atom index = x + nx*(y + ny*z);
  * neighbour sets: 1D nearest (block tridiagonal), 2D nearest + next-nearest (8 in-plane
    offsets), 3D cut-off 1.8a (all 26 offsets in {-1,0,1}^3), or the square lattice's nearest
    neighbours only ("2dnn"); open boundaries, or wrapped along the periodic axes (Gamma point:
    one block per neighbouring pair of atoms of the cell, at least 3 atoms per periodic axis);
  * onsite block  H_aa = diag(U(-1,1)) + (G + G^T)/2, G ~ N(0, 0.1^2)  (o x o);
  * neighbour block H_ab ~ N(0, 0.1^2), H_ba = H_ab^T;
  * overlap S_aa = I, S_ab = c W_ab with W_ab ~ U(-1,1), W_ba = W_ab^T and
    c = min(0.05, 0.75 / max_i sum_j |W_ij|), so that lambda_min(S) >= 0.25;
  * H and S share one block pattern (every onsite block and every neighbour block),
    stored as CSR with sorted column indices in the original basis order.

The matrices are real symmetric, as for Gamma-point Kohn-Sham matrices of the paper's
Sec. II.A; z*S - H is then complex symmetric for complex z.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import itertools
import numpy as np

SEED_BASE = 1005008800

# name -> lattice description; sizes follow the benchmark configurations.
CONFIGS = {
    "C1": dict(shape=(64, 1, 1), orbitals=8, neighbours="1d", kT=0.01, poles=40,
               precision="fp64", label="1D chain 64 atoms x 8 orbitals (N=512)"),
    "C2": dict(shape=(32, 32, 1), orbitals=4, neighbours="2d", kT=0.01, poles=80,
               precision="fp64", label="2D square sheet 32x32 atoms x 4 orbitals (N=4096)"),
    "C3": dict(shape=(16, 16, 16), orbitals=4, neighbours="3d", kT=0.01, poles=80,
               precision="split", label="3D cubic 16^3 atoms x 4 orbitals (N=16384)"),
    "C5": dict(shape=(24, 24, 24), orbitals=8, neighbours="3d", kT=0.002, poles=160,
               precision="split", label="3D cubic 24^3 atoms x 8 orbitals (N=110592)"),
}

# Twelve systems of uneven size for the batched configuration (N from 2048 to 32768).
BATCHED_SYSTEMS = [
    dict(shape=(512, 1, 1), orbitals=4, neighbours="1d"),
    dict(shape=(1024, 1, 1), orbitals=8, neighbours="1d"),
    dict(shape=(2048, 1, 1), orbitals=6, neighbours="1d"),
    dict(shape=(4096, 1, 1), orbitals=8, neighbours="1d"),
    dict(shape=(32, 32, 1), orbitals=4, neighbours="2d"),
    dict(shape=(40, 40, 1), orbitals=5, neighbours="2d"),
    dict(shape=(48, 48, 1), orbitals=6, neighbours="2d"),
    dict(shape=(64, 64, 1), orbitals=8, neighbours="2d"),
    dict(shape=(8, 8, 8), orbitals=4, neighbours="3d"),
    dict(shape=(12, 12, 12), orbitals=8, neighbours="3d"),
    dict(shape=(16, 16, 16), orbitals=6, neighbours="3d"),
    dict(shape=(16, 16, 16), orbitals=8, neighbours="3d"),
]


@dataclass
class System:
    """A sparse symmetric pair (H, S) on one CSR pattern plus the geometry of its atoms."""
    n: int                      # number of basis functions
    rowptr: np.ndarray          # int64 [n+1]
    col: np.ndarray             # int32 [nnz], sorted within each row
    H: np.ndarray               # float64 [nnz]
    S: np.ndarray               # float64 [nnz]
    centers: np.ndarray         # float64 [n_atoms, 3]
    atom_of_basis: np.ndarray   # int32 [n]
    n_electrons: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_atoms(self) -> int:
        return int(self.centers.shape[0])

    def dense(self):
        """Dense copies of H and S (small systems only)."""
        Hd = np.zeros((self.n, self.n))
        Sd = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        Hd[rows, self.col] = self.H
        Sd[rows, self.col] = self.S
        return Hd, Sd

    def rows(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr))


def _offsets(neighbours: str):
    if neighbours == "1d":
        return [(1, 0, 0)]
    if neighbours == "2dnn":           # square lattice, nearest neighbours only
        return [(1, 0, 0), (0, 1, 0)]
    if neighbours == "2d":
        return [(1, 0, 0), (0, 1, 0), (1, 1, 0), (1, -1, 0)]
    if neighbours == "3d":
        out = []
        for d in itertools.product((-1, 0, 1), repeat=3):
            if d > (0, 0, 0):          # one of each +/- pair
                out.append(d)
        return out
    raise ValueError(neighbours)


def _atom_pairs(shape, neighbours, periodic=(False, False, False)):
    """Sorted unique pairs (a, b), a < b, of neighbouring atoms on the grid (open, or wrapped
    along the periodic axes, which need at least 3 atoms)."""
    nx, ny, nz = shape
    for n_ax, per in zip(shape, periodic):
        if per and n_ax < 3:
            raise ValueError("a periodic axis needs at least 3 atoms")
    xs, ys, zs = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    xs, ys, zs = xs.ravel(), ys.ravel(), zs.ravel()
    idx = xs + nx * (ys + ny * zs)
    pa, pb = [], []
    for dx, dy, dz in _offsets(neighbours):
        x2, y2, z2 = xs + dx, ys + dy, zs + dz
        if periodic[0]:
            x2 = x2 % nx
        if periodic[1]:
            y2 = y2 % ny
        if periodic[2]:
            z2 = z2 % nz
        ok = (x2 >= 0) & (x2 < nx) & (y2 >= 0) & (y2 < ny) & (z2 >= 0) & (z2 < nz)
        a = idx[ok]
        b = (x2 + nx * (y2 + ny * z2))[ok]
        pa.append(np.minimum(a, b))
        pb.append(np.maximum(a, b))
    pa = np.concatenate(pa)
    pb = np.concatenate(pb)
    key = np.unique(pa.astype(np.int64) * (nx * ny * nz) + pb)
    return key // (nx * ny * nz), key % (nx * ny * nz)


def _assemble_csr(n_atoms, o, pa, pb, onsite_H, onsite_S, pair_H, pair_S):
    """CSR of the block matrix with onsite blocks and symmetric pair blocks."""
    n = n_atoms * o
    # block list: onsite, (a,b) and (b,a)=transpose
    ba = np.concatenate([np.arange(n_atoms), pa, pb])
    bb = np.concatenate([np.arange(n_atoms), pb, pa])
    blkH = np.concatenate([onsite_H, pair_H, np.transpose(pair_H, (0, 2, 1))])
    blkS = np.concatenate([onsite_S, pair_S, np.transpose(pair_S, (0, 2, 1))])
    ii, jj = np.meshgrid(np.arange(o), np.arange(o), indexing="ij")
    rows = (ba[:, None, None] * o + ii[None]).ravel()
    cols = (bb[:, None, None] * o + jj[None]).ravel()
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    Hv = blkH.ravel()[order]
    Sv = blkS.ravel()[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return n, rowptr, cols.astype(np.int32), Hv.astype(np.float64), Sv.astype(np.float64)


def lattice_system(shape, orbitals, neighbours, seed, onsite_range=1.0, hop_std=0.1,
                   overlap=0.05, electrons=None, periodic=(False, False, False)) -> System:
    """Draw one seeded (H, S) pair on a lattice, open or periodic per axis (see module
    docstring; meta["cell"] holds the periodic cell lengths, 0 for open axes)."""
    shape = tuple(int(v) for v in shape) + (1,) * (3 - len(shape))
    periodic = tuple(bool(p) for p in periodic) + (False,) * (3 - len(periodic))
    nx, ny, nz = shape
    n_atoms = nx * ny * nz
    o = int(orbitals)
    rng = np.random.Generator(np.random.PCG64(seed))
    pa, pb = _atom_pairs(shape, neighbours, periodic)
    npair = pa.shape[0]
    eps = rng.uniform(-onsite_range, onsite_range, size=(n_atoms, o))
    G = rng.normal(0.0, hop_std, size=(n_atoms, o, o))
    onsite_H = 0.5 * (G + np.transpose(G, (0, 2, 1)))
    onsite_H[:, np.arange(o), np.arange(o)] += eps
    pair_H = rng.normal(0.0, hop_std, size=(npair, o, o))
    W = rng.uniform(-1.0, 1.0, size=(npair, o, o))
    # Gershgorin bound of the symmetric W (row sums over both orientations)
    rs = np.zeros(n_atoms * o)
    absW = np.abs(W)
    np.add.at(rs, (pa[:, None] * o + np.arange(o)[None]).ravel(), absW.sum(axis=2).ravel())
    np.add.at(rs, (pb[:, None] * o + np.arange(o)[None]).ravel(), absW.sum(axis=1).ravel())
    c = overlap if npair == 0 else min(overlap, 0.75 / float(rs.max()))
    onsite_S = np.broadcast_to(np.eye(o), (n_atoms, o, o)).copy()
    pair_S = c * W
    n, rowptr, col, Hv, Sv = _assemble_csr(n_atoms, o, pa, pb, onsite_H, onsite_S, pair_H, pair_S)
    xs, ys, zs = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cen = np.zeros((n_atoms, 3))
    idx = (xs + nx * (ys + ny * zs)).ravel()
    cen[idx, 0] = xs.ravel()
    cen[idx, 1] = ys.ravel()
    cen[idx, 2] = zs.ravel()
    aob = np.repeat(np.arange(n_atoms, dtype=np.int32), o)
    ne = float(n) / 2.0 if electrons is None else float(electrons)
    return System(n, rowptr, col, Hv, Sv, cen, aob, ne,
                  dict(shape=shape, orbitals=o, neighbours=neighbours, seed=seed,
                       overlap_scale=c,
                       cell=tuple(float(n_ax) if per else 0.0 for n_ax, per in zip(shape, periodic))))


def chain_nntb(n_atoms, a=0.0, b=-1.0, s=0.0, electrons=None) -> System:
    """s-valent nearest-neighbour tight-binding chain: onsite a, hopping b, overlap s.

    One orbital per atom, open ends; the model of the paper's Sec. II.C.1 and Fig. 1.
    """
    n = int(n_atoms)
    rows, cols, hv, sv = [], [], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                hv.append(a if i == j else b)
                sv.append(1.0 if i == j else s)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, np.array(rows) + 1, 1)
    rowptr = np.cumsum(rowptr)
    cen = np.zeros((n, 3))
    cen[:, 0] = np.arange(n)
    ne = float(n) / 2.0 if electrons is None else float(electrons)
    return System(n, rowptr, np.array(cols, dtype=np.int32), np.array(hv), np.array(sv), cen,
                  np.arange(n, dtype=np.int32), ne, dict(shape=(n, 1, 1), orbitals=1))


def csr_from_dense(Hd, Sd, centers=None, atom_of_basis=None, electrons=None) -> System:
    """CSR System from dense symmetric matrices (pattern = nonzeros of H or S or diagonal)."""
    n = Hd.shape[0]
    mask = (Hd != 0) | (Sd != 0) | np.eye(n, dtype=bool)
    rows, cols = np.nonzero(mask)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    if centers is None:
        centers = np.zeros((n, 3))
        centers[:, 0] = np.arange(n)
    if atom_of_basis is None:
        atom_of_basis = np.arange(n, dtype=np.int32)
    ne = float(n) / 2.0 if electrons is None else float(electrons)
    return System(n, rowptr, cols.astype(np.int32), Hd[rows, cols].astype(np.float64),
                  Sd[rows, cols].astype(np.float64), np.asarray(centers, dtype=np.float64),
                  np.asarray(atom_of_basis, dtype=np.int32), ne, {})


def config_system(name: str, system_index: int = 0) -> System:
    """The seeded system of a named benchmark configuration."""
    cfg = CONFIGS[name]
    cidx = {"C1": 0, "C2": 1, "C3": 2, "C4": 3, "C5": 4}[name]
    sysm = lattice_system(cfg["shape"], cfg["orbitals"], cfg["neighbours"],
                          SEED_BASE + cidx + system_index)
    sysm.meta.update(name=name, kT=cfg["kT"], poles=cfg["poles"], label=cfg["label"])
    return sysm


def batched_systems(count=None):
    """The twelve uneven systems of the batched configuration (seeded per system)."""
    out = []
    for i, d in enumerate(BATCHED_SYSTEMS[:count]):
        s = lattice_system(d["shape"], d["orbitals"], d["neighbours"], SEED_BASE + 3 + i)
        s.meta.update(name=f"C4.{i}", kT=0.01, poles=120)
        out.append(s)
    return out


def c5_family_systems(count, seed):
    """Small seeded systems of the 3D metallic workload's recipe (3D cubic lattice, cut-off 1.8a,
    8 orbitals per atom, onsite U(-1,1), hopping N(0, 0.1^2), overlap 0.05) for the
    chemical-potential seed: cubes and boxes of 4 to 7 atoms per side (N 512..2744), kT drawn in
    [0.0015, 0.003] Ha and the filling in [0.2, 0.3] electrons per orbital (the workload has 0.25).
    Returns (System, kT) pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        shape = tuple(int(v) for v in rng.integers(4, 8, size=3))
        n = int(np.prod(shape)) * 8
        filling = float(rng.uniform(0.2, 0.3))
        sysm = lattice_system(shape, 8, "3d", int(rng.integers(1 << 30)), electrons=round(n * filling))
        out.append((sysm, float(rng.uniform(0.0015, 0.003))))
    return out


def mu_training_systems(count, seed):
    """Small seeded systems with varied recipe parameters for the chemical-potential seed.

    Shapes, orbital counts, onsite range, hopping spread, overlap scale, filling and kT are
    drawn per system; every system uses the lattice recipe above.  Returns (System, kT) pairs.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = [((3, 3, 3), "3d"), ((4, 3, 2), "3d"), ((6, 5, 1), "2d"), ((5, 5, 1), "2d"),
              ((24, 1, 1), "1d")]
    out = []
    for i in range(count):
        shape, nb = shapes[int(rng.integers(len(shapes)))]
        o = int(rng.integers(2, 5))
        n = int(np.prod(shape)) * o
        filling = float(rng.uniform(0.15, 0.85))
        sysm = lattice_system(shape, o, nb, int(rng.integers(1 << 30)),
                              onsite_range=float(rng.uniform(0.5, 1.5)),
                              hop_std=float(rng.uniform(0.05, 0.2)),
                              overlap=float(rng.uniform(0.01, 0.08)),
                              electrons=round(2.0 * n * filling))
        out.append((sysm, float(rng.uniform(0.005, 0.02))))
    return out
