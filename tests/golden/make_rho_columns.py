"""Write tests/golden/rho_columns_<name>.txt: sampled columns of the density matrix from the
oracle alone, for workloads too large for the dense routes.

For each seeded column j, rho e_j = S^{-1} e_j + sum_p w_p Re[(alpha_p S - H)^{-1} e_j] (Eq. 8,
alpha_p = mu + i z_p kT, w_p = -4 R_p kT) by the oracle's Krylov solves (oracle/krylov.py), each
to a true relative residual of 1e-13; the file stores the values at the pattern entries of those
columns and the a-posteriori error bound of the solves.  With --direct the same columns are also
computed by SuperLU solves per pole (oracle/dense.py density_columns) and the largest difference
between the two routes is recorded.

Workloads (systems from synth, with the bench's mu = -0.12):
  C3    - 3D cubic 16^3 atoms x 4 orbitals (N = 16384), kT 0.01, 80 poles;
  C5    - 3D cubic 24^3 atoms x 8 orbitals (N = 110592), kT 0.002, 160 poles;
  wide  - 3D cubic 12 x 12 x 13 atoms x 8 orbitals (N = 14976), kT 0.01, 40 poles, dissected
          with innermost domains of up to 900 atoms (two domains of 6912 orbitals under a
          1152-orbital separator): the long inner dimensions of the slicing and GEMM steps.

Run from the repository root:  python tests/golden/make_rho_columns.py C3 [--direct]
C3 takes about a minute on 8 cores (the SuperLU check about 15 minutes), wide a few minutes,
C5 about half an hour.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.krylov import density_columns_krylov, krylov_threads  # noqa: E402
from synth import SEED_BASE, config_system, lattice_system  # noqa: E402

MU = -0.12
N_COLUMNS = 8


def workload(name):
    """(system, kT, M, leaf_atoms) of a named workload."""
    if name in ("C3", "C5"):
        s = config_system(name)
        return s, s.meta["kT"], s.meta["poles"], 20
    if name == "wide":
        return lattice_system((12, 12, 13), 8, "3d", SEED_BASE + 7), 0.01, 40, 900
    raise ValueError(name)


def columns(system, count=N_COLUMNS, seed=8800):
    """Seeded distinct columns, always including the first and the last basis function."""
    rng = np.random.default_rng(seed)
    inner = rng.choice(np.arange(1, system.n - 1), count - 2, replace=False)
    return sorted([0, system.n - 1] + inner.tolist())


def main():
    name = sys.argv[1]
    s, kT, M, leaf = workload(name)
    cols = columns(s)
    t0 = time.perf_counter()
    rho, info = density_columns_krylov(s, MU, kT, M, cols)
    t_kry = time.perf_counter() - t0
    direct = None
    if "--direct" in sys.argv:
        from oracle.dense import density_columns
        t0 = time.perf_counter()
        ref = density_columns(s, MU, kT, M, cols)
        direct = (float(np.max(np.abs(ref - rho))), time.perf_counter() - t0)
    rows = s.rows()
    path = os.path.join(ROOT, "tests", "golden", f"rho_columns_{name}.txt")
    with open(path, "w") as fh:
        fh.write(f"# rho on the pattern entries of sampled columns, workload {name} (N = {s.n}), "
                 f"mu = {MU}, kT = {kT}, {M} poles, leaf_atoms {leaf}\n")
        fh.write("# written by tests/golden/make_rho_columns.py from the oracle's Krylov solves (Eq. 8)\n")
        fh.write(f"# columns: {' '.join(str(c) for c in cols)}\n")
        fh.write(f"# error bound (max-abs, a posteriori): {info['bound']:.3e}; max residual "
                 f"{info['max_residual']:.3e}; {info['iterations']} iterations; {t_kry:.0f} s on "
                 f"{krylov_threads()} threads\n")
        if direct:
            fh.write(f"# SuperLU route (density_columns): max |difference| {direct[0]:.3e} ({direct[1]:.0f} s)\n")
        fh.write("# pattern_index value\n")
        for c, j in enumerate(cols):
            for k in np.nonzero(s.col == j)[0]:
                fh.write(f"{int(k)} {rho[rows[k], c]:.17e}\n")
    print(name, info, f"{t_kry:.1f} s", direct)


if __name__ == "__main__":
    main()
