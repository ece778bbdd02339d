"""Write tests/golden/c4_electron_counts.txt: Tr(rho S) of the batched workload's systems with
N <= 16384 (`synth.batched_systems()`, indices listed in the file) at mu = -0.12, kT = 0.01 with
the 120-pole truncated Fermi function, from the oracle alone: generalised eigenvalues by LAPACK
and N_e = sum_nu 2 f_M((eps_nu - mu)/kT) (Eqs. 2, 5, 40).  The three systems with N = 24576 or
32768 are left out (dense eigenvalues too costly here).  Takes several minutes.

Run from the repository root:  python tests/golden/make_c4_electron_counts.py
"""
import os
import sys

import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.dense import electron_count_eig  # noqa: E402
from synth import batched_systems  # noqa: E402

MU, KT, M, NMAX = -0.12, 0.01, 120, 16384


def main():
    lines = []
    for i, s in enumerate(batched_systems()):
        if s.n > NMAX:
            continue
        Hd, Sd = s.dense()
        eps = scipy.linalg.eigh(Hd, Sd, eigvals_only=True)
        ne = electron_count_eig(eps, MU, KT, M)
        lines.append(f"{i} {s.n} {ne:.12f}")
        print(lines[-1], flush=True)
    path = os.path.join(ROOT, "tests", "golden", "c4_electron_counts.txt")
    with open(path, "w") as fh:
        fh.write("# Tr(rho S) of the batched workload's systems (index, N, count) at mu = -0.12, kT = 0.01,\n")
        fh.write("# 120 poles; oracle eigenvalues; written by tests/golden/make_c4_electron_counts.py\n")
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
