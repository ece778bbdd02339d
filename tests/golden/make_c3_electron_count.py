"""Write tests/golden/c3_electron_count.txt: Tr(rho S) of the 3D cubic workload (16^3 atoms x 4
orbitals, N = 16384, seeded as `synth.config_system("C3")`) at mu = -0.12, kT = 0.01 with the
80-pole truncated Fermi function, from the oracle alone: the generalised eigenvalues by LAPACK
and N_e = sum_nu 2 f_M((eps_nu - mu)/kT) (Eqs. 2, 5, 40).  Takes a few minutes on a few cores.

Run from the repository root:  python tests/golden/make_c3_electron_count.py
"""
import os
import sys

import numpy as np
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.dense import electron_count_eig  # noqa: E402
from synth import config_system  # noqa: E402

MU, KT, M = -0.12, 0.01, 80


def main():
    s = config_system("C3")
    Hd, Sd = s.dense()
    eps = scipy.linalg.eigh(Hd, Sd, eigvals_only=True)
    ne = electron_count_eig(eps, MU, KT, M)
    path = os.path.join(ROOT, "tests", "golden", "c3_electron_count.txt")
    with open(path, "w") as fh:
        fh.write("# Tr(rho S) of config C3 (N = 16384) at mu = -0.12, kT = 0.01, 80 poles; oracle eigenvalues\n")
        fh.write("# written by tests/golden/make_c3_electron_count.py\n")
        fh.write(f"{ne:.12f}\n")
    print(ne)


if __name__ == "__main__":
    main()
