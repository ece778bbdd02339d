"""GPU parity at full size, element by element, against the oracle.

* The 3D cubic workload (16^3 atoms x 4 orbitals, N = 16384, 80 poles) and the 3D metallic
  workload (24^3 x 8, N = 110592, kT = 0.002, 160 poles): rho on every pattern entry of eight
  sampled columns against the oracle's Krylov columns of Eq. 8, stored with their a-posteriori
  error bound by tests/golden/make_rho_columns.py (oracle only).
* A 3D lattice of 12 x 12 x 13 atoms x 8 orbitals dissected into innermost domains of up to 900
  atoms: two domains of 6912 orbitals under a 1152-orbital separator, so the factor and
  selected-inversion GEMMs have inner dimensions of 1152 to 6912 (the slicer's two-row and
  one-row blocks, dozens of 256-element chunks per tile) - compared the same way.
* The 2D sheet (32 x 32 atoms x 4 orbitals, N = 4096, 80 poles): rho on every pattern entry
  against the oracle's dense eigendecomposition route.
Tolerances: 1e-10 (FP64 path) and 1e-9 (split path) max-abs on rho.
"""
import numpy as np
import pytest

from synth import SEED_BASE, config_system, lattice_system
from oracle.dense import generalized_eig, density_eig, on_pattern
from tests.conftest import golden_path
from tests.libtools import lib
from tests.test_gpu_parity import _density

pytestmark = pytest.mark.gpu

MU = -0.12
TOL = {0: 1e-10, 1: 1e-9}


def _stored(name):
    """(columns, {pattern index: rho}, error bound, mu, kT, M, leaf) of a stored oracle file."""
    import re
    vals, cols, bound, meta = {}, None, None, None
    with open(golden_path(f"rho_columns_{name}.txt")) as fh:
        for ln in fh:
            if ln.startswith("#"):
                m = re.search(r"mu = ([-\d.eE+]+), kT = ([-\d.eE+]+), (\d+) poles, leaf_atoms (\d+)", ln)
                if m:
                    meta = (float(m.group(1)), float(m.group(2)), int(m.group(3)), int(m.group(4)))
                m = re.search(r"# columns: (.*)", ln)
                if m:
                    cols = [int(c) for c in m.group(1).split()]
                m = re.search(r"a posteriori\): ([\d.eE+-]+);", ln)
                if m:
                    bound = float(m.group(1))
                continue
            k, v = ln.split()
            vals[int(k)] = float(v)
    return cols, vals, bound, meta


def _check_stored(system, name, precision, **opts):
    import gc
    import torch
    gc.collect()                    # plans of earlier tests release their device workspaces
    torch.cuda.empty_cache()
    cols, vals, bound, (mu, kT, M, leaf) = _stored(name)
    assert bound < 1e-11            # the oracle's own error is far inside the tolerance
    rho, ne = _density(system, mu, kT, M, precision=precision, leaf_atoms=leaf, **opts)
    idx = np.fromiter(vals.keys(), dtype=np.int64)
    ref = np.fromiter(vals.values(), dtype=np.float64)
    # every stored entry belongs to a stored column, and every column is complete
    assert set(system.col[idx].tolist()) == set(cols)
    assert idx.size == int(np.isin(system.col, cols).sum())
    err = float(np.max(np.abs(rho[idx] - ref)))
    print(f"{name} precision {precision}: max |rho - oracle| = {err:.2e} on {idx.size} entries")
    assert err < TOL[precision]
    return rho, ne


@pytest.mark.parametrize("precision", [1, 0])
def test_density_C3_matches_oracle_columns(precision):
    _check_stored(config_system("C3"), "C3", precision)


def test_density_long_inner_dimensions_match_oracle_columns():
    # split path only: the FP64 path would spend minutes on these 8064-wide fronts
    s = lattice_system((12, 12, 13), 8, "3d", SEED_BASE + 7)
    nd = lib()
    plan = nd.analyze_system(s, leaf_atoms=900)
    info = nd.ndsi_plan_info(plan)
    assert info["max_front"] == 6912 + 1152 and info["n_nodes"] == 3
    del plan
    _check_stored(s, "wide", 1)


def test_density_C5_split_matches_oracle_columns():
    s = config_system("C5")
    rho, ne = _check_stored(s, "C5", 1)
    assert abs(ne - float(np.dot(rho, s.S))) < 1e-6


def test_density_C5_split_without_far_pole_relaxation():
    # every pole on the full slice count: the same columns, for the accuracy the relaxation costs
    _check_stored(config_system("C5"), "C5", 1, split_far_ratio=-1.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_density_C2_every_pattern_entry(precision):
    s = config_system("C2")
    kT, M = s.meta["kT"], s.meta["poles"]
    Hd, Sd = s.dense()
    eps, C = generalized_eig(Hd, Sd)
    ref = on_pattern(density_eig(eps, C, MU, kT, M), s)
    rho, ne = _density(s, MU, kT, M, precision=precision)
    err = float(np.max(np.abs(rho - ref)))
    print(f"C2 precision {precision}: max |rho - oracle| over {s.nnz} entries = {err:.2e}")
    assert err < TOL[precision]
