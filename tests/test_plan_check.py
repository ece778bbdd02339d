"""The host-side schedule check (bounds of every index the kernels follow, no overlapping writes
or read-after-write hazards between the work items of one launch) over many plans."""
import numpy as np
import pytest

from synth import batched_systems, config_system, lattice_system
from tests.libtools import lib


@pytest.mark.parametrize("name", ["C1", "C2", "C3", "C5"])
@pytest.mark.parametrize("precision", [0, 1])
def test_config_plans_pass(name, precision):
    nd = lib()
    nd.ndsi_plan_check(nd.analyze_system(config_system(name), precision=precision))


def test_batched_plan_passes():
    nd = lib()
    nd.ndsi_plan_check(nd.analyze_batched(batched_systems(), precision=1))


@pytest.mark.parametrize("opts", [dict(block=32), dict(block=64, outer_block=256), dict(outer_block=64),
                                  dict(leaf_atoms=3), dict(leaf_atoms=60, block=32, outer_block=96),
                                  dict(block=64, outer_block=128), dict(outer_block=32, leaf_atoms=40)])
@pytest.mark.parametrize("shape,o,nb", [((9, 8, 1), 4, "2d"), ((5, 5, 5), 3, "3d"), ((120, 1, 1), 2, "1d")])
def test_option_variants_pass(opts, shape, o, nb):
    nd = lib()
    s = lattice_system(shape, o, nb, 17)
    nd.ndsi_plan_check(nd.analyze_system(s, **opts))


@pytest.mark.parametrize("shape,nb,periodic", [((16, 16, 1), "2dnn", (True, True, False)),
                                               ((6, 5, 7), "3d", (True, True, True))])
def test_periodic_and_screened_plans_pass(shape, nb, periodic):
    nd = lib()
    s = lattice_system(shape, 2, nb, 18, periodic=periodic)
    nd.ndsi_plan_check(nd.analyze_system(s, cell=s.meta["cell"], precision=1))
    from tests.test_oracle_nd import _long_tail_system
    t = _long_tail_system(lattice_system((10, 9, 1), 2, "2d", 8), 3, 4.0, 2)
    nd.ndsi_plan_check(nd.analyze_system(t, screen_degree=12))
