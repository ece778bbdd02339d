"""Seeded synthetic tight-binding systems shared by the oracle, the tests and the bench.

This package only draws inputs (H, S, atom centres, the basis-to-atom map).  It holds
none of the method's arithmetic: no poles, no ordering, no factorisation.
"""
from .lattice import (  # noqa: F401
    SEED_BASE,
    CONFIGS,
    BATCHED_SYSTEMS,
    System,
    lattice_system,
    chain_nntb,
    config_system,
    batched_systems,
    csr_from_dense,
    mu_training_systems,
    c5_family_systems,
)
