"""Seeded synthetic inputs shared by the CPU oracle checks, the GPU tests and the benchmark.

This package draws random structures (positions, species, cells) and random model weights. It holds none of
the method's arithmetic: no neighbour search, no radial integral, no spherical harmonic. Both sides of every
parity test receive the same arrays from here.
"""
from .structures import (  # noqa: F401
    System,
    random_cell_atoms,
    config_tiny,
    config_batch,
    config_diff,
    config_large,
    config_mlp,
    CONFIGS,
    linear_weights,
    mlp_initial_params,
    mlp_training_draws,
    small_cell_system,
    gpr_sparse_draws,
)
