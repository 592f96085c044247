"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This package holds no arithmetic of the nabla method: it only turns node
coordinates (longitude, latitude in radians, passed in by the caller) and
seeds into field values.  Both the oracle side and the GPU side consume the
arrays it returns, so neither computes its own inputs.
"""
from .fields import (  # noqa: F401
    NOISE_SIGMA,
    SEED_SCALAR,
    SEED_U,
    SEED_V,
    base_scalar,
    base_vector,
    level_scalar,
    level_vector,
    normal,
    padded,
    sample_nodes,
)
