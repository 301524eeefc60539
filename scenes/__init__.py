"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke test.

This package only draws random numbers and lays out arrays.  It holds none of
the method's arithmetic, so both the FP64 oracle and the CUDA library can be fed
from it without sharing any computation.
"""

from .synthetic import (  # noqa: F401
    FieldSpec, LatentScene, FullScene, field_weights, latent_scene,
    full_scene, latent_config1, latent_config3, full_config2, tiny_latent,
)
