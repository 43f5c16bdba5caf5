"""Seeded synthetic REI instances (inputs only; no part of the inference method)."""
from .gen import (  # noqa: F401
    CONFIGS,
    Instance,
    make_instance,
    make_config,
    pack_strings,
    type1_instance,
    type2_instance,
    poisson_trace,
    printed_instance,
    wide_large_instance,
)
