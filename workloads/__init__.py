"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This package only draws inputs (sphere centres, Janus axes, workload
parameters). It holds none of the collision-resolution arithmetic: no contact
matrix, no mobility, no LCP. Both the CPU oracle and the CUDA path consume
what it produces.
"""
from .packing import (  # noqa: F401
    WORKLOADS,
    Instance,
    janus_axes,
    make_instance,
    random_packing,
    batched_instances,
    serving_simulations,
)
