"""Seeded synthetic inputs for the AMR raycaster: hierarchies, fields, cameras, transfer functions.

This package holds input generation only. It contains none of the rendering method's
arithmetic (no kD-tree, no interpolation, no traversal, no compositing); both the FP64
oracle and the CUDA path consume what it produces.
"""
from .amr import (  # noqa: F401
    Hierarchy,
    Camera,
    make_c1,
    make_c2,
    make_hierarchy_from_boxes,
    make_uniform,
    orbit_camera,
    ramp_tf,
    tf_variants,
    c1_workload,
    c2_workload,
)
