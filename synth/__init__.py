"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package only *generates inputs*: oriented point clouds on analytic shapes
(sphere, real spherical-harmonic star bodies, a travelling-wave ellipsoid),
uniform query points and the serving request mix.  It contains none of the
reconstruction method's arithmetic (no splat, divergence, solve, iso-value,
marching cubes, distance or adjoint).  Everything is computed in float64 with
numpy and handed out as contiguous float32 arrays.
"""
from .shapes import (  # noqa: F401
    CONFIG_SEEDS,
    real_sh,
    sh_count,
    sh_surface,
    sh_surface_vjp,
    sphere_cloud,
    sh_body_cloud,
    sh_fixed_dirs_cloud,
    random_sh_body_theta,
    wave_ellipsoid_cloud,
    uniform_queries,
    uniform_dirs,
    serving_requests,
    config_inputs,
)
