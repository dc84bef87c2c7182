"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package holds scene *data* only: primitive lists, materials, cameras,
parameter bindings, initial and reference parameters, kernel bandwidths and
estimator settings. It contains none of the estimator's or the renderer's
arithmetic (no random-number generator of the method, no ray tracing, no loss),
so that the CUDA library and the FP64 oracle can both consume it without
sharing any computation.
"""
from .scenes import (  # noqa: F401
    PRIM_SPHERE, PRIM_QUAD, PRIM_BOX,
    MAT_DIFFUSE, MAT_MIRROR, MAT_DIELECTRIC,
    BIND_PRIM_POS, BIND_SPHERE_RADIUS, BIND_MAT_ALBEDO, BIND_MAT_EMISSION, BIND_TEXTURE,
    SAMPLER_RADIAL, SAMPLER_PERDIM, SAMPLER_GAUSS,
    Scene, Workload, SceneBuilder,
    config_small, config_occlusion, config_gi_box, config_caustic, config_small_albedo, config_gi_albedo, config_texture,
    all_configs, scaled, serving_mix,
)
