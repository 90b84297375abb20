"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This module makes data only: analytic scenes (unions of spheres, boxes and
cylinders inside the unit cube that stands for the paper's normalized object
coordinate space, §III-A), pinhole cameras, ray batches with RGB-D targets and
object/background labels (§III-B, "Training Data"), noisy prior occupancy grids,
stratified uniforms, random background colours and initial parameters.  It
holds none of the method's arithmetic: no sampling, encoding, MLP, rendering,
loss or optimiser step lives here, and it imports neither the oracle nor the
CUDA package.
"""

from .scenes import (  # noqa: F401
    Primitive,
    Scene,
    scene_sphere_box,
    scene_random_csg,
    cameras_on_sphere,
    RayPool,
    make_ray_pool,
    object_pose,
    keyframe_cameras,
    render_keyframe,
    prior_grid,
    stratified_uniforms,
    random_colours,
    init_params,
    sample_batch,
)
