"""Seeded synthetic inputs for the depth-weighted voxel fusion workloads.

This package is the one module that both the CPU oracle's tests and the CUDA
path's tests and bench read.  It holds none of the fusion method's arithmetic:
it draws seeded scenes (numpy PCG64), ray-casts them through pixel centres
into planar depth maps and object-id maps (the inputs a NeRF / 2DGS renderer
hands to the fusion stage, Sec. 3.1 "Preliminaries"), builds occupancy priors
(Sec. 3.5 "Occupancy by Morton-scattered opacity") and soft masks (Sec. 3.4),
and samples points near the surfaces (the Gaussian centres Pass 1 of
Sec. 3.6 labels).

Recipes follow the five workload shapes of the fusion hot path:
``config1`` (tiny sphere scene), ``config2`` (forward-facing dense),
``config3`` (unbounded sparse, contracted), ``config4`` (config 2 with mask
logits), ``session_mix`` (many uneven sessions).
"""
from .scenes import (  # noqa: F401
    Camera,
    Grid,
    Scene,
    Workload,
    config1,
    config2,
    config3,
    config4,
    gaussians,
    nerf_density,
    with_nerf_tuple,
    look_at,
    render_tuple,
    session_mix,
    session_workload,
    prompts,
    quaternions,
    with_tuple,
)
