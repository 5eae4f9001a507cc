"""Depth-weighted multi-view voxel fusion (DivAS, arXiv 2601.04860) on B300.

The hot path -- occupancy-prior gate and active list, projection of every
active voxel into every view, depth and mask gates, Gaussian depth-weighted
votes, normalisation and consensus threshold, Pass 1 labelling of points --
runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/divas_fuse.h``.  This package is the thin Python binding.
"""
from ._lib import (  # noqa: F401
    MASK_F16,
    MASK_F32,
    MASK_LOGIT_F32,
    DivasError,
    load,
)
from .fusion import (  # noqa: F401
    FusionParams,
    NerfParams,
    PreparedViews,
    TupleParams,
    VoxelFusion,
    density_floor,
    seg_bits_to_bool,
)
from .autograd import DivasFuseFunction, fuse  # noqa: F401,E402
from .batch import Autotuner, Batch, Schedule  # noqa: F401,E402
from .serve import Server, latency_summary, poisson_requests, serve_plain  # noqa: F401,E402
from .occupancy import OccupancyParams, SceneFrame, occupancy, scene_frame  # noqa: F401,E402
