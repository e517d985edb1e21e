"""Seeded synthetic inputs shared by the CPU oracle tests and the CUDA path.

This package only *draws* inputs: voxel keys (level, i, j, k), per-voxel
parameter records, sensor descriptors and ray subsamples.  It contains none of
the rendering arithmetic (no traversal, no field evaluation, no compositing),
so that the oracle and the GPU path can both consume it without sharing any of
the method's code.
"""

from .scenes import (  # noqa: F401
    SceneData,
    RECORD_SCALARS,
    draw_params,
    tiny_scene,
    driving_scene,
    random_multilevel_scene,
    deep_scene,
    single_voxel_scene,
    shuffle_scene,
)
from .actors import actor_shell, actor_tracks  # noqa: F401
from .sensors import (  # noqa: F401
    pinhole,
    fisheye,
    panorama,
    lidar,
    explicit_rays,
    camera_pose_looking,
    lidar_pose,
    yaw_matrix,
    sample_ray_indices,
    n_rays,
)
