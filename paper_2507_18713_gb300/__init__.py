"""GB300 (sm_103a) ray-cast renderer for SaLF sparse local fields (arXiv 2507.18713).

The compute path lives in libsalf.so (hand-written CUDA kernels behind the C
ABI of include/salf.h); this package is the thin Python binding.
"""

from ._lib import SalfError, library_path, load  # noqa: F401
from .api import (Context, HostFrames, RenderBatchFn, RenderFn, Scene, Server, VoxelSet,  # noqa: F401
                  device_view, n_rays, rays_sensor)
