"""ctypes mirror of include/salf.h and the loader of libsalf.so.

Argument marshalling only: every step of rendering runs in the library's
CUDA kernels.  There is no fallback: if libsalf.so cannot be built or loaded
the import fails loudly.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

c_int32, c_int64, c_float, c_double, c_void_p = C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_void_p

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_OVERLAP, ERR_AGAIN, ERR_TIMEOUT, ERR_NOT_FOUND, \
    ERR_SHUTDOWN, ERR_DEVICE, ERR_IO = range(11)
STATUS_NAMES = ["OK", "INVALID", "OOM", "CUDA", "OVERLAP", "AGAIN", "TIMEOUT", "NOT_FOUND",
                "SHUTDOWN", "DEVICE", "IO"]
KIND = {"pinhole": 0, "fisheye": 1, "pano": 2, "lidar": 3, "explicit": 4}
MODE = {"exp": 0, "sdf": 1}
DTYPE = {"f32": 0, "bf16": 1}


class SceneDesc(C.Structure):
    _fields_ = [("n", c_int64), ("origin", c_double * 3), ("s0", c_double), ("dims", c_int32 * 3),
                ("max_level", c_int32), ("level", c_void_p), ("ijk", c_void_p), ("mode", c_int32),
                ("dtype", c_int32), ("params", c_void_p), ("params_on_device", c_int32),
                ("keys_on_device", c_int32)]


class Sensor(C.Structure):
    _fields_ = [("kind", c_int32), ("width", c_int32), ("height", c_int32), ("fx", c_float),
                ("fy", c_float), ("cx", c_float), ("cy", c_float), ("fov", c_float),
                ("elev_min", c_float), ("elev_max", c_float), ("pose0", c_double * 12),
                ("pose1", c_double * 12), ("t0", c_double), ("t1", c_double),
                ("rolling_shutter", c_int32), ("t_near", c_float), ("t_far", c_float),
                ("rays", c_void_p)]


class RenderOpts(C.Structure):
    _fields_ = [("t_min_transmittance", c_float), ("background", c_float * 3),
                ("want_intensity", c_int32), ("visits_cap", c_int32), ("ray_segments", c_int32)]


class Outputs(C.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("opacity", c_void_p),
                ("intensity", c_void_p), ("saved", c_void_p), ("valid", c_void_p),
                ("visit_count", c_void_p), ("visits", c_void_p), ("ray_dump", c_void_p),
                ("steps", c_void_p), ("on_host", c_int32), ("max_alpha", c_void_p),
                ("raydrop", c_void_p)]


class SceneInfo(C.Structure):
    _fields_ = [("n", c_int64), ("mode", c_int32), ("dtype", c_int32), ("max_level", c_int32),
                ("dims", c_int32 * 3), ("n_level0_cells", c_int64), ("n_nodes", c_int64),
                ("device_bytes", c_int64), ("dev_params", c_void_p), ("dev_order", c_void_p)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("rejected", c_int64),
                ("launches", c_int64), ("rays", c_int64), ("p50_ms", c_double),
                ("p99_ms", c_double), ("max_ms", c_double), ("peak_bytes", c_int64),
                ("requests_launched", c_int64), ("max_batch", c_int64),
                ("mixed_launches", c_int64), ("latency_window", c_int64)]


class Actor(C.Structure):
    _fields_ = [("actor", c_void_p), ("pose0", c_double * 12), ("pose1", c_double * 12),
                ("id_base", c_int32), ("reserved", c_int32)]


class RefineCounts(C.Structure):
    _fields_ = [("n_new", c_int64), ("n_kept", c_int64), ("n_split", c_int64),
                ("n_pruned", c_int64)]


class SecondaryOpts(C.Structure):
    _fields_ = [("kind", c_int32), ("eta", c_float), ("light_dir", c_float * 3),
                ("min_opacity", c_float), ("offset", c_float), ("t_far", c_float)]


SECONDARY = {"reflect": 0, "refract": 1, "shadow": 2}


class RasterStats(C.Structure):
    _fields_ = [("visible_voxels", c_int64), ("pairs", c_int64), ("tiles", c_int32),
                ("key_bits", c_int32), ("kernels", c_int32), ("reserved", c_int32)]


# Every symbol include/salf.h declares, with its ctypes signature.
SIGNATURES = {
    "salf_create": ([c_int32, C.POINTER(c_void_p)], c_int32),
    "salf_destroy": ([c_void_p], None),
    "salf_build_scene": ([c_void_p, C.POINTER(SceneDesc), C.POINTER(c_void_p)], c_int32),
    "salf_scene_destroy": ([c_void_p], None),
    "salf_scene_get_info": ([c_void_p, C.POINTER(SceneInfo)], c_int32),
    "salf_scene_update_params": ([c_void_p, c_void_p, c_int32, c_void_p], c_int32),
    "salf_scene_params": ([c_void_p, C.POINTER(c_void_p), C.POINTER(c_void_p)], c_int32),
    "salf_render_rays": ([c_void_p, C.POINTER(Sensor), C.POINTER(RenderOpts), C.POINTER(Outputs),
                          c_void_p], c_int32),
    "salf_render_rays_actors": ([c_void_p, C.POINTER(Actor), c_int32, C.POINTER(Sensor),
                                 C.POINTER(RenderOpts), C.POINTER(Outputs), c_void_p], c_int32),
    "salf_scene_refine_plan": ([c_void_p, c_void_p, c_void_p, C.c_float, C.c_float,
                                C.POINTER(RefineCounts), c_void_p], c_int32),
    "salf_scene_refine_apply": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
                                c_int32),
    "salf_scene_reg_loss": ([c_void_p, c_void_p, C.c_float, C.c_float, C.c_float, c_void_p,
                             c_void_p, c_void_p], c_int32),
    "salf_secondary_rays": ([c_void_p, C.POINTER(Sensor), c_void_p, c_void_p,
                             C.POINTER(SecondaryOpts), c_void_p, c_void_p], c_int32),
    "salf_render_raster": ([c_void_p, C.POINTER(Sensor), C.POINTER(RenderOpts),
                            C.POINTER(Outputs), C.POINTER(RasterStats), c_void_p], c_int32),
    "salf_render_rays_host_noalloc": ([c_void_p, C.POINTER(Sensor), C.POINTER(RenderOpts),
                                       C.POINTER(Outputs), c_void_p], c_int32),
    "salf_render_backward": ([c_void_p, C.POINTER(Sensor), C.POINTER(RenderOpts), c_void_p,
                              c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p], c_int32),
    "salf_render_backward_actors": ([c_void_p, C.POINTER(Actor), c_int32, C.POINTER(Sensor),
                                     C.POINTER(RenderOpts), c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "salf_render_rays_batch": ([c_void_p, c_int32, C.POINTER(Sensor), C.POINTER(RenderOpts),
                                C.POINTER(Outputs), c_void_p], c_int32),
    "salf_render_backward_batch": ([c_void_p, c_int32, C.POINTER(Sensor), C.POINTER(RenderOpts),
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p], c_int32),
    "salf_scene_check": ([c_void_p], c_int32),
    "salf_scene_save": ([c_void_p, C.c_char_p], c_int32),
    "salf_scene_load": ([c_void_p, C.c_char_p, C.POINTER(c_void_p)], c_int32),
    "salf_serve_create": ([c_void_p, C.c_size_t, c_int32, C.POINTER(c_void_p)], c_int32),
    "salf_serve_submit": ([c_void_p, C.POINTER(Sensor), C.POINTER(RenderOpts),
                           C.POINTER(C.c_uint64)], c_int32),
    "salf_serve_poll": ([c_void_p, C.c_uint64, c_int32, C.POINTER(Outputs), C.POINTER(c_int32)],
                        c_int32),
    "salf_serve_release": ([c_void_p, C.c_uint64], c_int32),
    "salf_serve_get_stats": ([c_void_p, C.POINTER(ServeStats)], c_int32),
    "salf_serve_hold": ([c_void_p, c_int32], c_int32),
    "salf_serve_destroy": ([c_void_p], None),
    "salf_launch_param_bytes": ([], C.c_size_t),
    "salf_measure_l2_read": ([C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_double)], C.c_int),
    "salf_last_error": ([], C.c_char_p),
}

_lock = threading.Lock()
_lib = None


class SalfError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: SALF_ERR_{name}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsalf.so (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libsalf.so not found at {path}; run "
                                   "`python -m paper_2507_18713_gb300.build`")
            lib = C.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def check(status: int, where: str):
    if status != OK:
        msg = load().salf_last_error()
        raise SalfError(status, where, msg.decode() if msg else "")
