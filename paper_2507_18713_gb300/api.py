"""Python binding of libsalf: the names of include/salf.h, torch tensors for
device memory and streams.  Marshalling only -- no rendering arithmetic here.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import _lib as L

_ctx_cache: dict = {}


def _stream_ptr(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Context:
    """A libsalf context bound to one CUDA device (salf_create)."""

    def __init__(self, device: int = 0):
        lib = L.load()
        torch.cuda.init()
        h = C.c_void_p()
        L.check(lib.salf_create(int(device), C.byref(h)), "salf_create")
        self.device = int(device)
        self._h = h

    @classmethod
    def default(cls, device: int = 0) -> "Context":
        if device not in _ctx_cache:
            _ctx_cache[device] = cls(device)
        return _ctx_cache[device]

    def __del__(self):
        try:
            if self._h:
                L.load().salf_destroy(self._h)
                self._h = None
        except Exception:
            pass


def sensor_struct(sensor: dict, keep: list) -> L.Sensor:
    """salf_sensor from a descriptor dict (synth.sensors format)."""
    s = L.Sensor()
    s.kind = L.KIND[sensor["kind"]]
    s.width, s.height = int(sensor["width"]), int(sensor["height"])
    s.fx, s.fy, s.cx, s.cy = (float(sensor[k]) for k in ("fx", "fy", "cx", "cy"))
    s.fov, s.elev_min, s.elev_max = (float(sensor[k]) for k in ("fov", "elev_min", "elev_max"))
    s.pose0[:] = [float(v) for v in np.asarray(sensor["pose0"], np.float64).ravel()]
    s.pose1[:] = [float(v) for v in np.asarray(sensor["pose1"], np.float64).ravel()]
    s.t0, s.t1 = float(sensor["t0"]), float(sensor["t1"])
    s.rolling_shutter = int(bool(sensor["rolling_shutter"]))
    s.t_near, s.t_far = float(sensor["t_near"]), float(sensor["t_far"])
    if sensor["kind"] == "explicit":
        rays = sensor["rays"]
        if isinstance(rays, np.ndarray):
            rays = torch.from_numpy(np.ascontiguousarray(rays, np.float32)).cuda()
        rays = rays.contiguous()
        keep.append(rays)
        s.rays = rays.data_ptr()
    return s


def opts_struct(t_min=1e-4, background=(0.0, 0.0, 0.0), want_intensity=False,
                visits_cap=0, ray_segments=0) -> L.RenderOpts:
    o = L.RenderOpts()
    o.t_min_transmittance = float(t_min)
    o.background[:] = [float(v) for v in background]
    o.want_intensity = int(bool(want_intensity))
    o.visits_cap = int(visits_cap)
    o.ray_segments = int(ray_segments)
    return o


def n_rays(sensor: dict) -> int:
    return int(sensor["width"]) * int(sensor["height"])


def rays_sensor(rays) -> dict:
    """Explicit-ray sensor over an (R, 8) float32 CUDA tensor of rows
    (origin, direction, t_near, t_far), e.g. from Scene.secondary_rays."""
    R = int(rays.shape[0])
    return dict(kind="explicit", width=R, height=1, fx=0.0, fy=0.0, cx=0.0, cy=0.0, fov=0.0,
                elev_min=0.0, elev_max=0.0, pose0=np.eye(3, 4), pose1=np.eye(3, 4), t0=0.0,
                t1=0.0, rolling_shutter=False, t_near=0.0, t_far=0.0, rays=rays)


class VoxelSet:
    """A voxel set on a scene grid (what salf_build_scene takes): origin, s0,
    dims, max_level, level (n,), ijk (n, 3), params (n, 32), mode."""

    def __init__(self, origin, s0, dims, max_level, level, ijk, params, mode):
        self.origin, self.s0, self.dims, self.max_level = origin, s0, dims, max_level
        self.level, self.ijk, self.params, self.mode = level, ijk, params, mode


class Scene:
    """A built scene (salf_build_scene).  `scene` is a synth.SceneData (or any
    object with origin, s0, dims, max_level, level, ijk, params, mode)."""

    def __init__(self, scene, dtype: str = "f32", ctx: Context | None = None, params=None):
        self.ctx = ctx or Context.default()
        lib = L.load()
        p = scene.params if params is None else params
        keys_dev = isinstance(scene.level, torch.Tensor) and scene.level.is_cuda
        if keys_dev:  # the whole build runs on the GPU
            level = scene.level.contiguous().to(torch.uint8)
            ijk = scene.ijk.contiguous().to(torch.int32)
            if not (isinstance(p, torch.Tensor) and p.is_cuda):
                p = torch.as_tensor(np.asarray(p, dtype=np.float32), device=level.device)
        else:
            level = np.ascontiguousarray(scene.level, dtype=np.uint8)
            ijk = np.ascontiguousarray(scene.ijk, dtype=np.int32)
        on_dev = isinstance(p, torch.Tensor) and p.is_cuda
        if on_dev:
            p = p.contiguous().float()
        elif isinstance(p, torch.Tensor):
            p = np.ascontiguousarray(p.numpy(), dtype=np.float32)
        else:
            p = np.ascontiguousarray(p, dtype=np.float32)
        d = L.SceneDesc()
        d.n = int(level.shape[0])
        d.keys_on_device = int(keys_dev)
        d.origin[:] = [float(v) for v in scene.origin]
        d.s0 = float(scene.s0)
        d.dims[:] = [int(v) for v in scene.dims]
        d.max_level = int(scene.max_level)
        if keys_dev:
            d.level, d.ijk = level.data_ptr(), ijk.data_ptr()
        else:
            d.level, d.ijk = level.ctypes.data, ijk.ctypes.data
        d.mode = L.MODE[scene.mode]
        d.dtype = L.DTYPE[dtype]
        d.params = p.data_ptr() if on_dev else p.ctypes.data
        d.params_on_device = int(on_dev)
        h = C.c_void_p()
        if on_dev or keys_dev:
            torch.cuda.synchronize()
        L.check(lib.salf_build_scene(self.ctx._h, C.byref(d), C.byref(h)), "salf_build_scene")
        self._h = h
        self.n = d.n
        self.mode = scene.mode
        self.dtype = dtype
        self.geometry = dict(origin=tuple(float(v) for v in scene.origin), s0=float(scene.s0),
                             dims=tuple(int(v) for v in scene.dims),
                             max_level=int(scene.max_level))

    def save(self, path: str) -> None:
        """salf_scene_save: grid, keys and current records to a scene file."""
        L.check(L.load().salf_scene_save(self._h, os.fsencode(path)), "salf_scene_save")

    @classmethod
    def load(cls, path: str, ctx: Context | None = None) -> "Scene":
        """salf_scene_load: the scene a file written by save() describes."""
        self = cls.__new__(cls)
        self.ctx = ctx or Context.default()
        lib = L.load()
        h = C.c_void_p()
        L.check(lib.salf_scene_load(self.ctx._h, os.fsencode(path), C.byref(h)), "salf_scene_load")
        self._h = h
        info = L.SceneInfo()
        L.check(lib.salf_scene_get_info(h, C.byref(info)), "salf_scene_get_info")
        self.n = int(info.n)
        self.mode = {v: k for k, v in L.MODE.items()}[info.mode]
        self.dtype = {v: k for k, v in L.DTYPE.items()}[info.dtype]
        # origin and s0 from the file's header (after the 8-byte magic and 4 int32 + 1 int64)
        with open(path, "rb") as f:
            f.seek(8 + 16 + 8)
            geo = np.frombuffer(f.read(32), dtype="<f8")
        self.geometry = dict(origin=tuple(float(v) for v in geo[:3]), s0=float(geo[3]),
                             dims=tuple(int(v) for v in info.dims), max_level=int(info.max_level))
        return self

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.synchronize()
            L.load().salf_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = L.SceneInfo()
        L.check(L.load().salf_scene_get_info(self._h, C.byref(i)), "salf_scene_get_info")
        return {k: getattr(i, k) for k, _ in L.SceneInfo._fields_ if k != "dims"} | \
            {"dims": tuple(i.dims)}

    def check(self):
        L.check(L.load().salf_scene_check(self._h), "salf_scene_check")

    def grads_view(self) -> torch.Tensor:
        """salf_scene_params: zero-copy (n, 32) float32 CUDA view of the scene's
        own gradient buffer (input order), which backward(d_params="scene")
        accumulates into; library-owned, valid while the scene lives."""
        g = C.c_void_p()
        L.check(L.load().salf_scene_params(self._h, None, C.byref(g)), "salf_scene_params")
        return device_view(g.value, (self.n, 32), "<f4")

    def params_view(self) -> torch.Tensor:
        """salf_scene_params: zero-copy (n, 32) view of the scene's records in
        its storage dtype and internal voxel order (info()["dev_order"] maps
        internal -> input index)."""
        p = C.c_void_p()
        L.check(L.load().salf_scene_params(self._h, C.byref(p), None), "salf_scene_params")
        return device_view(p.value, (self.n, 32), "<f4" if self.dtype == "f32" else "<u2")

    def update_params(self, params, stream=None):
        """salf_scene_update_params: params (n, 32) float32, input order."""
        lib = L.load()
        if isinstance(params, torch.Tensor) and params.is_cuda:
            params = params.detach().contiguous().float()
            L.check(lib.salf_scene_update_params(self._h, params.data_ptr(), 1,
                                                 _stream_ptr(stream)), "salf_scene_update_params")
        else:
            arr = np.ascontiguousarray(params, dtype=np.float32)
            L.check(lib.salf_scene_update_params(self._h, arr.ctypes.data, 0,
                                                 _stream_ptr(stream)), "salf_scene_update_params")

    def render(self, sensor: dict, t_min=1e-4, background=(0.0, 0.0, 0.0), want_intensity=False,
               visits_cap=0, outputs=("rgb", "depth", "opacity"), saved=False, valid=True,
               stream=None, out: dict | None = None, ray_dump: bool = False,
               steps: bool = False, max_alpha=None, ray_segments: int = 0) -> dict:
        """salf_render_rays into (new or given) CUDA tensors; asynchronous on
        `stream` (default: torch's current stream).  `max_alpha` (n float32 CUDA
        tensor, input order) is max-accumulated with each voxel's largest
        composited alpha.  `ray_segments`: spans per ray walked in parallel
        (0 = the library's choice, 1 = whole rays)."""
        R = n_rays(sensor)
        dev = torch.device("cuda", self.ctx.device)
        res = {} if out is None else dict(out)
        shapes = {"rgb": (R, 3), "depth": (R,), "opacity": (R,), "intensity": (R,),
                  "raydrop": (R,)}
        for k in outputs:
            if k not in res:
                res[k] = torch.empty(shapes[k], dtype=torch.float32, device=dev)
        if saved and "saved" not in res:
            res["saved"] = torch.empty((R, 8), dtype=torch.float32, device=dev)
        if valid and "valid" not in res:
            res["valid"] = torch.empty((R,), dtype=torch.uint8, device=dev)
        if visits_cap > 0:
            res.setdefault("visit_count", torch.empty((R,), dtype=torch.int32, device=dev))
            res.setdefault("visits", torch.empty((R, visits_cap), dtype=torch.int32, device=dev))
        o = L.Outputs()
        if ray_dump and "ray_dump" not in res:
            res["ray_dump"] = torch.empty((R, 8), dtype=torch.float32, device=dev)
        if steps and "steps" not in res:
            res["steps"] = torch.empty((R,), dtype=torch.int32, device=dev)
        for k in ("rgb", "depth", "opacity", "intensity", "saved", "valid", "visit_count", "visits",
                  "ray_dump", "steps", "raydrop"):
            if k in res:
                setattr(o, k, res[k].data_ptr())
        if max_alpha is not None:
            assert max_alpha.is_cuda and max_alpha.dtype == torch.float32 and max_alpha.numel() == self.n
            o.max_alpha = max_alpha.data_ptr()
        keep: list = []
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, visits_cap, ray_segments)
        L.check(L.load().salf_render_rays(self._h, C.byref(s), C.byref(op), C.byref(o),
                                          _stream_ptr(stream)), "salf_render_rays")
        if keep:
            res["_keep"] = keep
        return res

    def render_batch(self, sensors, t_min=1e-4, background=(0.0, 0.0, 0.0),
                     want_intensity=False, outputs=("rgb", "depth", "opacity"), saved=False,
                     valid=True, stream=None, outs=None, ray_segments: int = 0) -> list:
        """salf_render_rays_batch: every sensor in one launch (list of output
        dicts of CUDA tensors, new or the given `outs`); asynchronous."""
        dev = torch.device("cuda", self.ctx.device)
        n = len(sensors)
        res = []
        arr = (L.Outputs * max(1, n))()
        sarr = (L.Sensor * max(1, n))()
        keep: list = []
        for i, sen in enumerate(sensors):
            R = n_rays(sen)
            d = {} if outs is None else dict(outs[i])
            shapes = {"rgb": (R, 3), "depth": (R,), "opacity": (R,), "intensity": (R,),
                      "raydrop": (R,)}
            for k in outputs:
                if k not in d:
                    d[k] = torch.empty(shapes[k], dtype=torch.float32, device=dev)
            if saved and "saved" not in d:
                d["saved"] = torch.empty((R, 8), dtype=torch.float32, device=dev)
            if valid and "valid" not in d:
                d["valid"] = torch.empty((R,), dtype=torch.uint8, device=dev)
            for k in ("rgb", "depth", "opacity", "intensity", "saved", "valid", "raydrop"):
                if k in d:
                    setattr(arr[i], k, d[k].data_ptr())
            sarr[i] = sensor_struct(sen, keep)
            res.append(d)
        op = opts_struct(t_min, background, want_intensity, 0, ray_segments)
        L.check(L.load().salf_render_rays_batch(self._h, n, sarr, C.byref(op), arr,
                                                _stream_ptr(stream)), "salf_render_rays_batch")
        if keep:
            res[0]["_keep"] = keep
        return res

    def backward_batch(self, sensors, saved, d_rgb=None, d_depth=None, d_opacity=None,
                       d_intensity=None, d_params=None, t_min=1e-4, background=(0.0, 0.0, 0.0),
                       want_intensity=False, stream=None):
        """salf_render_backward_batch: the adjoint of every sensor in one launch,
        summed into d_params (n, 32) float32 (new, given, or "scene").  saved
        and the d_* are lists (one tensor or None per sensor) or None."""
        dev = torch.device("cuda", self.ctx.device)
        own = isinstance(d_params, str) and d_params == "scene"
        if own:
            d_params = self.grads_view()
        elif d_params is None:
            d_params = torch.zeros((self.n, 32), dtype=torch.float32, device=dev)
        n = len(sensors)
        keep: list = []

        def ptrs(lst):
            if lst is None:
                return None
            ts = [None if t is None else t.contiguous() for t in lst]
            keep.extend(t for t in ts if t is not None)
            return C.cast((C.c_void_p * max(1, n))(*[None if t is None else t.data_ptr()
                                                    for t in ts]), C.c_void_p)

        sarr = (L.Sensor * max(1, n))()
        for i, sen in enumerate(sensors):
            sarr[i] = sensor_struct(sen, keep)
        op = opts_struct(t_min, background, want_intensity, 0)
        L.check(L.load().salf_render_backward_batch(
            self._h, n, sarr, C.byref(op), ptrs(saved), ptrs(d_rgb), ptrs(d_depth),
            ptrs(d_opacity), ptrs(d_intensity), None if own else d_params.data_ptr(),
            _stream_ptr(stream)), "salf_render_backward_batch")
        return d_params

    def render_raster(self, sensor: dict, t_min=1e-4, background=(0.0, 0.0, 0.0),
                      want_intensity=False, visits_cap=0, outputs=("rgb", "depth", "opacity"),
                      saved=False, valid=True, stream=None, out: dict | None = None,
                      stats: dict | None = None) -> dict:
        """salf_render_raster (tile rasterisation, pinhole cameras with one pose)
        into (new or given) CUDA tensors; the same outputs as `render`.  Waits
        on `stream` once (for the tile-list size).  `stats`, if given, receives
        the frame's visible voxels, (voxel, tile) pairs, tiles and key bits."""
        R = n_rays(sensor)
        dev = torch.device("cuda", self.ctx.device)
        res = {} if out is None else dict(out)
        shapes = {"rgb": (R, 3), "depth": (R,), "opacity": (R,), "intensity": (R,),
                  "raydrop": (R,)}
        for k in outputs:
            if k not in res:
                res[k] = torch.empty(shapes[k], dtype=torch.float32, device=dev)
        if saved and "saved" not in res:
            res["saved"] = torch.empty((R, 8), dtype=torch.float32, device=dev)
        if valid and "valid" not in res:
            res["valid"] = torch.empty((R,), dtype=torch.uint8, device=dev)
        if visits_cap > 0:
            res.setdefault("visit_count", torch.empty((R,), dtype=torch.int32, device=dev))
            res.setdefault("visits", torch.empty((R, visits_cap), dtype=torch.int32, device=dev))
        o = L.Outputs()
        for k in ("rgb", "depth", "opacity", "intensity", "saved", "valid", "visit_count", "visits",
                  "raydrop"):
            if k in res:
                setattr(o, k, res[k].data_ptr())
        keep: list = []
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, visits_cap)
        st = L.RasterStats()
        L.check(L.load().salf_render_raster(self._h, C.byref(s), C.byref(op), C.byref(o),
                                            C.byref(st), _stream_ptr(stream)),
                "salf_render_raster")
        if stats is not None:
            stats.update(visible_voxels=st.visible_voxels, pairs=st.pairs, tiles=st.tiles,
                         key_bits=st.key_bits, kernels=st.kernels)
        return res

    def refine(self, params, grads, max_alpha, split_threshold, prune_alpha=1e-3, stream=None):
        """Densify and prune (Sec. III-C): salf_scene_refine_plan + apply.  All
        tensors are CUDA, input order: params and grads (n, 32) float32,
        max_alpha (n,) float32.  Returns (VoxelSet with the new level / ijk
        / params as CUDA tensors, which Scene() builds on the GPU, counts dict)."""
        lib = L.load()
        params = params.contiguous().float()
        grads = grads.contiguous().float()
        max_alpha = max_alpha.contiguous().float()
        c = L.RefineCounts()
        L.check(lib.salf_scene_refine_plan(self._h, grads.data_ptr(), max_alpha.data_ptr(),
                                           float(split_threshold), float(prune_alpha),
                                           C.byref(c), _stream_ptr(stream)), "salf_scene_refine_plan")
        m = int(c.n_new)
        dev = params.device
        lv = torch.empty((m,), dtype=torch.uint8, device=dev)
        ij = torch.empty((m, 3), dtype=torch.int32, device=dev)
        pr = torch.empty((m, 32), dtype=torch.float32, device=dev)
        L.check(lib.salf_scene_refine_apply(self._h, params.data_ptr(), lv.data_ptr() if m else None,
                                            ij.data_ptr() if m else None,
                                            pr.data_ptr() if m else None, _stream_ptr(stream)),
                "salf_scene_refine_apply")
        g = self.geometry
        vs = VoxelSet(g["origin"], g["s0"], g["dims"], g["max_level"], lv, ij, pr, self.mode)
        return vs, dict(n_new=m, n_kept=int(c.n_kept), n_split=int(c.n_split),
                        n_pruned=int(c.n_pruned))

    def reg_loss(self, params, lambda_s, lambda_alpha, lambda_n, grads=None, loss=None,
                 stream=None):
        """salf_scene_reg_loss (Eq. 7 L_reg): returns (loss (1,) CUDA tensor,
        grads (n, 32)), both accumulated into the given tensors if any."""
        params = params.contiguous().float()
        if grads is None:
            grads = torch.zeros((self.n, 32), dtype=torch.float32, device=params.device)
        if loss is None:
            loss = torch.zeros((1,), dtype=torch.float32, device=params.device)
        L.check(L.load().salf_scene_reg_loss(self._h, params.data_ptr(), float(lambda_s),
                                             float(lambda_alpha), float(lambda_n), loss.data_ptr(),
                                             grads.data_ptr(), _stream_ptr(stream)),
                "salf_scene_reg_loss")
        return loss, grads

    def secondary_rays(self, sensor: dict, depth, opacity, kind="reflect", eta=1.0 / 1.33,
                       light_dir=(0.0, 0.0, 1.0), min_opacity=0.5, offset=1e-3, t_far=0.0,
                       out=None, stream=None):
        """salf_secondary_rays: (R, 8) CUDA tensor of explicit rays spawned at
        the expected hit points of a render of `sensor` (its depth and opacity
        outputs).  Trace them with render(rays_sensor(rays))."""
        R = n_rays(sensor)
        dev = torch.device("cuda", self.ctx.device)
        rays = out if out is not None else torch.empty((R, 8), dtype=torch.float32, device=dev)
        o = L.SecondaryOpts()
        o.kind = L.SECONDARY[kind]
        o.eta = float(eta)
        o.light_dir[:] = [float(v) for v in light_dir]
        o.min_opacity, o.offset, o.t_far = float(min_opacity), float(offset), float(t_far)
        keep: list = []
        s = sensor_struct(sensor, keep)
        depth, opacity = depth.contiguous(), opacity.contiguous()
        L.check(L.load().salf_secondary_rays(self._h, C.byref(s), depth.data_ptr(),
                                             opacity.data_ptr(), C.byref(o), rays.data_ptr(),
                                             _stream_ptr(stream)), "salf_secondary_rays")
        return rays

    def render_actors(self, sensor: dict, actors, t_min=1e-4, background=(0.0, 0.0, 0.0),
                      want_intensity=False, visits_cap=0, outputs=("rgb", "depth", "opacity"),
                      saved=False, valid=True, stream=None, out: dict | None = None) -> dict:
        """salf_render_rays_actors: this scene plus dynamic actors.  `actors` is a
        list of (Scene, pose0, pose1, id_base) with 3x4 canonical -> world poses
        at the sensor's t0 and t1.  Asynchronous on `stream`."""
        R = n_rays(sensor)
        dev = torch.device("cuda", self.ctx.device)
        res = {} if out is None else dict(out)
        shapes = {"rgb": (R, 3), "depth": (R,), "opacity": (R,), "intensity": (R,),
                  "raydrop": (R,)}
        for k in outputs:
            if k not in res:
                res[k] = torch.empty(shapes[k], dtype=torch.float32, device=dev)
        if saved and "saved" not in res:
            res["saved"] = torch.empty((R, 8), dtype=torch.float32, device=dev)
        if valid and "valid" not in res:
            res["valid"] = torch.empty((R,), dtype=torch.uint8, device=dev)
        if visits_cap > 0:
            res.setdefault("visit_count", torch.empty((R,), dtype=torch.int32, device=dev))
            res.setdefault("visits", torch.empty((R, visits_cap), dtype=torch.int32, device=dev))
        o = L.Outputs()
        for k in ("rgb", "depth", "opacity", "intensity", "saved", "valid", "visit_count", "visits",
                  "raydrop"):
            if k in res:
                setattr(o, k, res[k].data_ptr())
        arr = (L.Actor * max(1, len(actors)))()
        for k, (sc, p0, p1, base) in enumerate(actors):
            arr[k].actor = sc._h
            arr[k].pose0[:] = [float(v) for v in np.asarray(p0, dtype=np.float64).ravel()]
            arr[k].pose1[:] = [float(v) for v in np.asarray(p1, dtype=np.float64).ravel()]
            arr[k].id_base = int(base)
        keep: list = [arr, [a[0] for a in actors]]
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, visits_cap)
        L.check(L.load().salf_render_rays_actors(self._h, arr, len(actors), C.byref(s),
                                                 C.byref(op), C.byref(o), _stream_ptr(stream)),
                "salf_render_rays_actors")
        res["_keep"] = keep
        return res

    def render_host(self, sensor: dict, t_min=1e-4, background=(0.0, 0.0, 0.0),
                    want_intensity=False, outputs=("rgb", "depth", "opacity"), out=None,
                    stream=None, ray_segments: int = 0, sync: bool = True) -> dict:
        """salf_render_rays with host output buffers (on_host = 1): synchronous,
        results land in (pinned, if given) host memory.  sync=False (on_host = 2):
        `out` must be pinned; the call returns after the launch and the buffers
        hold the results once `stream` has drained."""
        R = n_rays(sensor)
        shapes = {"rgb": (R, 3), "depth": (R,), "opacity": (R,), "intensity": (R,),
                  "raydrop": (R,)}
        res = out if out is not None else {
            k: torch.empty(shapes[k], dtype=torch.float32, pin_memory=not sync) for k in outputs}
        o = L.Outputs()
        for k, v in res.items():
            setattr(o, k, v.data_ptr())
        o.on_host = 1 if sync else 2
        keep: list = []
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, 0, ray_segments)
        L.check(L.load().salf_render_rays(self._h, C.byref(s), C.byref(op), C.byref(o),
                                          _stream_ptr(stream)), "salf_render_rays(host)")
        return res

    def render_host_noalloc(self, sensor: dict, t_min=1e-4, background=(0.0, 0.0, 0.0),
                            want_intensity=False, outputs=("rgb", "depth", "opacity"), out=None,
                            stream=None, ray_segments: int = 0) -> dict:
        """salf_render_rays_host_noalloc: like render_host, but the library
        stages the outputs in its fixed device array instead of allocating."""
        R = n_rays(sensor)
        shapes = {"rgb": (R, 3), "depth": (R,), "opacity": (R,), "intensity": (R,), "valid": (R,),
                  "raydrop": (R,)}
        res = out if out is not None else {
            k: torch.empty(shapes[k], dtype=torch.uint8 if k == "valid" else torch.float32)
            for k in outputs}
        o = L.Outputs()
        for k, v in res.items():
            setattr(o, k, v.data_ptr())
        keep: list = []
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, 0, ray_segments)
        L.check(L.load().salf_render_rays_host_noalloc(self._h, C.byref(s), C.byref(op),
                                                       C.byref(o), _stream_ptr(stream)),
                "salf_render_rays_host_noalloc")
        return res

    def backward(self, sensor: dict, saved, d_rgb=None, d_depth=None, d_opacity=None,
                 d_intensity=None, d_params=None, t_min=1e-4, background=(0.0, 0.0, 0.0),
                 want_intensity=False, stream=None, raydrop=None, d_raydrop=None):
        """salf_render_backward: returns d_params (n, 32) float32 (accumulated
        into the given tensor if any; the string "scene" accumulates into the
        scene's own buffer, grads_view()).  With d_raydrop, `raydrop` is the
        forward's raydrop output."""
        dev = torch.device("cuda", self.ctx.device)
        own = isinstance(d_params, str) and d_params == "scene"
        if own:
            d_params = self.grads_view()
        elif d_params is None:
            d_params = torch.zeros((self.n, 32), dtype=torch.float32, device=dev)

        def ptr(t):
            return None if t is None else t.contiguous().data_ptr()

        keep = [t.contiguous() for t in (d_rgb, d_depth, d_opacity, d_intensity, raydrop,
                                         d_raydrop) if t is not None]
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, 0)
        L.check(L.load().salf_render_backward(
            self._h, C.byref(s), C.byref(op), saved.data_ptr(), ptr(d_rgb), ptr(d_depth),
            ptr(d_opacity), ptr(d_intensity), ptr(raydrop), ptr(d_raydrop),
            None if own else d_params.data_ptr(), _stream_ptr(stream)),
            "salf_render_backward")
        return d_params


    def backward_actors(self, sensor: dict, actors, saved, d_rgb=None, d_depth=None,
                        d_opacity=None, d_intensity=None, d_params=None, actor_d_params=None,
                        t_min=1e-4, background=(0.0, 0.0, 0.0), want_intensity=False,
                        stream=None):
        """salf_render_backward_actors: the adjoint of render_actors (same
        actors, poses, sensor and options; `saved` from that render).  Returns
        (d_params (n, 32), [actor k's (n_k, 32)]) float32, accumulated into
        the given tensors if any (d_params="scene": the scene's own buffer)."""
        dev = torch.device("cuda", self.ctx.device)
        own = isinstance(d_params, str) and d_params == "scene"
        if own:
            d_params = self.grads_view()
        elif d_params is None:
            d_params = torch.zeros((self.n, 32), dtype=torch.float32, device=dev)
        if actor_d_params is None:
            actor_d_params = [torch.zeros((a[0].n, 32), dtype=torch.float32, device=dev)
                              for a in actors]

        def ptr(t):
            return None if t is None else t.contiguous().data_ptr()

        keep = [t.contiguous() for t in (d_rgb, d_depth, d_opacity, d_intensity) if t is not None]
        arr = (L.Actor * max(1, len(actors)))()
        for k, (sc, p0, p1, base) in enumerate(actors):
            arr[k].actor = sc._h
            arr[k].pose0[:] = [float(v) for v in np.asarray(p0, dtype=np.float64).ravel()]
            arr[k].pose1[:] = [float(v) for v in np.asarray(p1, dtype=np.float64).ravel()]
            arr[k].id_base = int(base)
        aptr = (C.c_void_p * max(1, len(actors)))(*[ptr(t) for t in actor_d_params])
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, 0)
        L.check(L.load().salf_render_backward_actors(
            self._h, arr, len(actors), C.byref(s), C.byref(op), saved.data_ptr(), ptr(d_rgb),
            ptr(d_depth), ptr(d_opacity), ptr(d_intensity), None if own else d_params.data_ptr(),
            C.cast(aptr, C.c_void_p), _stream_ptr(stream)),
            "salf_render_backward_actors")
        return d_params, actor_d_params


class RenderFn(torch.autograd.Function):
    """Differentiable render: (params) -> (rgb, depth, opacity).

    forward uploads `params` (n x 32 FP32, input order) into the scene (in
    the scene's storage dtype) and renders with saved per-ray totals; backward
    runs the hand-written adjoint kernel and returns dL/dparams."""

    @staticmethod
    def forward(ctx, params, scene: Scene, sensor: dict, t_min: float = 1e-4,
                background=(0.0, 0.0, 0.0)):
        scene.update_params(params)
        out = scene.render(sensor, t_min=t_min, background=background, saved=True,
                           outputs=("rgb", "depth", "opacity"))
        ctx.scene, ctx.sensor, ctx.t_min, ctx.background = scene, sensor, t_min, background
        ctx.save_for_backward(out["saved"])
        return out["rgb"], out["depth"], out["opacity"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_opacity):
        # accumulate into the scene's own gradient buffer (salf_scene_params),
        # then hand autograd a copy it may keep
        (saved,) = ctx.saved_tensors
        own = ctx.scene.grads_view()
        own.zero_()
        ctx.scene.backward(ctx.sensor, saved, d_rgb=g_rgb, d_depth=g_depth, d_opacity=g_opacity,
                           t_min=ctx.t_min, background=ctx.background, d_params="scene")
        return own.clone(), None, None, None, None


class RenderBatchFn(torch.autograd.Function):
    """Differentiable render of several sensors in one launch each way:
    (params) -> (rgb_0, depth_0, opacity_0, rgb_1, ...).  forward uploads
    `params` into the scene and calls salf_render_rays_batch; backward calls
    salf_render_backward_batch into the scene's own gradient buffer and hands
    autograd a copy."""

    @staticmethod
    def forward(ctx, params, scene: Scene, sensors, t_min: float = 1e-4,
                background=(0.0, 0.0, 0.0)):
        scene.update_params(params)
        outs = scene.render_batch(sensors, t_min=t_min, background=background, saved=True,
                                  outputs=("rgb", "depth", "opacity"))
        ctx.scene, ctx.sensors, ctx.t_min, ctx.background = scene, sensors, t_min, background
        ctx.save_for_backward(*[o["saved"] for o in outs])
        return tuple(t for o in outs for t in (o["rgb"], o["depth"], o["opacity"]))

    @staticmethod
    def backward(ctx, *grads):
        saved = list(ctx.saved_tensors)
        own = ctx.scene.grads_view()
        own.zero_()
        ctx.scene.backward_batch(ctx.sensors, saved, d_rgb=list(grads[0::3]),
                                 d_depth=list(grads[1::3]), d_opacity=list(grads[2::3]),
                                 t_min=ctx.t_min, background=ctx.background, d_params="scene")
        return own.clone(), None, None, None, None


class HostFrames:
    """Frames of one sensor shape delivered to page-locked host memory with
    `depth` frames in flight: each frame renders into its own device buffers on
    a render stream (salf_render_rays), and the copy engine moves the previous
    frame's outputs to the host on a copy stream meanwhile.  submit() returns a
    slot; result(slot) waits for that frame and returns its host tensors, which
    stay valid until the slot is submitted again (every `depth` frames)."""

    def __init__(self, scene: Scene, sensor: dict, outputs=("rgb", "depth", "opacity"),
                 depth: int = 2, t_min=1e-4, background=(0.0, 0.0, 0.0), want_intensity=False):
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.scene, self.outputs, self.depth = scene, tuple(outputs), depth
        self.kw = dict(t_min=t_min, background=background, want_intensity=want_intensity)
        R = n_rays(sensor)
        shape = lambda k: (R, 3) if k == "rgb" else (R,)
        dev = scene.ctx.device
        self.dev = [{k: torch.empty(shape(k), device=f"cuda:{dev}") for k in self.outputs}
                    for _ in range(depth)]
        self.host = [{k: torch.empty(shape(k), pin_memory=True) for k in self.outputs}
                     for _ in range(depth)]
        self.render_stream = torch.cuda.Stream(device=dev)
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.rendered = [torch.cuda.Event() for _ in range(depth)]
        self.copied = [torch.cuda.Event() for _ in range(depth)]
        self.used = [False] * depth
        self.n = 0

    def submit(self, sensor: dict) -> int:
        b = self.n % self.depth
        self.n += 1
        if self.used[b]:  # the copy that last read these device buffers has run
            self.render_stream.wait_event(self.copied[b])
        self.scene.render(sensor, out=self.dev[b], outputs=self.outputs, valid=False,
                          stream=self.render_stream, **self.kw)
        self.rendered[b].record(self.render_stream)
        self.copy_stream.wait_event(self.rendered[b])
        with torch.cuda.stream(self.copy_stream):
            for k in self.outputs:
                self.host[b][k].copy_(self.dev[b][k], non_blocking=True)
        self.copied[b].record(self.copy_stream)
        self.used[b] = True
        return b

    def result(self, slot: int) -> dict:
        self.copied[slot].synchronize()
        return self.host[slot]


class Server:
    """Continuous-batching render server (salf_serve_*)."""

    def __init__(self, scene: Scene, mem_budget_bytes: int, n_streams: int = 2):
        h = C.c_void_p()
        L.check(L.load().salf_serve_create(scene._h, int(mem_budget_bytes), int(n_streams),
                                           C.byref(h)), "salf_serve_create")
        self._h = h
        self.scene = scene
        self._sensors: dict = {}

    def submit(self, sensor: dict, t_min=1e-4, background=(0.0, 0.0, 0.0),
               want_intensity=False, ray_segments: int = 0) -> int:
        keep: list = []
        s = sensor_struct(sensor, keep)
        op = opts_struct(t_min, background, want_intensity, 0, ray_segments)
        t = C.c_uint64()
        L.check(L.load().salf_serve_submit(self._h, C.byref(s), C.byref(op), C.byref(t)),
                "salf_serve_submit")
        self._sensors[t.value] = (sensor, keep)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Returns None if not done within timeout_ms, else a dict of raw
        device pointers {rgb, depth, opacity, intensity, valid} (library-owned)."""
        o = L.Outputs()
        done = L.c_int32()
        st = L.load().salf_serve_poll(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(o),
                                      C.byref(done))
        if st == L.ERR_TIMEOUT:
            return None
        L.check(st, "salf_serve_poll")
        return {k: getattr(o, k) for k in ("rgb", "depth", "opacity", "intensity", "valid")}

    def fetch(self, ticket: int, timeout_ms: int = -1, copy: bool = True) -> dict | None:
        """poll + tensors over the results (copies unless copy=False, in which
        case the views are valid until release)."""
        ptrs = self.poll(ticket, timeout_ms)
        if ptrs is None:
            return None
        sensor = self._sensors[ticket][0]
        R = n_rays(sensor)
        res = {}
        for k, shape, ts in (("rgb", (R, 3), "<f4"), ("depth", (R,), "<f4"),
                             ("opacity", (R,), "<f4"), ("intensity", (R,), "<f4"),
                             ("valid", (R,), "|u1")):
            if ptrs[k]:
                t = device_view(ptrs[k], shape, ts)
                res[k] = t.clone() if copy else t
        return res

    def release(self, ticket: int):
        L.check(L.load().salf_serve_release(self._h, C.c_uint64(ticket)), "salf_serve_release")
        self._sensors.pop(ticket, None)

    def hold(self, on: bool = True):
        """salf_serve_hold: while held, submitted requests wait; releasing the
        hold starts them together."""
        L.check(L.load().salf_serve_hold(self._h, int(bool(on))), "salf_serve_hold")

    def stats(self) -> dict:
        s = L.ServeStats()
        L.check(L.load().salf_serve_get_stats(self._h, C.byref(s)), "salf_serve_get_stats")
        return {k: getattr(s, k) for k, _ in L.ServeStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            L.load().salf_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevBuf:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2,
                                         "strides": None}


def device_view(ptr: int, shape, typestr: str) -> torch.Tensor:
    """Zero-copy torch view of library-owned device memory."""
    return torch.as_tensor(_DevBuf(ptr, shape, typestr), device="cuda")
