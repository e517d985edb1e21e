"""ctypes binding of the C oracle (salf_oracle.c).  Test infrastructure only."""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "salf_oracle.c")
_HDR = os.path.join(_HERE, "salf_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libsalf_oracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"pinhole": 0, "fisheye": 1, "pano": 2, "lidar": 3, "explicit": 4}


def library_path() -> str:
    return _OUT


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = (not os.path.exists(_OUT) or
             os.path.getmtime(_OUT) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


class _SceneDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("origin", C.c_double * 3), ("s0", C.c_double),
                ("dims", C.c_int32 * 3), ("max_level", C.c_int32), ("mode", C.c_int32),
                ("level", C.c_void_p), ("ijk", C.c_void_p), ("params", C.c_void_p)]


class _Sensor(C.Structure):
    _fields_ = [("kind", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("fov", C.c_double), ("elev_min", C.c_double), ("elev_max", C.c_double),
                ("pose0", C.c_double * 12), ("pose1", C.c_double * 12), ("t0", C.c_double),
                ("t1", C.c_double), ("rolling_shutter", C.c_int32), ("t_near", C.c_double),
                ("t_far", C.c_double), ("rays", C.c_void_p), ("rays64", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("t_min", C.c_double), ("background", C.c_double * 3),
                ("want_intensity", C.c_int32), ("brute_force", C.c_int32),
                ("want_raydrop", C.c_int32)]


class _Outputs(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("opacity", C.c_void_p),
                ("intensity", C.c_void_p), ("t_end", C.c_void_p), ("term_gap", C.c_void_p),
                ("n_visits", C.c_void_p), ("valid", C.c_void_p), ("visits", C.c_void_p),
                ("visits_cap", C.c_int32), ("max_alpha", C.c_void_p), ("raydrop", C.c_void_p)]


class _Actor(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("pose0", C.c_double * 12), ("pose1", C.c_double * 12),
                ("id_base", C.c_int32)]


class _Hit(C.Structure):
    _fields_ = [("voxel", C.c_int32), ("t_in", C.c_double), ("t_out", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_OUT)
            vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            lib.orc_scene_create.argtypes = [C.POINTER(_SceneDesc), C.POINTER(vp)]
            lib.orc_scene_create.restype = C.c_int
            lib.orc_scene_free.argtypes = [vp]
            lib.orc_scene_lookup.argtypes = [vp, i32, i32, i32, i32]
            lib.orc_scene_lookup.restype = i64
            lib.orc_gen_rays.argtypes = [C.POINTER(_Sensor), vp, i64, vp, vp, vp, vp, vp, vp]
            lib.orc_pose_at.argtypes = [C.POINTER(_Sensor), dp, vp, vp]
            lib.orc_sh_basis.argtypes = [vp, vp]
            lib.orc_field.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            lib.orc_trace.argtypes = [vp, vp, vp, dp, dp, i32, vp, i64]
            lib.orc_trace.restype = i64
            lib.orc_trace_eps.argtypes = [vp, vp, vp, dp, dp, dp, dp, i32, vp, vp, vp, i64]
            lib.orc_trace_eps.restype = i64
            lib.orc_render.argtypes = [vp, C.POINTER(_Sensor), C.POINTER(_Opts), vp, i64,
                                       C.POINTER(_Outputs)]
            lib.orc_backward.argtypes = [vp, C.POINTER(_Sensor), C.POINTER(_Opts), vp, i64, vp,
                                         vp, vp, vp, vp, vp]
            lib.orc_backward_bound.argtypes = lib.orc_backward.argtypes
            lib.orc_scene_set_record.argtypes = [vp, i64, vp]
            lib.orc_conditioned.argtypes = [vp, C.POINTER(_Sensor), vp, i64, dp, dp, vp]
            lib.orc_backward_actors.argtypes = [vp, vp, i32, C.POINTER(_Sensor), C.POINTER(_Opts),
                                                vp, i64, vp, vp, vp, vp, vp, vp]
            lib.orc_backward_actors_bound.argtypes = lib.orc_backward_actors.argtypes
            lib.orc_num_threads.restype = C.c_int
            lib.orc_subdivide_record.argtypes = [vp, i32, vp]
            lib.orc_render_actors.argtypes = [vp, vp, i32, C.POINTER(_Sensor), C.POINTER(_Opts),
                                              vp, i64, C.POINTER(_Outputs)]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def num_threads() -> int:
    return int(_load().orc_num_threads())


class OracleScene:
    """A scene held by the oracle (FP64 copy of the records)."""

    def __init__(self, scene, params=None):
        lib = _load()
        p = scene.params if params is None else params
        self._level = np.ascontiguousarray(scene.level, dtype=np.uint8)
        self._ijk = np.ascontiguousarray(scene.ijk, dtype=np.int32)
        self._params = np.ascontiguousarray(p, dtype=np.float64)
        self.n = int(self._level.shape[0])
        self.mode = scene.mode
        self.origin = np.asarray(scene.origin, dtype=np.float64)
        self.s0 = float(scene.s0)
        self.dims = tuple(int(v) for v in scene.dims)
        self.max_level = int(scene.max_level)
        d = _SceneDesc()
        d.n = self.n
        d.origin[:] = [float(v) for v in scene.origin]
        d.s0 = float(scene.s0)
        d.dims[:] = [int(v) for v in scene.dims]
        d.max_level = int(scene.max_level)
        d.mode = 0 if scene.mode == "exp" else 1
        d.level, d.ijk, d.params = _ptr(self._level), _ptr(self._ijk), _ptr(self._params)
        h = C.c_void_p()
        self.status = lib.orc_scene_create(C.byref(d), C.byref(h))
        self._h = h if self.status == 0 else None

    @property
    def ok(self):
        return self._h is not None

    def set_record(self, v: int, rec) -> None:
        """Replace voxel v's 32 record scalars (input order), e.g. for finite
        differences."""
        r = np.ascontiguousarray(np.asarray(rec, dtype=np.float64).reshape(32))
        if _load().orc_scene_set_record(self._h, int(v), _ptr(r)) != 0:
            raise ValueError(f"set_record({v}) rejected")
        self._params[int(v)] = r

    def close(self):
        if self._h is not None:
            _load().orc_scene_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lookup(self, level, i, j, k) -> int:
        return int(_load().orc_scene_lookup(self._h, level, i, j, k))


def _sensor(s):
    c = _Sensor()
    c.kind = KIND[s["kind"]]
    c.width, c.height = int(s["width"]), int(s["height"])
    c.fx, c.fy, c.cx, c.cy = (float(s[k]) for k in ("fx", "fy", "cx", "cy"))
    c.fov, c.elev_min, c.elev_max = float(s["fov"]), float(s["elev_min"]), float(s["elev_max"])
    c.pose0[:] = [float(v) for v in np.asarray(s["pose0"], dtype=np.float64).ravel()]
    c.pose1[:] = [float(v) for v in np.asarray(s["pose1"], dtype=np.float64).ravel()]
    c.t0, c.t1 = float(s["t0"]), float(s["t1"])
    c.rolling_shutter = int(bool(s["rolling_shutter"]))
    c.t_near, c.t_far = float(s["t_near"]), float(s["t_far"])
    keep = None
    if s["kind"] == "explicit":
        if np.asarray(s["rays"]).dtype == np.float64:
            keep = np.ascontiguousarray(s["rays"], dtype=np.float64)
            c.rays64 = keep.ctypes.data
        else:
            keep = np.ascontiguousarray(s["rays"], dtype=np.float32)
            c.rays = keep.ctypes.data
    return c, keep


def _opts(t_min=1e-4, background=(0.0, 0.0, 0.0), want_intensity=False, brute_force=False,
          want_raydrop=False):
    o = _Opts()
    o.t_min = float(t_min)
    o.background[:] = [float(v) for v in background]
    o.want_intensity = int(bool(want_intensity))
    o.brute_force = int(bool(brute_force))
    o.want_raydrop = int(bool(want_raydrop))
    return o


def _idx(sensor, idx):
    R = int(sensor["width"]) * int(sensor["height"])
    if idx is None:
        return None, R
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    assert idx.size == 0 or (idx.min() >= 0 and idx.max() < R)
    return idx, int(idx.size)


def gen_rays(sensor, idx=None):
    lib = _load()
    s, keep = _sensor(sensor)
    idx, m = _idx(sensor, idx)
    o = np.zeros((m, 3)); d = np.zeros((m, 3)); tn = np.zeros(m); tf = np.zeros(m)
    tau = np.zeros(m); valid = np.zeros(m, np.uint8)
    lib.orc_gen_rays(C.byref(s), _ptr(idx), m, _ptr(o), _ptr(d), _ptr(tn), _ptr(tf), _ptr(tau),
                     _ptr(valid))
    del keep
    return dict(o=o, d=d, t_near=tn, t_far=tf, tau=tau, valid=valid.astype(bool))


def pose_at(sensor, tau):
    s, keep = _sensor(sensor)
    R = np.zeros(9); t = np.zeros(3)
    _load().orc_pose_at(C.byref(s), float(tau), _ptr(R), _ptr(t))
    return R.reshape(3, 3), t


def sh_basis(direction):
    d = np.ascontiguousarray(direction, dtype=np.float64)
    g = np.zeros(4)
    _load().orc_sh_basis(_ptr(d), _ptr(g))
    return g


def field(record, mode, x, direction):
    rec = np.ascontiguousarray(record, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    d = np.ascontiguousarray(direction, dtype=np.float64)
    sig = np.zeros(1); c = np.zeros(3); io = np.zeros(1)
    _load().orc_field(_ptr(rec), 0 if mode == "exp" else 1, _ptr(x), _ptr(d), _ptr(sig), _ptr(c),
                      _ptr(io))
    return float(sig[0]), c, float(io[0])


def trace(oscene, o, d, t_near=0.0, t_far=np.inf, brute_force=False, cap=1 << 16):
    """Hits of one ray: list of (voxel, t_in, t_out), sorted by entry."""
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    hits = (_Hit * cap)()
    n = _load().orc_trace(oscene._h, _ptr(o), _ptr(d), float(t_near), float(t_far),
                          int(bool(brute_force)), C.cast(hits, C.c_void_p), cap)
    return [(hits[i].voxel, hits[i].t_in, hits[i].t_out) for i in range(min(n, cap))]


def trace_eps(oscene, o, d, t_near, t_far, eps_abs, eps_rel, sign, cap=1 << 16,
              intervals=False):
    """Voxels hit when every box is grown (sign=+1) / shrunk (-1) by
    eps_abs + eps_rel * distance; ids sorted by entry (and the perturbed
    [t_in, t_out] per id if intervals)."""
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    ids = np.zeros(cap, np.int32)
    ti = np.zeros(cap)
    to = np.zeros(cap)
    n = _load().orc_trace_eps(oscene._h, _ptr(o), _ptr(d), float(t_near), float(t_far),
                              float(eps_abs), float(eps_rel), int(sign), _ptr(ids), _ptr(ti),
                              _ptr(to), cap)
    n = min(n, cap)
    if intervals:
        return ids[:n].tolist(), ti[:n], to[:n]
    return ids[:n].tolist()


def conditioned(oscene, sensor, eps_abs, eps_rel, idx=None):
    """Per ray: True if its visit list is the same for every voxel box shrunk
    and grown by eps_abs + eps_rel * distance (metres)."""
    lib = _load()
    s, keep = _sensor(sensor)
    idx, m = _idx(sensor, idx)
    ok = np.zeros(m, np.uint8)
    lib.orc_conditioned(oscene._h, C.byref(s), _ptr(idx), m, float(eps_abs), float(eps_rel),
                        _ptr(ok))
    del keep
    return ok.astype(bool)


def render(oscene, sensor, idx=None, t_min=1e-4, background=(0.0, 0.0, 0.0),
           want_intensity=False, brute_force=False, visits_cap=0, max_alpha=None,
           want_raydrop=False):
    """Render the selected rays (all if idx is None) in FP64.  `max_alpha`
    (n float64, input order) is max-accumulated with each voxel's largest
    composited alpha.  want_raydrop adds `raydrop`: sum of w * sigmoid(rho)
    over the composited voxels (rho = record slot 31) plus T_end."""
    lib = _load()
    s, keep = _sensor(sensor)
    idx, m = _idx(sensor, idx)
    o = _Outputs()
    res = dict(rgb=np.zeros((m, 3)), depth=np.zeros(m), opacity=np.zeros(m),
               intensity=np.zeros(m), t_end=np.zeros(m), term_gap=np.zeros(m),
               n_visits=np.zeros(m, np.int32), valid=np.zeros(m, np.uint8))
    for k, v in res.items():
        setattr(o, k, _ptr(v))
    if visits_cap > 0:
        res["visits"] = np.full((m, visits_cap), -1, np.int32)
        o.visits = _ptr(res["visits"])
        o.visits_cap = int(visits_cap)
    if max_alpha is not None:
        assert max_alpha.dtype == np.float64 and max_alpha.flags.c_contiguous
        o.max_alpha = _ptr(max_alpha)
    if want_raydrop:
        res["raydrop"] = np.zeros(m)
        o.raydrop = _ptr(res["raydrop"])
    opt = _opts(t_min, background, want_intensity, brute_force, want_raydrop)
    st = lib.orc_render(oscene._h, C.byref(s), C.byref(opt), _ptr(idx), m, C.byref(o))
    if st != 0:
        raise RuntimeError(f"oracle render failed: {st}")
    del keep
    res["valid"] = res["valid"].astype(bool)
    return res


def backward(oscene, sensor, g_rgb=None, g_depth=None, g_opacity=None, g_intensity=None,
             idx=None, t_min=1e-4, background=(0.0, 0.0, 0.0), want_intensity=False,
             brute_force=False, g_raydrop=None, bound=False):
    """Gradient (n, 32) of sum(g . outputs) w.r.t. every record scalar.  With
    bound=True, returns (gradient, rounding bound): the per-scalar magnitude
    sum of orc_backward_bound, which an FP32 evaluation is compared against."""
    lib = _load()
    s, keep = _sensor(sensor)
    idx, m = _idx(sensor, idx)
    grad = np.zeros((oscene.n, 32))

    def arr(a, shape):
        if a is None:
            return None
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))

    gr, gd, go, gi = arr(g_rgb, (m, 3)), arr(g_depth, (m,)), arr(g_opacity, (m,)), arr(g_intensity, (m,))
    gp = arr(g_raydrop, (m,))
    opt = _opts(t_min, background, want_intensity, brute_force, g_raydrop is not None)
    st = lib.orc_backward(oscene._h, C.byref(s), C.byref(opt), _ptr(idx), m, _ptr(gr), _ptr(gd),
                          _ptr(go), _ptr(gi), _ptr(gp), _ptr(grad))
    if st != 0:
        raise RuntimeError(f"oracle backward failed: {st}")
    if bound:
        bnd = np.zeros((oscene.n, 32))
        st = lib.orc_backward_bound(oscene._h, C.byref(s), C.byref(opt), _ptr(idx), m, _ptr(gr),
                                    _ptr(gd), _ptr(go), _ptr(gi), _ptr(gp), _ptr(bnd))
        if st != 0:
            raise RuntimeError(f"oracle backward bound failed: {st}")
        del keep
        return grad, bnd
    del keep
    return grad


def render_actors(oscene, actors, sensor, idx=None, t_min=1e-4, background=(0.0, 0.0, 0.0),
                  want_intensity=False, brute_force=False, visits_cap=0):
    """Render with dynamic actors (Sec. IV-A) in FP64.  `actors`: list of
    (OracleScene, pose0, pose1, id_base); poses are 3x4 canonical -> world at
    the sensor's t0 / t1."""
    lib = _load()
    s, keep = _sensor(sensor)
    idx, m = _idx(sensor, idx)
    arr = (_Actor * max(1, len(actors)))()
    for k, (osc, p0, p1, base) in enumerate(actors):
        arr[k].scene = osc._h
        arr[k].pose0[:] = [float(v) for v in np.asarray(p0, dtype=np.float64).ravel()]
        arr[k].pose1[:] = [float(v) for v in np.asarray(p1, dtype=np.float64).ravel()]
        arr[k].id_base = int(base)
    o = _Outputs()
    res = dict(rgb=np.zeros((m, 3)), depth=np.zeros(m), opacity=np.zeros(m),
               intensity=np.zeros(m), t_end=np.zeros(m), term_gap=np.zeros(m),
               n_visits=np.zeros(m, np.int32), valid=np.zeros(m, np.uint8))
    for k, v in res.items():
        setattr(o, k, _ptr(v))
    if visits_cap > 0:
        res["visits"] = np.full((m, visits_cap), -1, np.int32)
        o.visits = _ptr(res["visits"])
        o.visits_cap = int(visits_cap)
    opt = _opts(t_min, background, want_intensity, brute_force)
    st = lib.orc_render_actors(oscene._h, C.cast(arr, C.c_void_p), len(actors), C.byref(s),
                               C.byref(opt), _ptr(idx), m, C.byref(o))
    if st != 0:
        raise RuntimeError(f"oracle actor render failed: {st}")
    del keep
    res["valid"] = res["valid"].astype(bool)
    return res


def backward_actors(oscene, actors, sensor, g_rgb=None, g_depth=None, g_opacity=None,
                    g_intensity=None, idx=None, t_min=1e-4, background=(0.0, 0.0, 0.0),
                    want_intensity=False, brute_force=False, bound=False):
    """Adjoint of render_actors: (static gradient (n, 32), [actor k's gradient
    (n_k, 32)]) of sum(g . outputs) w.r.t. every record scalar.  With
    bound=True, also the FP32 rounding bounds, in the same shapes."""
    lib = _load()
    s, keep = _sensor(sensor)
    idx, m = _idx(sensor, idx)
    arr = (_Actor * max(1, len(actors)))()
    for k, (osc, p0, p1, base) in enumerate(actors):
        arr[k].scene = osc._h
        arr[k].pose0[:] = [float(v) for v in np.asarray(p0, dtype=np.float64).ravel()]
        arr[k].pose1[:] = [float(v) for v in np.asarray(p1, dtype=np.float64).ravel()]
        arr[k].id_base = int(base)

    def arrg(a, shape):
        if a is None:
            return None
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))

    gr, gd = arrg(g_rgb, (m, 3)), arrg(g_depth, (m,))
    go, gi = arrg(g_opacity, (m,)), arrg(g_intensity, (m,))
    opt = _opts(t_min, background, want_intensity, brute_force)
    out = []
    for fn in ([lib.orc_backward_actors] + ([lib.orc_backward_actors_bound] if bound else [])):
        g = np.zeros((oscene.n, 32))
        ag = [np.zeros((a[0].n, 32)) for a in actors]
        ptrs = (C.c_void_p * max(1, len(actors)))(*[a.ctypes.data for a in ag])
        st = fn(oscene._h, C.cast(arr, C.c_void_p), len(actors), C.byref(s), C.byref(opt),
                _ptr(idx), m, _ptr(gr), _ptr(gd), _ptr(go), _ptr(gi), _ptr(g),
                C.cast(ptrs, C.c_void_p))
        if st != 0:
            raise RuntimeError(f"oracle actor backward failed: {st}")
        out.append((g, ag))
    del keep
    return out if bound else out[0]


def voxel_at(oscene, X) -> int:
    """Index of the voxel whose box [lo, lo + edge) holds the point X (world
    metres), else -1.  The voxels are disjoint (Sec. III-D), so the cell
    holding X is looked up at each level and at most one level matches."""
    X = np.asarray(X, dtype=np.float64)
    for lev in range(oscene.max_level + 1):
        e = oscene.s0 / (1 << lev)
        c = np.floor((X - oscene.origin) / e).astype(np.int64)
        if (c < 0).any() or (c >= np.asarray(oscene.dims, np.int64) << lev).any():
            return -1
        v = oscene.lookup(lev, int(c[0]), int(c[1]), int(c[2]))
        if v >= 0:
            return v
    return -1


def secondary_rays(oscene, sensor, depth, opacity, kind="reflect", eta=1.0 / 1.33,
                   light_dir=(0.0, 0.0, 1.0), min_opacity=0.5, offset=1e-3, t_far=0.0, idx=None):
    """Secondary rays at the expected hit point of a render (Sec. V-C and
    Fig. 1 name reflection, refraction and shadows; the paper gives no
    construction, so this follows the library's stated one), in FP64:
    X = o + (D / O) d for rays with O >= min_opacity; the voxel holding X; its
    outward normal n = -W[0:3] / |W[0:3]|, turned so that n . d <= 0; then the
    mirror direction d - 2 (d . n) n, Snell's refraction with ratio eta (total
    internal reflection falls back to the mirror direction), or the unit light
    direction.  Rows (origin, direction, 0, t_far); no ray -> all zero."""
    r = gen_rays(sensor, idx)
    depth = np.asarray(depth, dtype=np.float64).ravel()
    opacity = np.asarray(opacity, dtype=np.float64).ravel()
    light = np.asarray(light_dir, dtype=np.float64)
    light = light / np.linalg.norm(light)
    out = np.zeros((len(r["o"]), 8))
    for i in range(len(r["o"])):
        O = opacity[i]
        if not r["valid"][i] or not (O >= min_opacity and O > 0.0):
            continue
        d = r["d"][i]
        X = r["o"][i] + (depth[i] / O) * d
        v = voxel_at(oscene, X)
        if v < 0:
            continue
        g = oscene._params[v, :3]
        gn = np.linalg.norm(g)
        if gn == 0.0:
            continue
        n = -g / gn
        if n @ d > 0.0:
            n = -n
        dn = n @ d
        side = 1.0
        if kind == "shadow":
            w = light
        else:
            c = -dn
            k = 1.0 - eta * eta * (1.0 - c * c)
            if kind == "refract" and k >= 0.0:
                w = eta * d + (eta * c - np.sqrt(k)) * n
                side = -1.0
            else:
                w = d - 2.0 * dn * n
        out[i, :3] = X + side * offset * n
        out[i, 3:6] = w
        out[i, 7] = t_far if t_far > 0.0 else 0.0
    return out


def subdivide_record(record, child):
    """Record of child `child` (0..7) of a voxel split in 8 (Sec. III-C)."""
    rec = np.ascontiguousarray(record, dtype=np.float64)
    out = np.zeros(32)
    _load().orc_subdivide_record(_ptr(rec), int(child), _ptr(out))
    return out


def refine(scene, grads, max_alpha, split_threshold, prune_alpha=1e-3):
    """Densify and prune (Sec. III-C) a voxel set: a voxel whose largest
    composited alpha is below prune_alpha is removed; otherwise a voxel below
    the finest level whose colour-field gradient L1 norm (record slots 4..12)
    exceeds split_threshold becomes its 8 children (order 0..7, bits x | y << 1
    | z << 2) carrying its fields; the rest are kept.  Output in input order,
    children in place of their parent.  Returns (level, ijk, params, actions)
    with actions 0 keep, 1 split, 2 prune."""
    level = np.asarray(scene.level).astype(np.int64)
    ijk = np.asarray(scene.ijk).astype(np.int64)
    params = np.asarray(scene.params, dtype=np.float64)
    g1 = np.abs(np.asarray(grads, dtype=np.float64)[:, 4:13]).sum(axis=1)
    ma = np.asarray(max_alpha, dtype=np.float64)
    act = np.zeros(len(level), np.int32)
    act[(level < scene.max_level) & (g1 > split_threshold)] = 1
    act[ma < prune_alpha] = 2
    lv, ij, pr = [], [], []
    for v in range(len(level)):
        if act[v] == 0:
            lv.append(level[v]); ij.append(ijk[v]); pr.append(params[v])
        elif act[v] == 1:
            for c in range(8):
                off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
                lv.append(level[v] + 1); ij.append(2 * ijk[v] + off)
                pr.append(subdivide_record(params[v], c))
    return (np.array(lv, np.uint8), np.array(ij, np.int32).reshape(-1, 3),
            np.array(pr, np.float64).reshape(-1, 32), act)


def _density_and_grad(g, rec, mode):
    """sigma(g) and d sigma / d(g, a, b) for the geometry value g (Eq. 1 / Eq. 6)."""
    if mode == "exp":
        s = np.exp(g)
        return s, s, 0.0, 0.0
    a, b = rec[25], rec[26]
    e = np.exp(-abs(g) / b)
    sg = np.sign(g)
    s = 0.5 * a + 0.5 * a * sg * (1.0 - e)
    ds_dg = 0.5 * a * e / b
    ds_da = s / a
    ds_db = -0.5 * a * g * e / (b * b)
    return s, ds_dg, ds_da, ds_db


def face_pairs(scene):
    """Face-adjacent voxel pairs (positive contact area), brute force:
    list of (i, j, axis, sign) with voxel j on the `sign` side of voxel i
    along `axis`, i no larger than j (one entry per pair)."""
    K = scene.max_level
    lvl = np.asarray(scene.level).astype(np.int64)
    e = (1 << (K - lvl)).astype(np.int64)                       # edges in finest cells
    lo = np.asarray(scene.ijk).astype(np.int64) * e[:, None]
    hi = lo + e[:, None]
    out = []
    n = len(lvl)
    for i in range(n):
        for j in range(n):
            if i == j or e[j] < e[i] or (e[j] == e[i] and j < i):
                continue
            for a in range(3):
                o = [b for b in range(3) if b != a]
                area = all(min(hi[i, b], hi[j, b]) > max(lo[i, b], lo[j, b]) for b in o)
                if not area:
                    continue
                if hi[i, a] == lo[j, a]:
                    out.append((i, j, a, +1))
                elif lo[i, a] == hi[j, a]:
                    out.append((i, j, a, -1))
    return out


def reg_loss(scene, params, lam_s, lam_alpha, lam_n):
    """Eq. 7's L_reg and its gradient w.r.t. the records (n x 32), over the
    face-adjacent pairs (i, j): lam_s |s_i - s_j| + lam_alpha |alpha_i -
    alpha_j| + lam_n (1 - n_i . n_j), where, at the centre X of the shared face
    (the smaller voxel's face): s_k = W_k . [x_k(X), 1] (record slots 0..3),
    alpha_k = 1 - exp(-sigma_k(s_k) l) with l the smaller voxel's edge (m), and
    n_k = W_k[0:3] / |W_k[0:3]| (0 if that is 0)."""
    K = scene.max_level
    sfin = scene.s0 / (1 << K)
    lvl = np.asarray(scene.level).astype(np.int64)
    e = (1 << (K - lvl)).astype(np.int64)
    lo = np.asarray(scene.ijk).astype(np.int64) * e[:, None]
    P = np.asarray(params, dtype=np.float64)
    grad = np.zeros_like(P)
    loss = 0.0
    for i, j, a, sgn in face_pairs(scene):
        X = lo[i] + 0.5 * e[i]
        X = X.astype(np.float64)
        X[a] += 0.5 * e[i] * sgn                               # centre of i's face towards j
        xs, ss, sig, dsg = [], [], [], []
        for k in (i, j):
            x = (X - (lo[k] + 0.5 * e[k])) / (0.5 * e[k])
            s = P[k, :3] @ x + P[k, 3]
            xs.append(x)
            ss.append(s)
            sk, ds_dg, ds_da, ds_db = _density_and_grad(s, P[k], scene.mode)
            sig.append(sk)
            dsg.append((ds_dg, ds_da, ds_db))
        ell = e[i] * sfin
        # s term
        d = ss[0] - ss[1]
        loss += lam_s * abs(d)
        for k, x, sg in ((i, xs[0], 1.0), (j, xs[1], -1.0)):
            grad[k, :3] += lam_s * np.sign(d) * sg * x
            grad[k, 3] += lam_s * np.sign(d) * sg
        # alpha term
        al = [1.0 - np.exp(-sig[q] * ell) for q in (0, 1)]
        da = al[0] - al[1]
        loss += lam_alpha * abs(da)
        for q, k, sg in ((0, i, 1.0), (1, j, -1.0)):
            dal_dsig = np.exp(-sig[q] * ell) * ell
            c = lam_alpha * np.sign(da) * sg * dal_dsig
            ds_dg, ds_da, ds_db = dsg[q]
            grad[k, :3] += c * ds_dg * xs[q]
            grad[k, 3] += c * ds_dg
            if scene.mode == "sdf":
                grad[k, 25] += c * ds_da
                grad[k, 26] += c * ds_db
        # normal term
        w = [P[i, :3], P[j, :3]]
        nn = [np.linalg.norm(v) for v in w]
        nv = [w[q] / nn[q] if nn[q] > 0 else np.zeros(3) for q in (0, 1)]
        loss += lam_n * (1.0 - nv[0] @ nv[1])
        for q, k in ((0, i), (1, j)):
            if nn[q] > 0:
                other = nv[1 - q]
                # d(n . m)/dw = (m - n (n . m)) / |w|
                grad[k, :3] += -lam_n * (other - nv[q] * (nv[q] @ other)) / nn[q]
    return loss, grad
