"""Secondary rays on the GPU (salf_secondary_rays, then the ray kernel over the
spawned explicit rays) against the FP64 oracle.

Generation: both sides start from the same primary depth / opacity (the GPU
render's), so the only differences are FP32 ray geometry: the rays must agree
element by element except where the construction is ill-conditioned (hit
point within rounding of a voxel face, grazing normal, refraction at the
critical angle), and those must stay rare.  Tracing: the GPU-spawned rays,
rendered by the GPU and by the oracle, must match within the tolerances."""

import numpy as np
import pytest

import synth
from tests.parity_util import compare_outputs, oracle_sensitivity, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def _ambiguous(oracle_lib, osc, sc, sensor, depth, opac, kind, eta, min_opacity, idx=None):
    """Rays whose secondary ray the FP32 and FP64 sides may legitimately
    construct differently."""
    r = oracle_lib.gen_rays(sensor, idx)
    sf = sc.s0 / (1 << sc.max_level)
    amb = np.zeros(len(depth), bool)
    for i in range(len(depth)):
        O = float(opac[i])
        if not r["valid"][i] or O <= 0:
            continue
        if abs(O - min_opacity) < 1e-6:
            amb[i] = True
            continue
        if O < min_opacity:
            continue
        ts = float(depth[i]) / O
        X = r["o"][i] + ts * r["d"][i]
        v = oracle_lib.voxel_at(osc, X)
        # within FP32 rounding of a boundary between two voxels (or a voxel
        # and empty space): the two sides may pick either
        delta = 1e-6 * (1.0 + abs(ts)) + 1e-5 * sf
        if any(oracle_lib.voxel_at(osc, X + sg * delta * e) != v
               for e in np.eye(3) for sg in (-1.0, 1.0)):
            amb[i] = True
            continue
        if v < 0:
            continue
        g = np.asarray(sc.params[v, :3], np.float64)
        if not g.any():
            continue
        c = abs(g @ r["d"][i]) / np.linalg.norm(g)
        if c < 1e-4:
            amb[i] = True
        elif kind == "refract" and abs(1.0 - eta * eta * (1.0 - c * c)) < 1e-4:
            amb[i] = True
    return amb


def _generation(salf, oracle_lib, sc, g, osc, sensor, kind, idx=None, **kw):
    prim = g.render(sensor, outputs=("depth", "opacity"))
    rays = g.secondary_rays(sensor, prim["depth"], prim["opacity"], kind=kind, **kw)
    torch.cuda.synchronize()
    rg = to_np(rays).astype(np.float64)
    depth, opac = to_np(prim["depth"]), to_np(prim["opacity"])
    if idx is not None:
        rg, depth, opac = rg[idx], depth[idx], opac[idx]
    ro = oracle_lib.secondary_rays(osc, sensor, depth, opac, kind=kind, idx=idx, **kw)
    amb = _ambiguous(oracle_lib, osc, sc, sensor, depth, opac, kind, kw.get("eta", 1 / 1.33),
                     kw.get("min_opacity", 0.5), idx)
    vg, vo = rg[:, 3:6].any(axis=1), ro[:, 3:6].any(axis=1)
    ok = ~amb
    assert np.array_equal(vg[ok], vo[ok]), (kind, np.where(ok & (vg != vo))[0][:5])
    both = ok & vg
    dd = np.abs(rg[both, 3:6] - ro[both, 3:6]).max(initial=0.0)
    scale = 1.0 + np.abs(ro[both, :3]).max(axis=1, initial=0.0)
    do = (np.abs(rg[both, :3] - ro[both, :3]).max(axis=1) / scale).max(initial=0.0)
    assert dd < 2e-5, (kind, dd)
    assert do < 2e-5, (kind, do)
    assert np.array_equal(rg[both, 6:], ro[both, 6:])
    assert amb.mean() <= 0.01, (kind, amb.mean())
    return rays, dict(n=len(rg), spawned=int(vg.sum()), ambiguous=int(amb.sum()), max_dir=dd,
                      max_org=do)


def _trace(salf, oracle_lib, g, osc, rays, t_min=1e-4):
    gr = g.render(salf.rays_sensor(rays), outputs=("rgb", "depth", "opacity"), t_min=t_min)
    gr = {k: to_np(v) for k, v in gr.items() if not k.startswith("_")}
    r32 = to_np(rays)
    sen = synth.explicit_rays(r32)
    orr = oracle_lib.render(osc, sen, t_min=t_min)
    sens = lambda pos: oracle_sensitivity(oracle_lib, osc,
                                          synth.explicit_rays(r32.astype(np.float64), np.float64),
                                          pos, t_min=t_min)
    return compare_outputs(gr, orr, t_min=t_min, sensitivity=sens)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_secondary_rays_small_scene(salf, oracle_lib, dtype):
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    params = None
    if dtype == "bf16":
        params = torch.from_numpy(sc.params).to(torch.bfloat16).double().numpy()
        sc = synth.SceneData(sc.origin, sc.s0, sc.dims, sc.max_level, sc.level, sc.ijk, params,
                             sc.mode, "bf16")
    g = salf.Scene(sc, dtype=dtype)
    osc = oracle_lib.OracleScene(sc)
    sensors = [synth.pinhole(64, 48, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
               synth.fisheye(40, 30, 190.0, synth.camera_pose_looking((0.4, 0.8, 1.0), 1.1)),
               synth.lidar(16, 90, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                           synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1)]
    cases = [("reflect", dict(offset=1e-3)), ("refract", dict(eta=1 / 1.33, offset=1e-3)),
             ("refract", dict(eta=1.4, offset=1e-3)),
             ("shadow", dict(light_dir=(0.3, -0.2, 1.0), offset=2e-3, t_far=6.0))]
    for sen in sensors:
        for kind, kw in cases:
            rays, st = _generation(salf, oracle_lib, sc, g, osc, sen, kind, min_opacity=0.3, **kw)
            assert st["spawned"] > 0.05 * st["n"], (sen["kind"], kind, st)
            _trace(salf, oracle_lib, g, osc, rays)
    g.check()


def test_secondary_rays_driving_1080p_sampled(salf, oracle_lib):
    sc = synth.driving_scene(2_000_000, seed=2)
    g = salf.Scene(sc)
    osc = oracle_lib.OracleScene(sc)
    cam = synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
    idx = synth.sample_ray_indices(1920 * 1080, 16384, 31)
    for kind, kw in (("reflect", {}), ("shadow", dict(light_dir=(0.4, 0.3, 1.0)))):
        rays, st = _generation(salf, oracle_lib, sc, g, osc, cam, kind, idx=idx, **kw)
        print(kind, st)
        sub = rays[torch.from_numpy(idx).cuda()].contiguous()
        _trace(salf, oracle_lib, g, osc, sub)
    g.check()


def test_secondary_rays_errors(salf):
    import ctypes as C
    from paper_2507_18713_gb300 import _lib as L
    from paper_2507_18713_gb300.api import sensor_struct
    sc = synth.random_multilevel_scene(seed=2, max_level=1, dims=(3, 3, 2), p_occ=0.7)
    g = salf.Scene(sc)
    cam = synth.pinhole(16, 8, 60.0, synth.camera_pose_looking((-1.5, 0.4, 0.8), 0.1))
    prim = g.render(cam, outputs=("depth", "opacity"))
    rays = torch.empty((128, 8), device="cuda")
    keep: list = []
    s = sensor_struct(cam, keep)

    def call(depth_ptr=None, rays_ptr=None, **f):
        o = L.SecondaryOpts()
        o.kind, o.eta, o.min_opacity, o.offset, o.t_far = 0, 0.75, 0.5, 1e-3, 0.0
        o.light_dir[:] = [0.0, 0.0, 1.0]
        for k, v in f.items():
            if k == "light_dir":
                o.light_dir[:] = v
            else:
                setattr(o, k, v)
        return L.load().salf_secondary_rays(
            g._h, C.byref(s), depth_ptr or prim["depth"].data_ptr(), prim["opacity"].data_ptr(),
            C.byref(o), rays_ptr or rays.data_ptr(), None)

    assert call() == 0
    torch.cuda.synchronize()
    for bad in (dict(kind=3), dict(kind=-1), dict(kind=1, eta=0.0), dict(kind=1, eta=-1.0),
                dict(kind=2, light_dir=[0.0, 0.0, 0.0]), dict(min_opacity=0.0),
                dict(min_opacity=1.5), dict(offset=-1.0), dict(offset=float("nan"))):
        assert call(**bad) == 1, bad
    host = np.zeros(128, np.float32)
    assert call(depth_ptr=host.ctypes.data) == 1             # host memory is refused
    assert call(rays_ptr=rays.data_ptr() + 4) == 1           # misaligned output
    g.check()
