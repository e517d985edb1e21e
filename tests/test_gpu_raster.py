"""Tile rasteriser (Sec. III-B, "Tile-based Splatting") vs the FP64 oracle and
vs the ray-cast kernel, through the C ABI.

The rasteriser composites each tile's voxels in the camera order (see
tests/test_raster_order.py), with the ray kernel's ray set-up, slab test and
field arithmetic, so its outputs must match the oracle at the ray path's
tolerances and equal the ray kernel's outputs wherever both visit the same
voxels (all but near-degenerate rays).
"""

import math

import numpy as np
import pytest

import synth
from tests.parity_util import (TOL_C, TOL_D, check_visits, visit_cap, compare_outputs, gpu_render,
                               oracle_sensitivity, to_np)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OUTS = ("rgb", "depth", "opacity", "intensity")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def raster(g, sensor, idx=None, **kw):
    out = g.render_raster(sensor, **kw)
    res = {k: to_np(v) for k, v in out.items() if not k.startswith("_")}
    if idx is not None:
        res = {k: v[idx] for k, v in res.items()}
    return res


def equal_frac(a, b, keys):
    """Fraction of pixels whose outputs are bitwise equal; max |a - b|."""
    same = np.ones(len(a["opacity"]), bool)
    worst = 0.0
    for k in keys:
        x, y = a[k].reshape(len(same), -1), b[k].reshape(len(same), -1)
        same &= (x == y).all(axis=1)
        worst = max(worst, float(np.abs(x - y).max()) if x.size else 0.0)
    return float(same.mean()), worst


def _parity(salf, oracle_lib, scene, sensor, dtype="f32", t_min=1e-4, want_intensity=False,
            background=(0.0, 0.0, 0.0), params_for_oracle=None, brute=None):
    g = salf.Scene(scene, dtype=dtype)
    osc = oracle_lib.OracleScene(scene, params=params_for_oracle)
    brute = scene.n <= 5000 if brute is None else brute
    kw = dict(t_min=t_min, want_intensity=want_intensity, background=background)
    st = {}
    gr = raster(g, sensor, outputs=OUTS, stats=st, **kw)
    orr = oracle_lib.render(osc, sensor, brute_force=brute, **kw)
    sens = lambda pos: oracle_sensitivity(oracle_lib, osc, sensor, pos, **kw)
    errs = compare_outputs(gr, orr, want_intensity=want_intensity, t_min=t_min, sensitivity=sens)
    ray = gpu_render(g, sensor, outputs=OUTS, **kw)
    frac, worst = equal_frac(gr, ray, OUTS + ("valid",))
    # visit lists at t_min = 0 against the oracle's exact lists
    cap = 256
    gv = raster(g, sensor, t_min=0.0, visits_cap=cap, outputs=("opacity",))
    ov = oracle_lib.render(osc, sensor, t_min=0.0, brute_force=brute, visits_cap=cap)
    vis = check_visits(oracle_lib, osc, sensor, scene, gv["visits"], gv["visit_count"],
                       ov["visits"], ov["n_visits"], None)
    g.check()
    g.close()
    return dict(errs=errs, equal_frac=frac, max_vs_ray=worst, visits=vis, stats=st)


def c1_camera(w=128, h=96):
    pose = np.concatenate([np.eye(3), [[3.2], [3.2], [-8.0]]], axis=1)
    return synth.pinhole(w, h, 60.0, pose)


def test_tiny_scene(salf, oracle_lib):
    res = _parity(salf, oracle_lib, synth.tiny_scene(seed=1), c1_camera())
    print(res)
    assert res["equal_frac"] >= 0.999 and res["max_vs_ray"] <= TOL_C, res
    n, bad = res["visits"]
    assert bad <= visit_cap(n), res
    assert res["stats"]["pairs"] > 0 and res["stats"]["visible_voxels"] > 0


@pytest.mark.parametrize("seed,K", [(0, 1), (1, 2), (2, 3)])
def test_multilevel_cameras(salf, oracle_lib, seed, K):
    """Cameras outside the grid, inside it, inside a voxel, on a split plane;
    image sizes that leave ragged tiles (and a 1 x 1 image)."""
    sc = synth.random_multilevel_scene(seed=seed, max_level=K, dims=(6, 5, 4), p_occ=0.6)
    lo = np.asarray(sc.origin)
    inside_voxel = lo + (sc.ijk[0] + 0.37) * sc.s0 / (1 << int(sc.level[0]))
    sensors = [
        synth.pinhole(61, 45, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
        synth.pinhole(100, 37, 90.0, synth.camera_pose_looking((0.9, 0.7, 0.95), 0.3)),
        synth.pinhole(17, 16, 110.0, synth.camera_pose_looking(tuple(inside_voxel), 2.0)),
        synth.pinhole(40, 33, 70.0, synth.camera_pose_looking((lo[0] + 2 * sc.s0, 0.7, 1.2), -0.4)),
        synth.pinhole(1, 1, 60.0, synth.camera_pose_looking((-2.0, 0.5, 1.1), 0.1)),
        synth.pinhole(48, 40, 70.0, synth.camera_pose_looking((0.2, 0.5, 1.0), 1.2), t_far=1.3),
    ]
    for sen in sensors:
        res = _parity(salf, oracle_lib, sc, sen, want_intensity=True, background=(0.1, 0.2, 0.3))
        assert res["max_vs_ray"] <= TOL_C, (sen["width"], res)
        n, bad = res["visits"]
        assert bad <= visit_cap(n), (sen["width"], res)


def test_sdf_and_bf16(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=4, max_level=2, dims=(6, 5, 4), p_occ=0.7, mode="sdf")
    sen = synth.pinhole(64, 48, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    res = _parity(salf, oracle_lib, sc, sen, want_intensity=True)
    assert res["max_vs_ray"] <= TOL_C, res
    tiny = synth.tiny_scene(seed=1)
    q = torch.from_numpy(tiny.params.astype(np.float32)).to(torch.bfloat16).double().numpy()
    res = _parity(salf, oracle_lib, tiny, c1_camera(), dtype="bf16", params_for_oracle=q)
    assert res["equal_frac"] >= 0.999 and res["max_vs_ray"] <= TOL_C, res


def test_empty_scene_and_rejections(salf):
    empty = synth.single_voxel_scene(np.zeros((0, 32)), dims=(3, 2, 2), cells=np.zeros((0, 3)),
                                     levels=())
    g = salf.Scene(empty)
    out = raster(g, synth.pinhole(17, 9, 60.0, synth.camera_pose_looking((-1, 1, 1), 0.0)),
                 background=(0.25, 0.5, 0.75))
    assert np.all(out["opacity"] == 0) and np.all(out["depth"] == 0)
    assert np.allclose(out["rgb"], [0.25, 0.5, 0.75])
    sc = synth.tiny_scene(seed=1)
    g = salf.Scene(sc)
    pose = synth.camera_pose_looking((3.2, 3.2, -8.0), 0.0)
    bad = [synth.fisheye(32, 24, 190.0, pose),
           synth.lidar(8, 64, synth.lidar_pose((0, 0, 1), 0.0), synth.lidar_pose((0, 0, 1), 0.0)),
           synth.pinhole(32, 24, 60.0, pose, synth.camera_pose_looking((3.0, 3.2, -8.0), 0.1),
                         t0=0.0, t1=0.05, rolling_shutter=True)]
    for s in bad:
        with pytest.raises(salf.SalfError) as e:
            g.render_raster(s)
        assert e.value.status == 1


def test_streams_and_saved_totals(salf):
    """Calls on two streams without a host wait between them give the lone
    results (the tile-list workspace is ordered between calls); the saved
    totals drive the adjoint exactly like the ray kernel's."""
    sc = synth.random_multilevel_scene(seed=1, max_level=2, dims=(6, 5, 4), p_occ=0.6)
    g = salf.Scene(sc)
    a = synth.pinhole(160, 120, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    b = synth.pinhole(96, 200, 60.0, synth.camera_pose_looking((-1.9, 0.2, 1.3), -0.2))
    lone_a, lone_b = raster(g, a), raster(g, b)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for _ in range(3):
        outs.append((g.render_raster(a, stream=s1), g.render_raster(b, stream=s2)))
    torch.cuda.synchronize()
    for oa, ob in outs:
        for k in ("rgb", "depth", "opacity"):
            assert np.array_equal(to_np(oa[k]), lone_a[k]) and np.array_equal(to_np(ob[k]), lone_b[k])
    fr = g.render_raster(a, saved=True)
    fy = g.render(a, saved=True)
    torch.cuda.synchronize()
    grad = torch.randn((a["width"] * a["height"], 3), device="cuda")
    d1 = g.backward(a, fr["saved"], d_rgb=grad)
    d2 = g.backward(a, fy["saved"], d_rgb=grad)
    torch.cuda.synchronize()
    assert torch.allclose(d1, d2, rtol=1e-5, atol=1e-6)


@pytest.fixture(scope="module")
def driving(salf, oracle_lib):
    sc = synth.driving_scene(2_000_000, seed=2)
    return sc, salf.Scene(sc), oracle_lib.OracleScene(sc)


@pytest.mark.parametrize("w,h,yaw", [(1920, 1080, 0.0), (960, 540, 0.7)])
def test_driving_frame(oracle_lib, driving, w, h, yaw):
    """Full frame vs the ray kernel, sampled pixels vs the oracle."""
    sc, g, osc = driving
    cam = synth.pinhole(w, h, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), yaw))
    st = {}
    full = raster(g, cam, outputs=OUTS, stats=st)
    ray = gpu_render(g, cam, outputs=OUTS)
    frac, worst = equal_frac(full, ray, OUTS + ("valid",))
    print(w, h, st, "bitwise-equal fraction vs ray kernel", frac, "max diff", worst)
    assert frac >= 0.999
    R = w * h
    idx = synth.sample_ray_indices(R, 32768, 21)
    gr = {k: v[idx] for k, v in full.items()}
    orr = oracle_lib.render(osc, cam, idx=idx)
    sens = lambda pos: oracle_sensitivity(oracle_lib, osc, cam, idx[pos], t_min=1e-4)
    errs = compare_outputs(gr, orr, t_min=1e-4, sensitivity=sens)
    print("vs oracle:", errs)
    cap = 512
    gv = raster(g, cam, idx=idx, t_min=0.0, visits_cap=cap, outputs=("opacity",))
    ov = oracle_lib.render(osc, cam, idx=idx, t_min=0.0, visits_cap=cap)
    n, bad = check_visits(oracle_lib, osc, cam, sc, gv["visits"], gv["visit_count"], ov["visits"],
                          ov["n_visits"], idx)
    assert bad <= visit_cap(n)
    g.check()
