"""GPU (sm_103a kernels, called through the C ABI) vs the FP64 oracle."""

import ctypes as C
import math

import numpy as np
import pytest

import synth
from tests.parity_util import (TOL_C, TOL_D, check_visits, visit_cap, compare_outputs, gpu_render,
                               oracle_sensitivity, to_np)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def c1_camera():
    pose = np.concatenate([np.eye(3), [[3.2], [3.2], [-8.0]]], axis=1)
    return synth.pinhole(128, 96, 60.0, pose)


def _full(salf, oracle_lib, scene, sensor, dtype="f32", t_min=1e-4, want_intensity=False,
          background=(0.0, 0.0, 0.0), visits=True, brute=None, params_for_oracle=None):
    g = salf.Scene(scene, dtype=dtype)
    osc = oracle_lib.OracleScene(scene, params=params_for_oracle)
    brute = scene.n <= 5000 if brute is None else brute
    kw = dict(t_min=t_min, want_intensity=want_intensity, background=background)
    gr = gpu_render(g, sensor, outputs=("rgb", "depth", "opacity", "intensity"), **kw)
    orr = oracle_lib.render(osc, sensor, brute_force=brute, **kw)
    sens = lambda pos: oracle_sensitivity(oracle_lib, osc, sensor, pos, **kw)
    errs = compare_outputs(gr, orr, want_intensity=want_intensity, t_min=t_min, sensitivity=sens)
    res = dict(errs=errs)
    if visits:
        cap = 256
        gv = gpu_render(g, sensor, t_min=0.0, visits_cap=cap, outputs=("opacity",))
        ov = oracle_lib.render(osc, sensor, t_min=0.0, brute_force=brute, visits_cap=cap)
        res["visits"] = check_visits(oracle_lib, osc, sensor, scene, gv["visits"],
                                     gv["visit_count"], ov["visits"], ov["n_visits"], None)
        res["mean_visits"] = float(ov["n_visits"].mean())
    g.check()
    g.close()
    return res


def test_tiny_scene_pinhole(salf, oracle_lib):
    """4,096 random voxels of a 64^3 grid, 128x96 pinhole, FP32 (the tiny case)."""
    sc = synth.tiny_scene(seed=1)
    res = _full(salf, oracle_lib, sc, c1_camera())
    n, bad = res["visits"]
    assert bad <= visit_cap(n), res
    res0 = _full(salf, oracle_lib, sc, c1_camera(), t_min=0.0, visits=False)
    assert res0["errs"]["max_c"] <= TOL_C


@pytest.mark.parametrize("seed,K", [(0, 1), (1, 2), (2, 3)])
def test_multilevel_all_sensors(salf, oracle_lib, seed, K):
    sc = synth.random_multilevel_scene(seed=seed, max_level=K, dims=(6, 5, 4), p_occ=0.6)
    sensors = [
        synth.pinhole(61, 45, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
        synth.fisheye(50, 37, 190.0, synth.camera_pose_looking((0.4, 0.8, 1.0), 1.1)),
        synth.panorama(64, 16, synth.camera_pose_looking((0.9, 0.7, 0.95), 0.3)),
        synth.lidar(16, 90, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                    synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1),
        synth.pinhole(33, 29, 60.0, synth.camera_pose_looking((-2.0, 0.2, 1.3), 0.0),
                      synth.camera_pose_looking((-1.6, 0.9, 1.2), 0.5), t0=0.0, t1=0.05,
                      rolling_shutter=True),
    ]
    for sen in sensors:
        res = _full(salf, oracle_lib, sc, sen, want_intensity=True, background=(0.1, 0.2, 0.3))
        n, bad = res["visits"]
        assert bad <= visit_cap(n), (sen["kind"], res)


def test_explicit_rays_edge_cases(salf, oracle_lib):
    """Caller-given rays: starting inside voxels, outside the root box, missing
    it, parallel to axes, with t_near / t_far clipping, and a ragged count."""
    sc = synth.random_multilevel_scene(seed=9, max_level=2, dims=(5, 4, 3), p_occ=0.7)
    rng = np.random.default_rng(3)
    org = np.array(sc.origin)
    ext = np.array(sc.dims) * sc.s0
    R = 1000
    o = org + rng.uniform(-0.5, 1.5, size=(R, 3)) * ext
    d = rng.normal(size=(R, 3))
    d[:50, 1:] = 0.0            # axis-parallel
    d[50:100, 0] = 0.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tn = np.where(rng.random(R) < 0.3, rng.uniform(0, 1, R), 0.0)
    tf = np.where(rng.random(R) < 0.3, tn + rng.uniform(0.1, 2, R), 0.0)
    rays = np.concatenate([o, d, tn[:, None], tf[:, None]], axis=1).astype(np.float32)
    sen = synth.explicit_rays(rays)
    res = _full(salf, oracle_lib, sc, sen, want_intensity=True)
    n, bad = res["visits"]
    assert bad <= visit_cap(n), res


def test_sdf_mode(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=4, max_level=2, dims=(6, 5, 4), p_occ=0.7, mode="sdf")
    sen = synth.pinhole(64, 48, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    res = _full(salf, oracle_lib, sc, sen, want_intensity=True)
    assert res["visits"][1] <= visit_cap(res["visits"][0]), res


def test_bf16_records(salf, oracle_lib):
    """BF16 storage: arithmetic parity against the oracle run on the
    dequantised records; the quantisation error itself is only reported."""
    sc = synth.tiny_scene(seed=1)
    q = torch.from_numpy(sc.params.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    res = _full(salf, oracle_lib, sc, c1_camera(), dtype="bf16", params_for_oracle=q)
    assert res["errs"]["max_c"] <= TOL_C
    # error of BF16 storage against the FP64 oracle on the FP32 records, per
    # output (reported, not asserted: it is the storage format's own error)
    osc32 = oracle_lib.OracleScene(sc)
    o32 = oracle_lib.render(osc32, c1_camera(), want_intensity=True)
    g = salf.Scene(sc, dtype="bf16")
    gb = gpu_render(g, c1_camera(), want_intensity=True,
                    outputs=("rgb", "depth", "opacity", "intensity"))
    errs = {k: float(np.abs(gb[k] - o32[k]).max()) for k in ("rgb", "depth", "opacity", "intensity")}
    print("BF16 storage error vs FP64 oracle on FP32 records (abs max):", errs)


def test_deep_octree_all_levels(salf, oracle_lib):
    """Voxels at every level 0..10 (edge down to 1/1024 of a level-0 cell);
    rays aimed at the spines' tips cross many tiny voxels."""
    sc = synth.deep_scene(max_level=10, dims=(2, 2, 2), seed=3)
    assert set(np.unique(sc.level)) == set(range(1, 11))
    osc = oracle_lib.OracleScene(sc)
    assert osc.status == 0
    tips = [(sc.ijk[v] + 0.5) / (1 << 10) * sc.s0 for v in np.where(sc.level == 10)[0]]
    rng = np.random.default_rng(0)
    rays = []
    for tip in tips:
        for _ in range(64):
            o = np.array(tip) + rng.normal(size=3) * 1.5
            d = np.array(tip) - o + rng.normal(size=3) * 1e-3
            rays.append(np.concatenate([o, d / np.linalg.norm(d), [0.0, 0.0]]))
    sen = synth.explicit_rays(np.array(rays))
    res = _full(salf, oracle_lib, sc, sen, t_min=0.0, brute=True)
    n, bad = res["visits"]
    assert bad <= visit_cap(n), res
    assert res["mean_visits"] > 3
    cam = synth.pinhole(96, 72, 80.0, synth.camera_pose_looking((-1.5, 0.9, 1.1), 0.1))
    res = _full(salf, oracle_lib, sc, cam, brute=True)
    assert res["visits"][1] <= visit_cap(res["visits"][0]), res


def test_size_limits_rejected(salf):
    r = np.zeros((1, 32), np.float32)
    too_wide = synth.single_voxel_scene(r, dims=(4097, 1, 1), max_level=10)
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(too_wide)            # dims << max_level > 2^21
    assert e.value.status == 1
    too_deep = synth.single_voxel_scene(r, max_level=11)
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(too_deep)
    assert e.value.status == 1
    g = salf.Scene(synth.single_voxel_scene(r))
    huge = synth.pinhole(65536, 65536, 60.0, synth.camera_pose_looking((-1, 0.5, 0.5), 0.0))
    with pytest.raises(salf.SalfError) as e:
        g.render(huge, outputs=("opacity",), valid=False)   # > 2^31 - 1 rays
    assert e.value.status == 1
    bad_fx = synth.pinhole(8, 8, 60.0, synth.camera_pose_looking((-1, 0.5, 0.5), 0.0))
    bad_fx["fx"] = 0.0
    with pytest.raises(salf.SalfError) as e:
        g.render(bad_fx)
    assert e.value.status == 1


def test_empty_and_degenerate_scenes(salf, oracle_lib):
    empty = synth.single_voxel_scene(np.zeros((0, 32)), dims=(3, 2, 2), cells=np.zeros((0, 3)),
                                     levels=())
    g = salf.Scene(empty)
    out = gpu_render(g, synth.pinhole(17, 9, 60.0, synth.camera_pose_looking((-1, 1, 1), 0.0)))
    assert np.all(out["rgb"] == 0) and np.all(out["opacity"] == 0) and np.all(out["depth"] == 0)
    # a single voxel, a single ray through its centre
    rec = np.zeros(32)
    rec[3] = math.log(2.0)
    one = synth.single_voxel_scene(rec)
    g1 = salf.Scene(one)
    sen = synth.explicit_rays(np.array([[-1.0, 0.5, 0.5, 1, 0, 0, 0, 0]], np.float32))
    r = gpu_render(g1, sen, t_min=0.0)
    assert abs(r["opacity"][0] - (1 - math.exp(-2.0))) < 1e-6
    assert abs(r["depth"][0] - 1.5 * (1 - math.exp(-2.0))) < 1e-5


def test_overlap_and_invalid_rejected(salf):
    r = np.zeros((2, 32), np.float32)
    dup = synth.single_voxel_scene(r, dims=(2, 1, 1), cells=((0, 0, 0), (0, 0, 0)), levels=(0, 0))
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(dup)
    assert e.value.status == 4
    anc = synth.single_voxel_scene(r, dims=(2, 1, 1), cells=((1, 0, 0), (3, 1, 0)), levels=(0, 1),
                                   max_level=1)
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(anc)
    assert e.value.status == 4
    out = synth.single_voxel_scene(r[:1], dims=(2, 1, 1), cells=((2, 0, 0),), levels=(0,))
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(out)
    assert e.value.status == 1
    bad = np.zeros((1, 32), np.float32)
    bad[0, 25] = -1.0
    sdf = synth.single_voxel_scene(bad, mode="sdf")
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(sdf)
    assert e.value.status == 1


def test_permutation_invariance_bitwise(salf):
    sc = synth.random_multilevel_scene(seed=6, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    sc2, perm = synth.shuffle_scene(sc, 1)
    sen = synth.pinhole(64, 48, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    a = gpu_render(salf.Scene(sc), sen, visits_cap=64, t_min=0.0)
    b = gpu_render(salf.Scene(sc2), sen, visits_cap=64, t_min=0.0)
    for k in ("rgb", "depth", "opacity"):
        assert np.array_equal(a[k], b[k]), k
    mapped = np.where(b["visits"] >= 0, perm[np.maximum(b["visits"], 0)], -1)
    assert np.array_equal(a["visits"], mapped)


def test_host_outputs_match_device_outputs(salf):
    sc = synth.tiny_scene(seed=1)
    g = salf.Scene(sc)
    dev = gpu_render(g, c1_camera(), want_intensity=True,
                     outputs=("rgb", "depth", "opacity", "intensity"))
    host = g.render_host(c1_camera(), want_intensity=True,
                         outputs=("rgb", "depth", "opacity", "intensity"))
    for k in ("rgb", "depth", "opacity", "intensity"):
        assert np.array_equal(dev[k], host[k].numpy()), k


def test_pinned_host_outputs_are_written_in_place(salf):
    """Page-locked host outputs are written by the kernel directly; pageable
    ones go through staging; both equal the device outputs bit for bit."""
    from paper_2507_18713_gb300.api import opts_struct, sensor_struct
    sc = synth.random_multilevel_scene(seed=5, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    sc.params[:, 31] = np.random.default_rng(2).normal(size=sc.n)
    g = salf.Scene(sc)
    cam = synth.pinhole(641, 479, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    lid = synth.lidar(32, 256, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                      synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1)
    for sen, outs, vcap in ((cam, ("rgb", "depth", "opacity"), 0),
                            (lid, ("depth", "opacity", "intensity", "raydrop"), 0),
                            (cam, ("opacity",), 16)):
        dev = g.render(sen, want_intensity=True, outputs=outs, saved=True, visits_cap=vcap)
        torch.cuda.synchronize()
        ref = {k: v.cpu() for k, v in dev.items() if not k.startswith("_")}
        for pinned in (True, False):
            host = {k: (torch.empty_like(v).pin_memory() if pinned else torch.empty_like(v))
                    for k, v in ref.items()}
            o = salf._lib.Outputs()
            for k, v in host.items():
                setattr(o, k, v.data_ptr())
            o.on_host = 1
            keep: list = []
            s = sensor_struct(sen, keep)
            op = opts_struct(1e-4, (0.0, 0.0, 0.0), True, vcap)
            st = salf._lib.load().salf_render_rays(g._h, C.byref(s), C.byref(op), C.byref(o), None)
            assert st == 0
            for k in ref:
                assert torch.equal(ref[k], host[k]), (sen["kind"], k, pinned)
    # explicit rays in page-locked memory, read by the kernel in place
    rng = np.random.default_rng(4)
    r = np.concatenate([rng.uniform(-1, 2, (777, 3)), rng.normal(size=(777, 3)),
                        np.zeros((777, 2))], axis=1).astype(np.float32)
    r[:, 3:6] /= np.linalg.norm(r[:, 3:6], axis=1, keepdims=True)
    pr = torch.from_numpy(r).pin_memory()
    sen_h = synth.explicit_rays(r)
    sen_h["rays"] = pr
    dev = g.render(synth.explicit_rays(r), outputs=("rgb", "depth"))
    host = g.render_host(sen_h, outputs=("rgb", "depth"),
                         out={"rgb": torch.empty((777, 3)).pin_memory(),
                              "depth": torch.empty(777).pin_memory()})
    torch.cuda.synchronize()
    assert torch.equal(dev["rgb"].cpu(), host["rgb"]) and torch.equal(dev["depth"].cpu(), host["depth"])
    g.check()


def test_async_pinned_host_outputs(salf):
    """on_host = 2: page-locked outputs written in place, the call returns after
    the launch; two frames in flight in their own buffers equal the device
    renders bit for bit once the stream drains.  Pageable buffers are refused."""
    sc = synth.random_multilevel_scene(seed=7, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    g = salf.Scene(sc)
    outs = ("rgb", "depth", "opacity")
    cams = [synth.pinhole(320, 240, 75.0, synth.camera_pose_looking((-2.2, 0.6 + 0.2 * i, 1.1),
                                                                     0.15)) for i in range(2)]
    refs = []
    for cam in cams:
        d = g.render(cam, outputs=outs)
        torch.cuda.synchronize()
        refs.append({k: d[k].cpu() for k in outs})
    bufs = [{k: torch.empty_like(v).pin_memory() for k, v in ref.items()} for ref in refs]
    for b in bufs:
        for v in b.values():
            v.fill_(-7.0)
    st = torch.cuda.Stream()
    for cam, b in zip(cams, bufs):  # both frames in flight before any wait
        g.render_host(cam, outputs=outs, out=b, sync=False, stream=st)
    st.synchronize()
    for ref, b in zip(refs, bufs):
        for k in outs:
            assert torch.equal(ref[k], b[k]), k
    with pytest.raises(salf.SalfError):
        g.render_host(cams[0], outputs=outs, out={k: torch.empty_like(v) for k, v in refs[0].items()},
                      sync=False)
    # on_host outside 0..2 is refused before any work
    from paper_2507_18713_gb300.api import opts_struct, sensor_struct
    o = salf._lib.Outputs()
    o.depth = bufs[0]["depth"].data_ptr()
    o.on_host = 3
    keep: list = []
    s = sensor_struct(cams[0], keep)
    op = opts_struct(1e-4, (0.0, 0.0, 0.0), False, 0)
    assert salf._lib.load().salf_render_rays(g._h, C.byref(s), C.byref(op), C.byref(o), None) != 0
    g.check()


def test_host_frames_pipeline(salf):
    """HostFrames: device renders with the copy engine moving each frame to
    page-locked memory while the next renders; every frame equals its device
    render bit for bit, including slots reused after `depth` frames."""
    sc = synth.random_multilevel_scene(seed=11, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    g = salf.Scene(sc)
    outs = ("rgb", "depth", "opacity")
    cams = [synth.pinhole(200, 150, 75.0, synth.camera_pose_looking((-2.2, 0.4 + 0.15 * i, 1.1),
                                                                     0.1 * i)) for i in range(5)]
    refs = []
    for cam in cams:
        d = g.render(cam, outputs=outs)
        torch.cuda.synchronize()
        refs.append({k: d[k].cpu() for k in outs})
    hf = salf.HostFrames(g, cams[0], outputs=outs, depth=2)
    prev = None
    for i, cam in enumerate(cams):
        slot = hf.submit(cam)
        if prev is not None:
            got = hf.result(prev[1])
            for k in outs:
                assert torch.equal(got[k], refs[prev[0]][k]), (prev[0], k)
        prev = (i, slot)
    got = hf.result(prev[1])
    for k in outs:
        assert torch.equal(got[k], refs[prev[0]][k]), (prev[0], k)
    g.check()


def test_update_params_matches_rebuild(salf):
    sc = synth.random_multilevel_scene(seed=2, max_level=2)
    sen = synth.pinhole(40, 30, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    rng = np.random.default_rng(0)
    p2 = sc.params.astype(np.float32) + rng.normal(0, 0.05, size=sc.params.shape).astype(np.float32)
    g = salf.Scene(sc)
    g.update_params(torch.from_numpy(p2).cuda())
    a = gpu_render(g, sen)
    b = gpu_render(salf.Scene(sc.with_params(p2)), sen)
    for k in ("rgb", "depth", "opacity"):
        assert np.array_equal(a[k], b[k])


# --------------------------------------------------------------------------
# Full-size driving scenes: sampled rays of the benchmark launch
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def driving(salf, oracle_lib):
    sc = synth.driving_scene(2_000_000, seed=2)
    return sc, salf.Scene(sc), oracle_lib.OracleScene(sc)


def _sampled(oracle_lib, driving, sensor, n_sample, seed, want_intensity=False, visits=True):
    sc, g, osc = driving
    R = sensor["width"] * sensor["height"]
    idx = synth.sample_ray_indices(R, n_sample, seed)
    kw = dict(want_intensity=want_intensity)
    gr = gpu_render(g, sensor, idx=idx, outputs=("rgb", "depth", "opacity", "intensity"), **kw)
    orr = oracle_lib.render(osc, sensor, idx=idx, **kw)
    sens = lambda pos: oracle_sensitivity(oracle_lib, osc, sensor, idx[pos], t_min=1e-4, **kw)
    errs = compare_outputs(gr, orr, want_intensity=want_intensity, t_min=1e-4, sensitivity=sens)
    out = dict(errs=errs, mean_visits=float(orr["n_visits"].mean()))
    if visits:
        cap = 512
        gv = gpu_render(g, sensor, idx=idx, t_min=0.0, visits_cap=cap, outputs=("opacity",))
        ov = oracle_lib.render(osc, sensor, idx=idx, t_min=0.0, visits_cap=cap)
        out["visits"] = check_visits(oracle_lib, osc, sensor, sc, gv["visits"], gv["visit_count"],
                                     ov["visits"], ov["n_visits"], idx)
    g.check()
    return out


def test_driving_1080p_pinhole_sampled(oracle_lib, driving):
    cam = synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
    res = _sampled(oracle_lib, driving, cam, 65536, 11)
    print("1080p pinhole:", res)
    n, bad = res["visits"]
    assert bad <= visit_cap(n)


def test_driving_lidar_sampled(oracle_lib, driving):
    lid = synth.lidar(128, 2048, synth.lidar_pose((0.0, 0.0, 1.9), 0.0),
                      synth.lidar_pose((1.0, 0.0, 1.9), 0.02), t0=0.0, t1=0.1)
    res = _sampled(oracle_lib, driving, lid, 65536, 12, want_intensity=True)
    print("LiDAR 128x2048:", res)
    n, bad = res["visits"]
    assert bad <= visit_cap(n)


def test_driving_fisheye_sampled(oracle_lib, driving):
    fe = synth.fisheye(1920, 1080, 190.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
    res = _sampled(oracle_lib, driving, fe, 32768, 13, visits=True)
    print("fisheye 1080p:", res)
    n, bad = res["visits"]
    assert bad <= visit_cap(n)


def test_driving_identical_rays(oracle_lib, driving):
    """Rendering parity with the ray-generation step taken out: both sides
    render the same FP32 rays (the oracle's own FP64 rays, rounded)."""
    sc, g, osc = driving
    cam = synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
    idx = synth.sample_ray_indices(1920 * 1080, 65536, 21)
    rays = oracle_lib.gen_rays(cam, idx)
    r32 = np.concatenate([rays["o"], rays["d"], np.zeros((len(idx), 2))], axis=1).astype(np.float32)
    sen = synth.explicit_rays(r32)
    gr = gpu_render(g, sen, outputs=("rgb", "depth", "opacity", "intensity"))
    orr = oracle_lib.render(osc, sen)
    r64 = r32.astype(np.float64)
    sens = lambda pos: oracle_sensitivity(oracle_lib, osc, synth.explicit_rays(r64, np.float64),
                                          pos, t_min=1e-4)
    res = compare_outputs(gr, orr, t_min=1e-4, sensitivity=sens, max_relaxed_frac=0.005)
    gv = gpu_render(g, sen, t_min=0.0, visits_cap=512, outputs=("opacity",))
    ov = oracle_lib.render(osc, sen, t_min=0.0, visits_cap=512)
    n, bad = check_visits(oracle_lib, osc, sen, sc, gv["visits"], gv["visit_count"], ov["visits"],
                          ov["n_visits"], None)
    print("identical rays:", res, "visit lists explained by eps:", bad, "of", n)
    assert bad <= visit_cap(n)


@pytest.mark.parametrize("kind", ["pinhole", "fisheye", "pano", "lidar", "rolling"])
def test_generated_rays_match_oracle(salf, oracle_lib, kind):
    """Ray generation alone (Fig. 2 sensor models, Sec. V-C per-ray pose):
    the kernel's rays (debug dump) against the oracle's FP64 rays."""
    sc = synth.tiny_scene(seed=1)
    g = salf.Scene(sc)
    p0 = synth.camera_pose_looking((1.3, -2.1, 1.7), 0.4)
    p1 = synth.camera_pose_looking((2.3, -1.1, 1.8), 0.9)
    sen = {"pinhole": synth.pinhole(333, 201, 70.0, p0),
           "fisheye": synth.fisheye(320, 240, 190.0, p0),
           "pano": synth.panorama(512, 128, p0),
           "lidar": synth.lidar(64, 1024, synth.lidar_pose((1.0, 2.0, 1.9), 0.3),
                                synth.lidar_pose((2.0, 2.5, 1.9), 0.32), t0=0.0, t1=0.1),
           "rolling": synth.pinhole(160, 121, 60.0, p0, p1, t0=0.0, t1=0.05,
                                    rolling_shutter=True)}[kind]
    out = g.render(sen, ray_dump=True, outputs=("opacity",))
    dump = to_np(out["ray_dump"]).astype(np.float64)
    ref = oracle_lib.gen_rays(sen)
    valid = ref["valid"]
    r = np.sqrt(((np.arange(320 * 240) % 320 + 0.5 - 160) ** 2 +
                 (np.arange(320 * 240) // 320 + 0.5 - 120) ** 2)) / sen["fx"] if kind == "fisheye" else None
    if kind == "fisheye":
        edge = np.abs(r - sen["fov"] / 2) < 1e-5
        assert np.array_equal((dump[:, 7] > 0)[~edge], valid[~edge])
    else:
        assert np.array_equal(dump[:, 7] > 0, valid)
    d = dump[:, 3:6] / np.linalg.norm(dump[:, 3:6], axis=1, keepdims=True)
    ang = np.linalg.norm(np.cross(d, ref["d"]), axis=1)[valid]
    lim = 1.5e-7 if kind == "pinhole" else 3e-7
    print(f"{kind}: max direction error {ang.max():.3g} rad, origin error "
          f"{np.abs(dump[:, :3] - ref['o']).max():.3g} m")
    assert ang.max() <= lim, (kind, ang.max())
    assert np.abs(dump[:, :3] - ref["o"]).max() <= 2e-6
    assert np.abs(dump[:, 6] - ref["tau"]).max() <= 1e-7 + 1e-6 * abs(sen["t1"])


def test_driving_full_frame_properties(driving):
    """Whole 1080p frame: invariants that hold at any size."""
    sc, g, _ = driving
    cam = synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
    out = g.render(cam, saved=True)
    O = to_np(out["opacity"])
    rgb = to_np(out["rgb"])
    s = to_np(out["saved"])
    assert np.isfinite(rgb).all() and np.isfinite(to_np(out["depth"])).all()
    assert (O >= 0).all() and (O <= 1 + 1e-6).all()
    assert np.abs(O - (1 - s[:, 6])).max() < 1e-5          # sum w = 1 - T_end
    assert (rgb <= O[:, None] + 1e-5).all() and (rgb >= 0).all()
    stopped = s[:, 6] < 1e-4
    assert stopped.any()
