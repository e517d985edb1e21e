"""Dynamic actors (Sec. IV-A) on the GPU (salf_render_rays_actors, through the
C ABI) against the FP64 oracle's actor rendering."""

import math

import numpy as np
import pytest

import synth
from tests.parity_util import KAPPA, TOL_C, compare_outputs, to_np

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


def _rigid(yaw, t):
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0, t[0]], [s, c, 0.0, t[1]], [0.0, 0.0, 1.0, t[2]]])


def _gpu(g, sensor, gactors, **kw):
    out = g.render_actors(sensor, gactors, **kw)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items() if not k.startswith("_")}


def actor_sensitivity(oracle, osc, oactors, sensor, idx, kappa=KAPPA, **kw):
    """Per ray: max oracle output change under +-kappa turns of its FP64 ray,
    with every actor fixed at its pose for that ray's time."""
    rays = oracle.gen_rays(sensor, idx)
    sc = np.zeros(len(idx))
    sd = np.zeros(len(idx))
    for i in range(len(idx)):
        o, d, tau = rays["o"][i], rays["d"][i], rays["tau"][i]
        tn = rays["t_near"][i]
        tf = rays["t_far"][i] if np.isfinite(rays["t_far"][i]) else 0.0
        placed = []
        for (a, p0, p1, base) in oactors:
            fake = dict(sensor, pose0=p0, pose1=p1)
            R, t = oracle.pose_at(fake, tau)
            P = np.concatenate([R, t[:, None]], axis=1)
            placed.append((a, P, P, base))

        def one(dd):
            row = np.concatenate([o, dd, [tn, tf]])[None, :]
            return oracle.render_actors(osc, placed, synth.explicit_rays(row, np.float64), **kw)
        base_r = one(d)
        for ref in (np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])):
            a = np.cross(d, ref)
            if np.linalg.norm(a) < 1e-3:
                a = np.cross(d, np.array([0.0, 1.0, 0.0]))
            a /= np.linalg.norm(a)
            for sgn in (-1.0, 1.0):
                d2 = d + sgn * kappa * a
                p = one(d2 / np.linalg.norm(d2))
                dc = max(np.abs(p["rgb"] - base_r["rgb"]).max(), abs(p["opacity"][0] - base_r["opacity"][0]),
                         abs(p["intensity"][0] - base_r["intensity"][0]))
                sc[i] = max(sc[i], dc)
                sd[i] = max(sd[i], abs(p["depth"][0] - base_r["depth"][0]))
    return sc, sd


def _parity(salf, oracle_lib, scene, actor_scenes, tracks, sensor, dtype="f32", idx=None,
            want_intensity=True, max_bad_visits=0.001):
    g = salf.Scene(scene, dtype=dtype)
    osc = oracle_lib.OracleScene(scene)
    gact, oact = [], []
    base = 1 << 20
    for k, (a, (p0, p1)) in enumerate(zip(actor_scenes, tracks)):
        gact.append((salf.Scene(a, dtype=dtype), p0, p1, base * (k + 1)))
        oact.append((oracle_lib.OracleScene(a), p0, p1, base * (k + 1)))
    kw = dict(t_min=1e-4, want_intensity=want_intensity, background=(0.05, 0.1, 0.15))
    gr = _gpu(g, sensor, gact, outputs=OUTS, **kw)
    orr = oracle_lib.render_actors(osc, oact, sensor, idx=idx, **kw)
    if idx is not None:
        gr = {k: v[idx] for k, v in gr.items()}
    ids = idx if idx is not None else np.arange(len(orr["opacity"]))
    sens = lambda pos: actor_sensitivity(oracle_lib, osc, oact, sensor, ids[pos], **kw)
    errs = compare_outputs(gr, orr, want_intensity=want_intensity, t_min=1e-4, sensitivity=sens)
    cap = 256
    gv = _gpu(g, sensor, gact, t_min=0.0, visits_cap=cap, outputs=("opacity",),
              want_intensity=want_intensity)
    ov = oracle_lib.render_actors(osc, oact, sensor, idx=idx, t_min=0.0, visits_cap=cap,
                                  want_intensity=want_intensity)
    vis, cnt = gv["visits"], gv["visit_count"]
    if idx is not None:
        vis, cnt = vis[idx], cnt[idx]
    bad = int(((cnt != ov["n_visits"]) | (vis != ov["visits"]).any(axis=1)).sum())
    n = len(cnt)
    actor_hits = int((ov["visits"] >= base).any(axis=1).sum())
    g.check()
    import os
    from tests.parity_util import VISIT_LOG
    VISIT_LOG.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0] + " (actors)", n,
                      bad))
    assert bad <= max(2, int(max_bad_visits * n)), (bad, n)
    return dict(errs=errs, bad_visits=bad, rays=n, rays_hitting_actors=actor_hits)


def _small_actors(k0=0):
    return [synth.actor_shell(1.0, 0.6, 0.5, seed=10 + k0),
            synth.actor_shell(0.8, 0.6, 0.7, seed=11 + k0),
            synth.actor_shell(1.2, 0.5, 0.4, seed=12 + k0)]


def test_multilevel_scene_with_actors_all_sensors(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=1, max_level=2, dims=(6, 5, 4), p_occ=0.35)
    acts = _small_actors()
    tracks = [(_rigid(0.3, (0.3, 0.4, 0.6)), _rigid(0.45, (0.5, 0.45, 0.6))),
              (_rigid(-0.5, (1.6, 1.3, 0.4)), _rigid(-0.5, (1.6, 1.3, 0.4))),
              (_rigid(1.2, (0.9, -0.2, 1.3)), _rigid(1.0, (1.1, -0.1, 1.25)))]
    sensors = [
        synth.pinhole(61, 45, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
        # (heights chosen so that no row's horizontal rays lie in a cell plane)
        synth.pinhole(40, 33, 70.0, synth.camera_pose_looking((-2.0, 0.2, 1.31), 0.0),
                      synth.camera_pose_looking((-1.7, 0.7, 1.17), 0.4), t0=0.0, t1=0.1,
                      rolling_shutter=True),
        synth.fisheye(50, 37, 190.0, synth.camera_pose_looking((0.1, 0.8, 1.03), 0.4)),
        synth.panorama(64, 16, synth.camera_pose_looking((1.0, 0.7, 0.95), 0.3)),
        synth.lidar(16, 90, synth.lidar_pose((0.2, 0.9, 1.05), 0.2),
                    synth.lidar_pose((0.8, 1.0, 1.05), 0.45), t0=0.0, t1=0.1),
    ]
    for sen in sensors:
        res = _parity(salf, oracle_lib, sc, acts, tracks, sen)
        print(sen["kind"], res)
        assert res["rays_hitting_actors"] > 10, sen["kind"]


def test_no_actors_equals_static_kernel(salf):
    """Without actors the merge reduces to the static walk: the same outputs
    and visit lists as salf_render_rays."""
    sc = synth.random_multilevel_scene(seed=2, max_level=2, dims=(6, 5, 4), p_occ=0.6)
    g = salf.Scene(sc)
    for sen in (synth.pinhole(64, 48, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
                synth.lidar(16, 128, synth.lidar_pose((0.3, 0.5, 1.0), 0.2),
                            synth.lidar_pose((0.6, 0.6, 1.0), 0.3), t0=0.0, t1=0.1)):
        a = _gpu(g, sen, [], outputs=OUTS, want_intensity=True, visits_cap=64)
        b = g.render(sen, outputs=OUTS, want_intensity=True, visits_cap=64)
        torch.cuda.synchronize()
        for k in OUTS + ("valid", "visits", "visit_count"):
            assert np.array_equal(a[k], to_np(b[k])), k


def test_identity_actor_matches_static_render(salf):
    """An actor at the identity pose over an empty static scene renders like
    the same voxels as a static scene (up to the actor frame's FP32 origin)."""
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(6, 5, 4), p_occ=0.6)
    empty = synth.single_voxel_scene(np.zeros((0, 32)), dims=(1, 1, 1), cells=np.zeros((0, 3)),
                                     levels=())
    ge, gs = salf.Scene(empty), salf.Scene(sc)
    I = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    sen = synth.pinhole(64, 48, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    a = _gpu(ge, sen, [(gs, I, I, 0)], outputs=OUTS, visits_cap=64)
    b = gs.render(sen, outputs=OUTS, visits_cap=64)
    torch.cuda.synchronize()
    assert np.abs(a["rgb"] - to_np(b["rgb"])).max() < 1e-4
    same = (a["visits"] == to_np(b["visits"])).all(axis=1).mean()
    assert same > 0.99


def test_actor_errors_and_interval_cap(salf):
    sc = synth.random_multilevel_scene(seed=2, max_level=2, dims=(6, 5, 4), p_occ=0.3)
    g = salf.Scene(sc)
    a = salf.Scene(synth.actor_shell(1.0, 0.6, 0.5, seed=1))
    sen = synth.pinhole(16, 12, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    P = _rigid(0.0, (0.5, 0.5, 0.5))
    with pytest.raises(salf.SalfError) as e:  # the same box twice
        g.render_actors(sen, [(a, P, P, 0), (a, P, P, 100)])
    assert e.value.status == 4
    ab = salf.Scene(synth.actor_shell(1.0, 0.6, 0.5, seed=1), dtype="bf16")
    with pytest.raises(salf.SalfError) as e:
        g.render_actors(sen, [(ab, P, P, 0)])
    assert e.value.status == 1
    # a ray along a row of 10 disjoint actors keeps the 8 nearest and flags it
    row = [(a, _rigid(0.0, (3.0 + 1.5 * k, 0.0, 0.0)), _rigid(0.0, (3.0 + 1.5 * k, 0.0, 0.0)), 0)
           for k in range(10)]
    rays = np.array([[0.0, 0.0, 0.25, 1.0, 0.0, 0.0, 0.0, 0.0]], np.float32)
    ge = salf.Scene(synth.single_voxel_scene(np.zeros((0, 32)), dims=(1, 1, 1),
                                             cells=np.zeros((0, 3)), levels=()))
    ge.render_actors(synth.explicit_rays(rays), row, t_min=0.0)
    torch.cuda.synchronize()
    with pytest.raises(salf.SalfError) as e:
        ge.check()
    assert e.value.status == 9


@pytest.fixture(scope="module")
def driving_actors(salf, oracle_lib):
    sc = synth.driving_scene(2_000_000, seed=2)
    tracks = synth.actor_tracks(24, seed=5)
    acts = [synth.actor_shell(*dims, seed=100 + k) for k, dims in
            enumerate([(4.4, 1.9, 1.6), (3.9, 1.8, 1.5), (4.8, 2.0, 1.8)] * 8)]
    return sc, acts, tracks


@pytest.mark.parametrize("which", ["camera", "lidar"])
def test_driving_scene_with_24_moving_actors(salf, oracle_lib, driving_actors, which):
    sc, acts, tracks = driving_actors
    if which == "camera":
        sen = synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
    else:
        sen = synth.lidar(128, 2048, synth.lidar_pose((0.0, 0.0, 1.9), 0.0),
                          synth.lidar_pose((1.0, 0.0, 1.9), 0.02), t0=0.0, t1=0.1)
    R = sen["width"] * sen["height"]
    idx = synth.sample_ray_indices(R, 16384, 31)
    res = _parity(salf, oracle_lib, sc, acts, tracks, sen, idx=idx,
                  want_intensity=which == "lidar")
    print(which, res)
    assert res["rays_hitting_actors"] > 100


def _front_wall_actor(seed):
    """An actor whose tight box reaches well past its front wall (one voxel in
    the far corner), so a ray leaves the wall and walks empty cells before its
    walk ends: the walk then ends in a round without a hit."""
    rng = np.random.default_rng(seed)
    cells = [(0, j, k) for j in range(4) for k in range(4)] + [(3, 3, 3)]
    params = synth.scenes.draw_params(rng, len(cells))
    params[:, 3] -= 1.5
    return synth.scenes.single_voxel_scene(params, s0=0.2, dims=(4, 4, 4), cells=cells,
                                           levels=[0] * len(cells), origin=(-0.4, -0.4, 0.0))


def test_actor_after_an_exhausted_actor_precedes_the_pending_static_hit(salf, oracle_lib):
    """Two translucent actors in a row in front of a static wall: once the
    first actor's walk ends, the second actor's box (entered before the wall)
    must open before the pending wall hit is composited (Eq. 3-4 take the
    hits in entry order, whichever walk found them)."""
    rng = np.random.default_rng(21)
    cells = [(10, j, k) for j in range(4) for k in range(4)]
    params = synth.scenes.draw_params(rng, len(cells))
    params[:, 3] -= 1.5  # thin wall: rays reach it with T well above t_min
    wall = synth.scenes.single_voxel_scene(params, dims=(12, 4, 4), cells=cells,
                                           levels=[0] * len(cells), origin=(0.0, -2.0, -2.0))
    acts = [_front_wall_actor(31), _front_wall_actor(32)]
    tracks = [(_rigid(0.0, (3.0, 0.0, -0.4)), _rigid(0.0, (3.0, 0.0, -0.4))),
              (_rigid(0.0, (6.0, 0.0, -0.4)), _rigid(0.0, (6.0, 0.0, -0.4)))]
    sen = synth.pinhole(16, 12, 6.0, synth.camera_pose_looking((0.0, 0.0, 0.0), 0.0))
    res = _parity(salf, oracle_lib, wall, acts, tracks, sen)
    print(res)
    assert res["rays_hitting_actors"] > 50
    assert res["bad_visits"] == 0
