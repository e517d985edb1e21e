"""Adjoint of the actor render (Sec. IV-A: actors are fitted together with the
static scene), through the C ABI, against the oracle's adjoint of its actor
render (pinned to central differences on the CPU), with the per-scalar bar of
the static adjoint: |gpu - oracle| <= 1e-3 |oracle| + 1e-6 + 4 u B."""

import math

import numpy as np
import pytest

import synth
from tests.test_gpu_backward import grad_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def _case(salf, oracle_lib, sc, acts, tracks, sen, idx=None, dtype="f32", want_intensity=True,
          t_min=0.0, seed=0):
    g = salf.Scene(sc, dtype=dtype)
    gact = [(salf.Scene(a, dtype=dtype), p0, p1, (k + 1) << 20)
            for k, (a, (p0, p1)) in enumerate(zip(acts, tracks))]
    q = (lambda p: torch.from_numpy(p.astype(np.float32)).to(torch.bfloat16).double().numpy()) \
        if dtype == "bf16" else (lambda p: p)
    osc = oracle_lib.OracleScene(sc, params=q(sc.params))
    oact = [(oracle_lib.OracleScene(a, params=q(a.params)), p0, p1, (k + 1) << 20)
            for k, (a, (p0, p1)) in enumerate(zip(acts, tracks))]
    R = sen["width"] * sen["height"]
    rng = np.random.default_rng(seed)
    gr = rng.normal(size=(R, 3)).astype(np.float32)
    gd = (rng.normal(size=R) * 0.1).astype(np.float32)
    go = rng.normal(size=R).astype(np.float32)
    gi = rng.normal(size=R).astype(np.float32)
    if idx is not None:
        mask = np.zeros(R, bool)
        mask[idx] = True
        for a in (gr, gd, go, gi):
            a[~mask] = 0
    kw = dict(t_min=t_min, background=(0.2, 0.1, 0.4), want_intensity=want_intensity)
    out = g.render_actors(sen, gact, saved=True, outputs=("rgb",), **kw)
    T = lambda a: torch.from_numpy(a).cuda()
    dg, dag = g.backward_actors(sen, gact, out["saved"], d_rgb=T(gr), d_depth=T(gd),
                                d_opacity=T(go), d_intensity=T(gi), **kw)
    torch.cuda.synchronize()
    g.check()
    sl = (lambda a: a[idx]) if idx is not None else (lambda a: a)
    f = lambda a: sl(a).astype(np.float64)
    (do, dao), (bo, bao) = oracle_lib.backward_actors(
        osc, oact, sen, g_rgb=f(gr), g_depth=f(gd), g_opacity=f(go), g_intensity=f(gi), idx=idx,
        brute_force=sc.n <= 5000, bound=True, **kw)
    return (dg.cpu().numpy(), [t.cpu().numpy() for t in dag]), (do, dao), (bo, bao)


def _small():
    sc = synth.random_multilevel_scene(seed=1, max_level=2, dims=(6, 5, 4), p_occ=0.35)
    acts = [synth.actor_shell(1.0, 0.6, 0.5, seed=10), synth.actor_shell(0.8, 0.6, 0.7, seed=11),
            synth.actor_shell(1.2, 0.5, 0.4, seed=12)]
    tracks = [(_rigid(0.3, (0.3, 0.4, 0.6)), _rigid(0.45, (0.5, 0.45, 0.6))),
              (_rigid(-0.5, (1.6, 1.3, 0.4)), _rigid(-0.5, (1.6, 1.3, 0.4))),
              (_rigid(1.2, (0.9, -0.2, 1.3)), _rigid(1.0, (1.1, -0.1, 1.25)))]
    return sc, acts, tracks


@pytest.mark.parametrize("kind", ["pinhole", "rolling", "lidar"])
def test_actor_adjoint_matches_oracle(salf, oracle_lib, kind):
    sc, acts, tracks = _small()
    if kind == "pinhole":
        sen = synth.pinhole(61, 45, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    elif kind == "rolling":
        sen = synth.pinhole(40, 33, 70.0, synth.camera_pose_looking((-2.0, 0.2, 1.31), 0.0),
                            synth.camera_pose_looking((-1.7, 0.7, 1.17), 0.4), t0=0.0, t1=0.1,
                            rolling_shutter=True)
    else:
        sen = synth.lidar(16, 90, synth.lidar_pose((0.2, 0.9, 1.05), 0.2),
                          synth.lidar_pose((0.8, 1.0, 1.05), 0.45), t0=0.0, t1=0.1)
    (dg, dag), (do, dao), (bo, bao) = _case(salf, oracle_lib, sc, acts, tracks, sen)
    stats = [grad_close(dg, do, bo)]
    for a, b, c in zip(dag, dao, bao):
        assert np.abs(b).max() > 0  # every actor is seen and gets a gradient
        stats.append(grad_close(a, b, c))
    print(kind, stats)


def test_actor_adjoint_after_an_exhausted_actor(salf, oracle_lib):
    """Two actors in a row whose walks end in empty cells, in front of a static
    wall: the adjoint takes the hits in the forward's entry order (the second
    actor's before the pending wall hit)."""
    from tests.test_gpu_actors import _front_wall_actor
    rng = np.random.default_rng(21)
    cells = [(10, j, k) for j in range(4) for k in range(4)]
    params = synth.scenes.draw_params(rng, len(cells))
    params[:, 3] -= 1.5
    wall = synth.scenes.single_voxel_scene(params, dims=(12, 4, 4), cells=cells,
                                           levels=[0] * len(cells), origin=(0.0, -2.0, -2.0))
    acts = [_front_wall_actor(31), _front_wall_actor(32)]
    tracks = [(_rigid(0.0, (3.0, 0.0, -0.4)), _rigid(0.0, (3.0, 0.0, -0.4))),
              (_rigid(0.0, (6.0, 0.0, -0.4)), _rigid(0.0, (6.0, 0.0, -0.4)))]
    sen = synth.pinhole(16, 12, 6.0, synth.camera_pose_looking((0.0, 0.0, 0.0), 0.0))
    (dg, dag), (do, dao), (bo, bao) = _case(salf, oracle_lib, wall, acts, tracks, sen)
    grad_close(dg, do, bo)
    for a, b, c in zip(dag, dao, bao):
        assert np.abs(b).max() > 0
        grad_close(a, b, c)


def test_actor_adjoint_bf16_sdf_and_early_termination(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=4, max_level=2, dims=(6, 5, 4), p_occ=0.35, mode="sdf")
    acts = [synth.actor_shell(1.0, 0.6, 0.5, seed=10, mode="sdf"),
            synth.actor_shell(0.8, 0.6, 0.7, seed=11, mode="sdf")]
    tracks = [(_rigid(0.3, (0.3, 0.4, 0.6)), _rigid(0.3, (0.3, 0.4, 0.6))),
              (_rigid(-0.5, (1.6, 1.3, 0.4)), _rigid(-0.5, (1.6, 1.3, 0.4)))]
    sen = synth.pinhole(48, 36, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    (dg, dag), (do, dao), (bo, bao) = _case(salf, oracle_lib, sc, acts, tracks, sen,
                                            dtype="bf16", t_min=1e-3)
    grad_close(dg, do, bo)
    for a, b, c in zip(dag, dao, bao):
        grad_close(a, b, c)


def test_actor_adjoint_driving_scene_sampled(salf, oracle_lib):
    """The 2M-voxel driving scene with 24 moving car shells, 1080p camera: the
    gradient of a seeded sample of rays (the whole frame launched)."""
    from tests.parity_util import conditioned_rays
    sc = synth.driving_scene(2_000_000, seed=2)
    tracks = synth.actor_tracks(24, seed=5)
    acts = [synth.actor_shell(*dims, seed=100 + k) for k, dims in
            enumerate([(4.4, 1.9, 1.6), (3.9, 1.8, 1.5), (4.8, 2.0, 1.8)] * 8)]
    sen = synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0))
    idx = synth.sample_ray_indices(1920 * 1080, 8192, 33)
    keep = conditioned_rays(oracle_lib, oracle_lib.OracleScene(sc), sen, idx, sc, t_min=1e-4)
    idx = idx[keep]
    (dg, dag), (do, dao), (bo, bao) = _case(salf, oracle_lib, sc, acts, tracks, sen, idx=idx,
                                            want_intensity=False, t_min=1e-4)
    stats = [grad_close(dg, do, bo)]
    seen = 0
    for a, b, c in zip(dag, dao, bao):
        stats.append(grad_close(a, b, c))
        seen += np.abs(b).max() > 0
    assert seen >= 4, seen
    print("actors seen", seen, stats[:3])


def test_actor_adjoint_without_actor_buffers(salf):
    """A null list of actor gradient buffers still yields the static gradient,
    equal to the run that also collects the actors'."""
    import ctypes as C
    from paper_2507_18713_gb300 import _lib as L
    from paper_2507_18713_gb300.api import opts_struct, sensor_struct
    sc, acts, tracks = _small()
    g = salf.Scene(sc)
    gact = [(salf.Scene(a), p0, p1, 0) for a, (p0, p1) in zip(acts, tracks)]
    sen = synth.pinhole(32, 24, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    out = g.render_actors(sen, gact, saved=True, outputs=("rgb",), t_min=0.0)
    w = torch.ones((32 * 24, 3), device="cuda")
    ref, _ = g.backward_actors(sen, gact, out["saved"], d_rgb=w, t_min=0.0)
    d = torch.zeros((sc.n, 32), device="cuda")
    arr = (L.Actor * len(gact))()
    for k, (a, p0, p1, b) in enumerate(gact):
        arr[k].actor = a._h
        arr[k].pose0[:] = [float(v) for v in np.asarray(p0).ravel()]
        arr[k].pose1[:] = [float(v) for v in np.asarray(p1).ravel()]
    keep = []
    s = sensor_struct(sen, keep)
    op = opts_struct(0.0)
    st = L.load().salf_render_backward_actors(g._h, arr, len(gact), C.byref(s), C.byref(op),
                                              out["saved"].data_ptr(), w.data_ptr(), None, None,
                                              None, d.data_ptr(), None, None)
    assert st == 0
    torch.cuda.synchronize()
    assert torch.allclose(d, ref, rtol=1e-5, atol=1e-6)
