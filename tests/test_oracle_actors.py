"""Pins of the oracle's dynamic-actor rendering (Sec. IV-A) against facts that
do not depend on it: reduction to the static oracle, invariance under a rigid
motion of everything, the closed form of Eq. 3-4 for an interleaved pair of
voxels, per-ray actor poses equal to a static render at the interpolated pose,
and brute force against the grid walk."""

import math

import numpy as np

import synth


def _empty_static():
    return synth.single_voxel_scene(np.zeros((0, 32)), dims=(1, 1, 1), cells=np.zeros((0, 3)),
                                    levels=())


def _rigid(yaw, t):
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0, t[0]], [s, c, 0.0, t[1]], [0.0, 0.0, 1.0, t[2]]])


def _compose(G, P):
    """G . P for 3x4 rigid maps."""
    R = G[:, :3] @ P[:, :3]
    t = G[:, :3] @ P[:, 3] + G[:, 3]
    return np.concatenate([R, t[:, None]], axis=1)


IDENT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)


def test_identity_actor_equals_static_render(oracle_lib):
    """An actor placed by the identity pose is the same voxel set as a static
    scene: outputs equal, visits shifted by id_base."""
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(6, 5, 4), p_occ=0.6)
    cam = synth.pinhole(40, 30, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    ref = oracle_lib.render(oracle_lib.OracleScene(sc), cam, want_intensity=True, visits_cap=64)
    empty = oracle_lib.OracleScene(_empty_static())
    act = oracle_lib.OracleScene(sc)
    got = oracle_lib.render_actors(empty, [(act, IDENT, IDENT, 1000)], cam, want_intensity=True,
                                   visits_cap=64)
    for k in ("rgb", "depth", "opacity", "intensity", "t_end"):
        assert np.array_equal(ref[k], got[k]), k
    exp_vis = np.where(ref["visits"] >= 0, ref["visits"] + 1000, -1)
    assert np.array_equal(exp_vis, got["visits"])


def test_rigid_motion_of_everything_is_invisible(oracle_lib):
    """Moving the camera and every actor by one rigid map changes nothing."""
    a1 = synth.actor_shell(4.4, 1.9, 1.6, seed=1)
    a2 = synth.actor_shell(3.8, 1.8, 1.5, seed=2)
    o1, o2 = oracle_lib.OracleScene(a1), oracle_lib.OracleScene(a2)
    empty = oracle_lib.OracleScene(_empty_static())
    P1, P2 = _rigid(0.3, (6.0, 1.0, 0.2)), _rigid(-0.2, (9.0, -2.5, 0.2))
    cam_pose = synth.camera_pose_looking((0.0, 0.0, 1.5), 0.0)
    cam = synth.pinhole(48, 32, 70.0, cam_pose)
    base = oracle_lib.render_actors(empty, [(o1, P1, P1, 0), (o2, P2, P2, 5000)], cam)
    G = _rigid(1.1, (-3.0, 7.0, 0.5))
    cam2 = synth.pinhole(48, 32, 70.0, _compose(G, cam_pose))
    moved = oracle_lib.render_actors(
        empty, [(o1, _compose(G, P1), _compose(G, P1), 0), (o2, _compose(G, P2), _compose(G, P2), 5000)],
        cam2)
    assert base["opacity"].max() > 0.2
    for k in ("rgb", "depth", "opacity"):
        assert np.abs(base[k] - moved[k]).max() < 1e-9, k


def test_interleaving_follows_entry_order(oracle_lib):
    """One static voxel and one actor voxel on a ray: whichever the ray
    enters first is composited first, by the closed form of Eq. 3-4."""
    rs = np.zeros(32); rs[3] = math.log(0.7); rs[13] = 2.0   # static: sigma 0.7
    ra = np.zeros(32); ra[3] = math.log(1.9); ra[17] = -1.0  # actor: sigma 1.9
    static = synth.single_voxel_scene(rs, s0=1.0, origin=(2.0, -0.5, -0.5))
    actor = synth.single_voxel_scene(ra, s0=1.0, origin=(-0.5, -0.5, -0.5))
    ost, oac = oracle_lib.OracleScene(static), oracle_lib.OracleScene(actor)
    for ax, first in ((0.0, "actor"), (5.0, "static")):
        P = _rigid(0.0, (ax, 0.0, 0.0))  # actor voxel spans x in [ax - 0.5, ax + 0.5]
        rays = np.array([[-1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0]], np.float64)
        sen = synth.explicit_rays(rays, dtype=np.float64)
        r = oracle_lib.render_actors(ost, [(oac, P, P, 10)], sen, t_min=0.0, visits_cap=4)
        sig = {"static": 0.7, "actor": 1.9}
        tmid = {"static": 3.5, "actor": ax + 1.0}  # static box x in [2, 3], ray from x = -1
        order = [first, "static" if first == "actor" else "actor"]
        T, D, O = 1.0, 0.0, 0.0
        for who in order:
            a = 1.0 - math.exp(-sig[who])
            D += T * a * tmid[who]
            O += T * a
            T *= 1.0 - a
        assert abs(r["opacity"][0] - O) < 1e-12 and abs(r["depth"][0] - D) < 1e-12
        assert list(r["visits"][0][:2]) == ([10, 0] if first == "actor" else [0, 10])
        assert r["n_visits"][0] == 2


def test_per_ray_actor_pose_is_the_interpolated_pose(oracle_lib):
    """A LiDAR sweep sees a moving actor, per ray, exactly as a static render
    with the actor at its interpolated pose for that ray's time."""
    act = synth.actor_shell(4.4, 1.9, 1.6, seed=4)
    oa = oracle_lib.OracleScene(act)
    empty = oracle_lib.OracleScene(_empty_static())
    P0, P1 = _rigid(0.0, (8.0, 0.0, 0.0)), _rigid(0.25, (9.5, 1.0, 0.0))
    lid = synth.lidar(16, 256, synth.lidar_pose((0.0, 0.0, 1.0), 0.0),
                      synth.lidar_pose((0.5, 0.0, 1.0), 0.05), t0=0.0, t1=0.1)
    full = oracle_lib.render_actors(empty, [(oa, P0, P1, 0)], lid, t_min=0.0)
    hit = np.where(full["opacity"] > 0.05)[0]
    assert len(hit) > 20
    rng = np.random.default_rng(0)
    for r in rng.choice(hit, size=12, replace=False):
        ray = oracle_lib.gen_rays(lid, [int(r)])
        s = (ray["tau"][0] - 0.0) / 0.1
        # actor pose at s: slerp of a rotation about z = linear yaw
        Ps = _rigid(0.25 * s, (8.0 + 1.5 * s, 1.0 * s, 0.0))
        row = np.concatenate([ray["o"][0], ray["d"][0], [ray["t_near"][0], 0.0]])[None, :]
        one = synth.explicit_rays(row.astype(np.float64), dtype=np.float64)
        ref = oracle_lib.render_actors(empty, [(oa, Ps, Ps, 0)], one, t_min=0.0)
        assert abs(ref["opacity"][0] - full["opacity"][r]) < 1e-9
        assert abs(ref["depth"][0] - full["depth"][r]) < 1e-8


def test_actor_brute_force_equals_grid_walk(oracle_lib):
    sc = synth.random_multilevel_scene(seed=2, max_level=2, dims=(6, 5, 4), p_occ=0.5)
    osc = oracle_lib.OracleScene(sc)
    acts = [(oracle_lib.OracleScene(synth.actor_shell(3.0, 1.6, 1.4, seed=k)),
             _rigid(0.4 * k, (1.0 + 0.9 * k, 0.5 - 0.3 * k, 0.1)),
             _rigid(0.4 * k + 0.1, (1.2 + 0.9 * k, 0.5 - 0.3 * k, 0.1)), 100000 * (k + 1))
            for k in range(2)]
    cam = synth.pinhole(30, 24, 80.0, synth.camera_pose_looking((-2.5, 0.4, 1.2), 0.1),
                        synth.camera_pose_looking((-2.3, 0.5, 1.2), 0.15), t0=0.0, t1=0.05,
                        rolling_shutter=True)
    a = oracle_lib.render_actors(osc, acts, cam, brute_force=True, visits_cap=128)
    b = oracle_lib.render_actors(osc, acts, cam, brute_force=False, visits_cap=128)
    assert np.array_equal(a["visits"], b["visits"])
    assert np.abs(a["rgb"] - b["rgb"]).max() < 1e-12


def test_view_direction_is_taken_in_the_actor_frame(oracle_lib):
    """Colour through the SH term depends on the view direction in the actor's
    frame: turning a symmetric single-voxel actor about z keeps its opacity
    and turns the direction its SH term sees."""
    rec = np.zeros(32); rec[3] = math.log(3.0); rec[14] = 4.0  # red driven by gamma_y (C1 * w_y)
    vox = synth.single_voxel_scene(rec, s0=1.0, origin=(-0.5, -0.5, -0.5))
    ov = oracle_lib.OracleScene(vox)
    empty = oracle_lib.OracleScene(_empty_static())
    rays = np.array([[-3.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0]], np.float64)
    sen = synth.explicit_rays(rays, dtype=np.float64)
    straight = oracle_lib.render_actors(empty, [(ov, IDENT, IDENT, 0)], sen, t_min=0.0)
    Rz = _rigid(math.pi / 2, (0, 0, 0))
    turned = oracle_lib.render_actors(empty, [(ov, Rz, Rz, 0)], sen, t_min=0.0)
    # in the actor frame turned by +90 deg about z, the world +x ray runs along -y
    assert abs(straight["opacity"][0] - turned["opacity"][0]) < 1e-12
    g = 0.48860251190291992
    op = straight["opacity"][0]
    assert abs(straight["rgb"][0][0] - op / (1.0 + math.exp(0.0))) < 1e-12
    assert abs(turned["rgb"][0][0] - op / (1.0 + math.exp(4.0 * g))) < 1e-12


def test_actor_adjoint_matches_finite_differences(oracle_lib):
    """The adjoint of the actor render (static and actor record scalars) equals
    central differences of the render itself, with moving actors seen by a
    rolling-shutter camera; its rounding bound dominates it."""
    sc = synth.random_multilevel_scene(seed=1, max_level=2, dims=(6, 5, 4), p_occ=0.35)
    acts = [synth.actor_shell(1.0, 0.6, 0.5, seed=10), synth.actor_shell(0.8, 0.6, 0.7, seed=11)]
    tracks = [(_rigid(0.3, (0.3, 0.4, 0.6)), _rigid(0.45, (0.5, 0.45, 0.6))),
              (_rigid(-0.5, (1.6, 1.3, 0.4)), _rigid(-0.4, (1.7, 1.3, 0.4)))]
    cam = synth.pinhole(24, 18, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15),
                        synth.camera_pose_looking((-2.0, 0.7, 1.1), 0.25), t0=0.0, t1=0.1,
                        rolling_shutter=True)
    R = 24 * 18
    rng = np.random.default_rng(7)
    g = dict(g_rgb=rng.normal(size=(R, 3)), g_depth=rng.normal(size=R) * 0.1,
             g_opacity=rng.normal(size=R), g_intensity=rng.normal(size=R))
    kw = dict(t_min=0.0, background=(0.3, 0.1, 0.7), want_intensity=True, brute_force=True)
    osc = oracle_lib.OracleScene(sc)
    oac = [oracle_lib.OracleScene(a) for a in acts]
    actors = [(o, p0, p1, 10000 * (k + 1)) for k, (o, (p0, p1)) in enumerate(zip(oac, tracks))]
    (grad, agrads), (bnd, abnds) = oracle_lib.backward_actors(osc, actors, cam, **g, **kw,
                                                              bound=True)
    assert np.all(bnd >= np.abs(grad))
    for a, b in zip(agrads, abnds):
        assert np.all(b >= np.abs(a))

    def loss():
        r = oracle_lib.render_actors(osc, actors, cam, **kw)
        return float((g["g_rgb"] * r["rgb"]).sum() + (g["g_depth"] * r["depth"]).sum() +
                     (g["g_opacity"] * r["opacity"]).sum() +
                     (g["g_intensity"] * r["intensity"]).sum())

    cols = list(range(0, 25)) + list(range(27, 31))
    checked = 0
    for target, gr, params in [(osc, grad, sc.params)] + \
            [(o, ag, a.params) for o, ag, a in zip(oac, agrads, acts)]:
        hit = np.where(np.abs(gr).sum(1) > 0)[0]
        assert len(hit) >= 3
        for v in rng.choice(hit, size=min(3, len(hit)), replace=False):
            rec = params[v].astype(np.float64).copy()
            for c in rng.choice(cols, size=8, replace=False):
                h = 1e-6 * max(1.0, abs(rec[c]))
                p = rec.copy()
                p[c] += h
                target.set_record(v, p)
                lp = loss()
                p[c] = rec[c] - h
                target.set_record(v, p)
                lm = loss()
                target.set_record(v, rec)
                fd = (lp - lm) / (2 * h)
                assert abs(fd - gr[v, c]) <= 1e-6 * abs(gr[v, c]) + 1e-8, (v, c, fd, gr[v, c])
                checked += 1
    assert checked >= 60
    # scalars the field mode does not use get no gradient
    assert np.all(grad[:, 25:27] == 0) and np.all(grad[:, 31] == 0)
