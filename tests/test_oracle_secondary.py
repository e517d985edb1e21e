"""Pins of the oracle's secondary rays (reflection, refraction, shadow at the
expected hit point; Sec. V-C, Fig. 1): each step checked against geometry the
formulas must satisfy, not against a retyped formula."""

import numpy as np

import synth


def _rec(g, b):
    r = np.zeros(32)
    r[:3] = g
    r[3] = b
    return r


def _slab(o, d, lo, hi):
    """Chord [ta, tb] of the ray with the box [lo, hi] (independent slab test)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - o) / d
        t2 = (hi - o) / d
    ta = np.nanmax(np.minimum(t1, t2))
    tb = np.nanmin(np.maximum(t1, t2))
    return max(ta, 0.0), tb


def _voxel_scene(g, b=0.0):
    return synth.single_voxel_scene(_rec(g, b), s0=1.0, dims=(1, 1, 1))


def test_hit_point_is_the_chord_midpoint(oracle_lib):
    """One voxel is composited once, at its chord's midpoint (Eq. 3-4 with a
    midpoint sample), so D / O is that midpoint's distance."""
    sc = _voxel_scene((0.3, -0.7, 0.4), 0.5)
    osc = oracle_lib.OracleScene(sc)
    cam = synth.pinhole(24, 18, 70.0, synth.camera_pose_looking((-1.6, 0.3, 0.6), 0.25))
    out = oracle_lib.render(osc, cam, t_min=0.0)
    rays = oracle_lib.gen_rays(cam)
    sec = oracle_lib.secondary_rays(osc, cam, out["depth"], out["opacity"], kind="shadow",
                                    min_opacity=1e-12, offset=0.0)
    n_hit = 0
    for i in range(len(sec)):
        ta, tb = _slab(rays["o"][i], rays["d"][i], np.zeros(3), np.ones(3))
        if tb - ta > 1e-9:
            n_hit += 1
            mid = rays["o"][i] + 0.5 * (ta + tb) * rays["d"][i]
            assert np.abs(sec[i, :3] - mid).max() < 1e-9, i
        else:
            assert not sec[i].any(), i
    assert n_hit > 50


def _law_checks(d, w, kind, eta, g):
    """Reflection / refraction laws about the plane normal to g (either sign)."""
    m = g / np.linalg.norm(g)
    assert abs(np.linalg.norm(w) - 1.0) < 1e-12
    # coplanar with d and the normal
    assert abs(np.linalg.det(np.stack([d, w, m]))) < 1e-12
    if kind == "reflect":
        assert abs(w @ m + d @ m) < 1e-12          # angle of reflection = incidence
        assert np.linalg.norm(np.cross(w - d, m)) < 1e-12
    else:
        # Snell: sin(transmitted) = eta sin(incident), continuing through
        assert abs(np.linalg.norm(np.cross(w, m)) - eta * np.linalg.norm(np.cross(d, m))) < 1e-12
        assert (w @ m) * (d @ m) > 0


def test_reflection_and_refraction_laws(oracle_lib):
    rng = np.random.default_rng(0)
    cam = synth.pinhole(20, 16, 70.0, synth.camera_pose_looking((-1.8, 0.5, 0.5), 0.2))
    for _ in range(6):
        g = rng.normal(size=3)
        sc = _voxel_scene(g, 0.2)
        osc = oracle_lib.OracleScene(sc)
        out = oracle_lib.render(osc, cam, t_min=0.0)
        rays = oracle_lib.gen_rays(cam)
        for kind, eta in (("reflect", 1.0), ("refract", 1 / 1.33), ("refract", 0.9)):
            sec = oracle_lib.secondary_rays(osc, cam, out["depth"], out["opacity"], kind=kind,
                                            eta=eta, min_opacity=1e-12, offset=0.0)
            ok = np.where(sec[:, 3:6].any(axis=1))[0]
            assert len(ok) > 30
            for i in ok:
                _law_checks(rays["d"][i], sec[i, 3:6], kind, eta, g)


def test_horizontal_interface_textbook_cases(oracle_lib):
    """Field growing upward (g = +z): the surface normal is vertical.  A ray
    going down mirrors to z -> -z above the surface; refraction scales the
    horizontal part by eta below it; past the critical angle it reflects."""
    sc = _voxel_scene((0.0, 0.0, 1.0), 0.0)
    osc = oracle_lib.OracleScene(sc)
    o = np.array([[0.5 - 2.0, 0.5, 0.5 + 1.0], [0.5 - 0.3, 0.5 + 0.1, 0.5 + 1.0],
                  [0.5 - 3.0, 0.5, 0.5 + 0.4]])
    target = np.array([0.5, 0.5, 0.5])
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, d, np.zeros((3, 2))], axis=1)
    sen = synth.explicit_rays(rays, np.float64)
    depth = np.linalg.norm(target - o, axis=1)  # D / O = distance to the target point
    opac = np.ones(3)
    X = target
    ref = oracle_lib.secondary_rays(osc, sen, depth, opac, kind="reflect", offset=0.01)
    for i in range(3):
        assert np.allclose(ref[i, 3:6], d[i] * np.array([1, 1, -1]), atol=1e-12)
        assert np.allclose(ref[i, :3], X + [0, 0, 0.01], atol=1e-12)   # incident side
    eta = 1 / 1.5
    rf = oracle_lib.secondary_rays(osc, sen, depth, opac, kind="refract", eta=eta, offset=0.01)
    for i in range(3):
        assert np.allclose(rf[i, 3:5], eta * d[i, :2], atol=1e-12)
        assert rf[i, 5] < 0 and abs(np.linalg.norm(rf[i, 3:6]) - 1) < 1e-12
        assert np.allclose(rf[i, :3], X - [0, 0, 0.01], atol=1e-12)    # far side
    # from the dense side (eta > 1) a grazing ray is totally reflected
    tir = oracle_lib.secondary_rays(osc, sen, depth, opac, kind="refract", eta=1.5, offset=0.0)
    sin_i = np.linalg.norm(d[:, :2], axis=1)
    for i in range(3):
        if 1.5 * sin_i[i] > 1.0:
            assert np.allclose(tir[i, 3:6], d[i] * np.array([1, 1, -1]), atol=1e-12)
        else:
            assert np.allclose(tir[i, 3:5], 1.5 * d[i, :2], atol=1e-12)
    assert (1.5 * sin_i > 1.0).any() and (1.5 * sin_i <= 1.0).any()


def test_shadow_direction_and_no_ray_cases(oracle_lib):
    sc = _voxel_scene((0.2, 0.1, -0.5), 0.0)
    osc = oracle_lib.OracleScene(sc)
    cam = synth.pinhole(16, 12, 70.0, synth.camera_pose_looking((-1.5, 0.5, 0.5), 0.0))
    out = oracle_lib.render(osc, cam, t_min=0.0)
    L = np.array([1.0, -2.0, 3.0])
    sh = oracle_lib.secondary_rays(osc, cam, out["depth"], out["opacity"], kind="shadow",
                                   light_dir=L, min_opacity=1e-12, t_far=7.0)
    ok = sh[:, 3:6].any(axis=1)
    assert ok.sum() > 20
    assert np.allclose(sh[ok, 3:6], L / np.linalg.norm(L), atol=1e-15)
    assert np.all(sh[ok, 7] == 7.0) and np.all(sh[ok, 6] == 0.0)
    # below the opacity threshold: no ray
    hi = oracle_lib.secondary_rays(osc, cam, out["depth"], out["opacity"], kind="shadow",
                                   min_opacity=1.0)
    assert not hi.any()
    # zero slopes: no normal, no ray
    flat = oracle_lib.OracleScene(_voxel_scene((0.0, 0.0, 0.0), 0.5))
    out0 = oracle_lib.render(flat, cam, t_min=0.0)
    assert not oracle_lib.secondary_rays(flat, cam, out0["depth"], out0["opacity"],
                                         min_opacity=1e-12).any()
    # the expected hit point falls in the empty cell between two equal voxels
    rec = _rec((0.0, 0.0, 1.0), np.log(0.05))
    two = synth.single_voxel_scene(np.stack([rec, rec]), s0=1.0, dims=(3, 1, 1),
                                   cells=[(0, 0, 0), (2, 0, 0)], levels=[0, 0])
    otwo = oracle_lib.OracleScene(two)
    ray = synth.explicit_rays(np.array([[-1.0, 0.5, 0.5, 1.0, 0.0, 0.0, 0.0, 0.0]]), np.float64)
    o2 = oracle_lib.render(otwo, ray, t_min=0.0)
    xs = -1.0 + o2["depth"][0] / o2["opacity"][0]
    assert 1.0 < xs < 2.0
    assert not oracle_lib.secondary_rays(otwo, ray, o2["depth"], o2["opacity"],
                                         min_opacity=1e-12).any()


def test_voxel_at_matches_brute_force(oracle_lib):
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(4, 3, 3), p_occ=0.6)
    osc = oracle_lib.OracleScene(sc)
    rng = np.random.default_rng(1)
    org = np.asarray(sc.origin)
    ext = np.asarray(sc.dims) * sc.s0
    edge = sc.s0 / (1 << sc.level.astype(np.int64))
    lo = org + sc.ijk * edge[:, None]
    hits = 0
    for X in org + rng.uniform(-0.1, 1.1, size=(400, 3)) * ext:
        inside = np.where(np.all((lo <= X) & (X < lo + edge[:, None]), axis=1))[0]
        want = int(inside[0]) if len(inside) else -1
        assert len(inside) <= 1
        assert oracle_lib.voxel_at(osc, X) == want
        hits += want >= 0
    assert hits > 100
