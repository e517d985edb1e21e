"""Pins of the oracle's densification and pruning (Sec. III-C)."""

import math

import numpy as np

import synth


def _rand_record(rng, mode):
    r = rng.normal(size=32)
    if mode == "sdf":
        r[25] = rng.uniform(0.5, 3.0)
        r[26] = rng.uniform(0.05, 0.5)
    r[31] = 0.0
    return r


def test_child_fields_equal_the_parent_field(oracle_lib):
    """Each child's density, colour and intensity at its local x equal the
    parent's at the same point, x_parent = (x_child + o) / 2."""
    rng = np.random.default_rng(0)
    for mode in ("exp", "sdf"):
        for _ in range(40):
            rec = _rand_record(rng, mode)
            c = int(rng.integers(8))
            child = oracle_lib.subdivide_record(rec, c)
            o = np.array([1.0 if (c >> a) & 1 else -1.0 for a in range(3)])
            x = rng.uniform(-1, 1, size=3)
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            sp, cp, ip = oracle_lib.field(rec, mode, (x + o) / 2.0, d)
            sc, cc, ic = oracle_lib.field(child, mode, x, d)
            assert abs(sp - sc) <= 1e-12 * max(1.0, abs(sp))
            assert np.abs(cp - cc).max() < 1e-12 and abs(ip - ic) < 1e-12
            assert child[25] == rec[25] and child[26] == rec[26]


def test_splitting_a_constant_voxel_changes_no_render(oracle_lib):
    """Constant fields: the 8 children composite to the parent's outputs
    (optical depths add up, colour is the same everywhere)."""
    rec = np.zeros(32)
    rec[3] = math.log(1.3)
    rec[13], rec[17], rec[21] = 1.0, -0.5, 0.25
    rec[30] = 0.7
    parent = synth.single_voxel_scene(rec, s0=1.0, dims=(1, 1, 1), max_level=1)
    lv, ij, pr, act = oracle_lib.refine(parent, np.ones((1, 32)), np.ones(1), 0.0)
    assert list(act) == [1] and len(lv) == 8
    kids = synth.SceneData(parent.origin, 1.0, (1, 1, 1), 1, lv, ij, pr, "exp", "kids")
    cam = synth.pinhole(24, 18, 80.0, synth.camera_pose_looking((-1.5, 0.4, 0.55), 0.2))
    a = oracle_lib.render(oracle_lib.OracleScene(parent), cam, t_min=0.0, want_intensity=True)
    b = oracle_lib.render(oracle_lib.OracleScene(kids), cam, t_min=0.0, want_intensity=True)
    assert a["opacity"].max() > 0.3
    for k in ("rgb", "opacity", "intensity"):
        assert np.abs(a[k] - b[k]).max() < 1e-12, k


def test_refine_bookkeeping(oracle_lib):
    """Volume is conserved except for pruned voxels, the result is disjoint,
    exactly the low-alpha voxels are pruned, finest voxels never split."""
    sc = synth.random_multilevel_scene(seed=6, max_level=2, dims=(6, 5, 4), p_occ=0.6)
    rng = np.random.default_rng(1)
    n = len(sc.level)
    grads = rng.normal(size=(n, 32)) * rng.uniform(0, 1, size=(n, 1))
    ma = rng.uniform(0, 0.01, size=n)
    thr = float(np.quantile(np.abs(grads[:, 4:13]).sum(axis=1), 0.7))
    lv, ij, pr, act = oracle_lib.refine(sc, grads, ma, thr, prune_alpha=1e-3)
    g1 = np.abs(grads[:, 4:13]).sum(axis=1)
    assert np.array_equal(act == 2, ma < 1e-3)
    assert np.array_equal(act == 1, (ma >= 1e-3) & (g1 > thr) & (sc.level < sc.max_level))
    assert (act == 1).sum() > 5 and (act == 2).sum() > 5
    vol = lambda lev: (0.5 ** lev.astype(float)) ** 3
    assert abs(vol(lv).sum() - vol(sc.level[act != 2]).sum()) < 1e-12
    out = synth.SceneData(sc.origin, sc.s0, sc.dims, sc.max_level, lv, ij, pr, sc.mode, "refined")
    assert oracle_lib.OracleScene(out).ok  # disjoint (no overlap reported)
    # kept voxels keep their records; children carry the parent's fields
    k = 0
    for v in range(n):
        if act[v] == 0:
            assert np.array_equal(pr[k], sc.params[v]); k += 1
        elif act[v] == 1:
            assert np.allclose(pr[k], oracle_lib.subdivide_record(sc.params[v], 0)); k += 8


def test_max_alpha_is_the_largest_composited_alpha(oracle_lib):
    """Recorded per-voxel alpha maxima equal a brute-force pass over the same
    rays' hits (trace + field at each midpoint)."""
    sc = synth.random_multilevel_scene(seed=7, max_level=1, dims=(4, 4, 3), p_occ=0.5)
    osc = oracle_lib.OracleScene(sc)
    cam = synth.pinhole(16, 12, 70.0, synth.camera_pose_looking((-2.0, 0.4, 1.0), 0.2))
    ma = np.zeros(len(sc.level))
    oracle_lib.render(osc, cam, t_min=0.0, max_alpha=ma)
    ref = np.zeros(len(sc.level))
    rays = oracle_lib.gen_rays(cam)
    for i in range(len(rays["o"])):
        o, d = rays["o"][i], rays["d"][i]
        for v, a, b in oracle_lib.trace(osc, o, d, 0.0, np.inf):
            e = sc.s0 / (1 << int(sc.level[v]))
            lo = np.asarray(sc.origin) + sc.ijk[v] * e
            tm = 0.5 * (max(a, 0.0) + b)
            x = (o + tm * d - (lo + 0.5 * e)) / (0.5 * e)
            sig = oracle_lib.field(sc.params[v], sc.mode, x, d)[0]
            ref[v] = max(ref[v], 1.0 - math.exp(-sig * (b - max(a, 0.0))))
    assert (ma > 0).sum() > 10
    assert np.abs(ma - ref).max() < 1e-12


def _affine_params(sc, A, c, rng):
    """Records whose geometry field is the restriction of one global affine
    field G(X) = A . X + c (X in metres)."""
    P = rng.normal(size=(len(sc.level), 32)) * 0.1
    if sc.mode == "sdf":
        P[:, 25] = 1.5
        P[:, 26] = 0.3
    for k in range(len(sc.level)):
        e = sc.s0 / (1 << int(sc.level[k]))
        ctr = np.asarray(sc.origin) + (sc.ijk[k] + 0.5) * e
        P[k, :3] = A * (0.5 * e)
        P[k, 3] = A @ ctr + c
    return P


def test_reg_pairs_known_configurations(oracle_lib):
    cells = [(i, j, k) for i in range(2) for j in range(2) for k in range(2)]
    block = synth.single_voxel_scene(np.zeros((8, 32)), dims=(2, 2, 2), cells=cells, levels=[0] * 8)
    assert len(oracle_lib.face_pairs(block)) == 12
    # a level-0 voxel facing four level-1 voxels across its +x face
    cells = [(0, 0, 0)] + [(2, j, k) for j in range(2) for k in range(2)]
    mixed = synth.single_voxel_scene(np.zeros((5, 32)), dims=(2, 1, 1), cells=cells,
                                     levels=[0, 1, 1, 1, 1], max_level=1)
    pairs = oracle_lib.face_pairs(mixed)
    assert len(pairs) == 8  # 4 big-small, 4 among the small ones
    assert sum(1 for p in pairs if p[0] == 0 or p[1] == 0) == 4


def test_reg_vanishes_for_a_global_affine_field(oracle_lib):
    rng = np.random.default_rng(3)
    for mode in ("exp", "sdf"):
        sc = synth.random_multilevel_scene(seed=4, max_level=2, dims=(4, 3, 3), p_occ=0.7, mode=mode)
        P = _affine_params(sc, np.array([0.3, -0.2, 0.5]), 0.1, rng)
        loss, _ = oracle_lib.reg_loss(sc, P, 1.0, 1.0, 1.0)
        assert len(oracle_lib.face_pairs(sc)) > 40
        assert abs(loss) < 1e-9, loss


def test_reg_gradient_matches_finite_differences(oracle_lib):
    rng = np.random.default_rng(5)
    for mode in ("exp", "sdf"):
        sc = synth.random_multilevel_scene(seed=5, max_level=2, dims=(3, 3, 2), p_occ=0.7, mode=mode)
        P = np.asarray(sc.params, dtype=np.float64).copy()
        lam = (0.7, 1.3, 0.4)
        _, grad = oracle_lib.reg_loss(sc, P, *lam)
        cols = [0, 1, 2, 3] + ([25, 26] if mode == "sdf" else [])
        for v in rng.choice(len(P), size=8, replace=False):
            for c in cols:
                h = 1e-6
                Pp, Pm = P.copy(), P.copy()
                Pp[v, c] += h
                Pm[v, c] -= h
                fd = (oracle_lib.reg_loss(sc, Pp, *lam)[0] - oracle_lib.reg_loss(sc, Pm, *lam)[0]) / (2 * h)
                assert abs(fd - grad[v, c]) <= 1e-5 * max(1.0, abs(fd)), (mode, v, c, fd, grad[v, c])
        assert np.all(grad[:, 4:25] == 0) and np.all(grad[:, 27:] == 0)
