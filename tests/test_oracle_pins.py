"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms
of Eq. 3-4, identities of the spherical-harmonic basis, hand-derived geometry
(tests/golden), an independent point-membership march, brute force, finite
differences, and analytic sensor geometry.
"""

import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(params, cells=((0, 0, 0),), levels=(0,), dims=(1, 1, 1), K=0, s0=1.0, mode="exp"):
    params = np.atleast_2d(np.asarray(params, dtype=np.float64))
    return synth.single_voxel_scene(params, mode=mode, s0=s0, dims=dims, cells=cells,
                                    levels=levels, max_level=K)


def _rec(**kw):
    r = np.zeros(32)
    for k, v in kw.items():
        if k == "wsig":
            r[0:4] = v
        elif k == "wc":
            r[4:13] = np.asarray(v, dtype=float).ravel()
        elif k == "wsh":
            r[13:25] = np.asarray(v, dtype=float).ravel()
        elif k == "a":
            r[25] = v
        elif k == "b":
            r[26] = v
        elif k == "wint":
            r[27:31] = v
    r[26] = r[26] if r[26] else 0.2
    r[25] = r[25] if r[25] else 1.0
    return r


def _ray_sensor(o, d, t_near=0.0, t_far=0.0):
    rays = np.array([[*o, *d, t_near, t_far]], dtype=np.float32)
    return synth.explicit_rays(rays)


# --------------------------------------------------------------------------
# Eq. 3-4 closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("sigma", [0.05, 0.7, 3.0, 25.0])
def test_single_constant_voxel_closed_form(oracle_lib, sigma):
    """Constant density sigma over a unit path: T = exp(-sigma L) (Eq. 3-4);
    colour sigmoid(0) = 1/2 when every colour weight is 0 (Eq. 2)."""
    sc = _scene(_rec(wsig=[0, 0, 0, math.log(sigma)]))
    osc = oracle_lib.OracleScene(sc)
    sen = _ray_sensor((-1.0, 0.5, 0.5), (1.0, 0.0, 0.0))
    r = oracle_lib.render(osc, sen, t_min=0.0)
    T = math.exp(-sigma * 1.0)
    assert r["t_end"][0] == pytest.approx(T, rel=1e-12)
    assert r["opacity"][0] == pytest.approx(1 - T, rel=1e-12)
    assert np.allclose(r["rgb"][0], 0.5 * (1 - T), rtol=1e-12)
    # entry at t = 1, exit at t = 2: midpoint 1.5
    assert r["depth"][0] == pytest.approx(1.5 * (1 - T), rel=1e-12)
    assert r["n_visits"][0] == 1


def test_chain_of_voxels_closed_form(oracle_lib):
    """Three disjoint voxels in a row: T_end = exp(-sum sigma_i delta_i) and
    the weights T_i alpha_i of Eq. 3 (colours made distinct through W_c at a
    known local coordinate)."""
    sig = [0.4, 1.3, 2.2]
    recs = []
    for i, s in enumerate(sig):
        wc = np.zeros((3, 3))
        wc[0, 1] = 1.0 + i          # red depends on local y
        recs.append(_rec(wsig=[0, 0, 0, math.log(s)], wc=wc))
    sc = _scene(np.array(recs), cells=((0, 0, 0), (1, 0, 0), (2, 0, 0)), levels=(0, 0, 0),
                dims=(3, 1, 1))
    osc = oracle_lib.OracleScene(sc)
    # y = 0.75 -> local y = +0.5 in every voxel
    sen = _ray_sensor((-0.5, 0.75, 0.5), (1.0, 0.0, 0.0))
    r = oracle_lib.render(osc, sen, t_min=0.0)
    T = [1.0]
    for s in sig:
        T.append(T[-1] * math.exp(-s))
    w = [T[i] * (1 - math.exp(-sig[i])) for i in range(3)]
    red = [1 / (1 + math.exp(-(1.0 + i) * 0.5)) for i in range(3)]
    assert r["t_end"][0] == pytest.approx(math.exp(-sum(sig)), rel=1e-12)
    assert r["rgb"][0, 0] == pytest.approx(sum(wi * ci for wi, ci in zip(w, red)), rel=1e-12)
    assert r["rgb"][0, 1] == pytest.approx(0.5 * sum(w), rel=1e-12)
    mids = [1.0, 2.0, 3.0]
    assert r["depth"][0] == pytest.approx(sum(wi * m for wi, m in zip(w, mids)), rel=1e-12)


def test_background_and_premultiplied_colour(oracle_lib):
    sc = _scene(_rec(wsig=[0, 0, 0, math.log(0.9)]))
    osc = oracle_lib.OracleScene(sc)
    sen = _ray_sensor((-1.0, 0.5, 0.5), (1.0, 0.0, 0.0))
    bg = (0.25, 0.5, 1.0)
    r0 = oracle_lib.render(osc, sen, t_min=0.0)
    r1 = oracle_lib.render(osc, sen, t_min=0.0, background=bg)
    assert np.allclose(r1["rgb"][0] - r0["rgb"][0], np.array(bg) * r0["t_end"][0], rtol=1e-12)


# --------------------------------------------------------------------------
# Midpoint sampling (Sec. III-A), hand-derived geometry
# --------------------------------------------------------------------------

def test_midpoint_sampling_hand_cases(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "midpoint_cases.json")))
    wsig = g["record_W_sigma"]
    wc = np.zeros((3, 3))
    wc[0, 1] = 2.0
    rec = _rec(wsig=wsig, wc=wc)
    sc = _scene(rec, cells=((1, 0, 0),), levels=(1,), dims=(1, 1, 1), K=1)
    osc = oracle_lib.OracleScene(sc)
    for case in g["cases"]:
        if "d" in case:
            d = np.array(case["d"])
            tm, delta = case["t_mid"], case["delta"]
        else:
            d = np.array(case["d_unnormalised"]) / math.sqrt(2.0)
            tm, delta = case["t_mid_over_sqrt2"] * math.sqrt(2), case["delta_over_sqrt2"] * math.sqrt(2)
        sen = _ray_sensor(case["o"], d)
        r = oracle_lib.render(osc, sen, t_min=0.0)
        sigma = math.exp(case["W_sigma_dot_xhat"])
        alpha = 1 - math.exp(-sigma * delta)
        assert r["opacity"][0] == pytest.approx(alpha, rel=1e-6)
        assert r["depth"][0] == pytest.approx(alpha * tm, rel=1e-6)
        red = 1 / (1 + math.exp(-2.0 * case["x_local"][1]))
        assert r["rgb"][0, 0] == pytest.approx(alpha * red, rel=1e-6)
        hits = oracle_lib.trace(osc, case["o"], d)
        assert len(hits) == 1
        if "t_entry" in case:
            assert hits[0][1] == pytest.approx(case["t_entry"], abs=1e-7)
            assert hits[0][2] == pytest.approx(case["t_exit"], abs=1e-7)


# --------------------------------------------------------------------------
# Eq. 5-6 (SDF -> density) special cases and symmetry
# --------------------------------------------------------------------------

def test_sdf_density_special_cases(oracle_lib):
    a, b = 3.0, 0.2
    x = np.zeros(3)
    d = np.array([0.0, 0.0, 1.0])

    def sig(s):
        rec = _rec(wsig=[0, 0, 0, s], a=a, b=b)
        return oracle_lib.field(rec, "sdf", x, d)[0]

    assert sig(0.0) == pytest.approx(a / 2, rel=1e-14)          # sign(0) = 0
    assert sig(50.0) == pytest.approx(a, rel=1e-12)             # deep inside
    assert sig(-50.0) == pytest.approx(0.0, abs=1e-12)          # far outside
    for s in [0.01, 0.1, 0.37, 1.2]:
        assert sig(s) + sig(-s) == pytest.approx(a, rel=1e-13)  # Laplace-CDF symmetry
        assert sig(s) > a / 2 > sig(-s)
    h = 1e-8   # slope at the surface a / (2 b); FD error ~ h / (2 b)
    assert (sig(h) - sig(-h)) / (2 * h) == pytest.approx(a / (2 * b), rel=1e-6)
    # Eq. 5: s is the affine field W_s . x-hat (here at x = (0.5, -0.25, 1))
    rec = _rec(wsig=[0.2, 0.4, -0.3, 0.05], a=a, b=b)
    s_val = 0.2 * 0.5 + 0.4 * -0.25 - 0.3 * 1.0 + 0.05
    got = oracle_lib.field(rec, "sdf", np.array([0.5, -0.25, 1.0]), d)[0]
    assert got == pytest.approx(sig(s_val), rel=1e-14)


def test_exp_density_is_exponential_of_affine_field(oracle_lib):
    rec = _rec(wsig=[0.5, -1.0, 0.25, 0.3])
    d = np.array([1.0, 0.0, 0.0])
    s0 = oracle_lib.field(rec, "exp", np.zeros(3), d)[0]
    assert s0 == pytest.approx(math.exp(0.3), rel=1e-14)
    # multiplicative in each coordinate: sigma(x+e_a) / sigma(x) = exp(W_a)
    for a, w in enumerate([0.5, -1.0, 0.25]):
        x = np.array([0.1, -0.2, 0.3])
        x2 = x.copy()
        x2[a] += 0.5
        r = oracle_lib.field(rec, "exp", x2, d)[0] / oracle_lib.field(rec, "exp", x, d)[0]
        assert r == pytest.approx(math.exp(0.5 * w), rel=1e-13)


# --------------------------------------------------------------------------
# gamma(omega): real SH of bands l <= 1
# --------------------------------------------------------------------------

def test_sh_basis_is_orthonormal_on_the_sphere(oracle_lib):
    """Gauss-Legendre x uniform-azimuth quadrature of gamma_i gamma_j over S^2
    must give the identity (real SH are orthonormal)."""
    nt, npz = 16, 32
    xs, ws = np.polynomial.legendre.leggauss(nt)
    G = np.zeros((4, 4))
    for ct, wt in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for k in range(npz):
            ph = 2 * math.pi * k / npz
            g = oracle_lib.sh_basis([st * math.cos(ph), st * math.sin(ph), ct])
            G += np.outer(g, g) * wt * (2 * math.pi / npz)
    assert np.allclose(G, np.eye(4), atol=1e-12)


def test_sh_addition_theorem(oracle_lib):
    """Unsold: sum_m Y_lm(w)^2 = (2l+1)/(4 pi); over l = 0, 1 that is 1/pi."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        g = oracle_lib.sh_basis(w)
        assert float(g @ g) == pytest.approx(1 / math.pi, rel=1e-13)
        assert g[0] ** 2 == pytest.approx(1 / (4 * math.pi), rel=1e-13)


def test_colour_view_dependence_is_odd_in_direction(oracle_lib):
    """Only the l = 1 part of gamma changes sign with the direction, so
    logit c(w) + logit c(-w) = 2 (W_c x + W_sh,0 gamma_0) (Eq. 2)."""
    rng = np.random.default_rng(3)
    rec = _rec(wc=rng.normal(size=9), wsh=rng.normal(size=12))
    x = np.array([0.3, -0.6, 0.2])
    w = np.array([0.48, -0.6, 0.64])
    _, c1, _ = oracle_lib.field(rec, "exp", x, w)
    _, c2, _ = oracle_lib.field(rec, "exp", x, -w)
    _, c0, _ = oracle_lib.field(_rec(wsh=np.tile([1.0, 0, 0, 0], 3)), "exp", np.zeros(3), w)
    g0 = math.log(c0[0] / (1 - c0[0]))            # gamma_0 recovered from a DC-only record
    logit = lambda c: np.log(c / (1 - c))
    wc = rec[4:13].reshape(3, 3)
    wsh = rec[13:25].reshape(3, 4)
    assert np.allclose(logit(c1) + logit(c2), 2 * (wc @ x + wsh[:, 0] * g0), rtol=1e-10)
    assert g0 == pytest.approx(0.5 / math.sqrt(math.pi), rel=1e-13)


# --------------------------------------------------------------------------
# Traversal (Sec. III-B: the octree only accelerates the exhaustive list)
# --------------------------------------------------------------------------

def _owner_grid(scene):
    """Dense finest-level owner map painted voxel by voxel (independent of
    the oracle's lookups)."""
    K = scene.max_level
    dims = [d << K for d in scene.dims]
    own = -np.ones(dims, dtype=np.int64)
    for v in range(scene.n):
        l = int(scene.level[v])
        sh = K - l
        lo = [int(c) << sh for c in scene.ijk[v]]
        hi = [c + (1 << sh) for c in lo]
        assert (own[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] == -1).all()
        own[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = v
    return own


def test_traversal_matches_point_membership_march(oracle_lib):
    """March each ray in steps of 1e-3 finest edges, look up the voxel that
    contains every sample point, and compare the run-length sequence with the
    oracle's hit list and segment lengths."""
    sc = synth.random_multilevel_scene(seed=7, max_level=2, dims=(5, 4, 3))
    osc = oracle_lib.OracleScene(sc)
    own = _owner_grid(sc)
    sf = sc.s0 / (1 << sc.max_level)
    org = np.array(sc.origin)
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(24):
        o = org + np.array([-0.7, rng.uniform(0.1, 1.9), rng.uniform(0.1, 1.4)])
        d = np.array([1.0, rng.uniform(-0.4, 0.4), rng.uniform(-0.3, 0.3)])
        d /= np.linalg.norm(d)
        h = 1e-3 * sf
        ts = np.arange(0.0, 4.5, h) + 0.5 * h
        p = (o[None, :] + ts[:, None] * d[None, :] - org) / sf
        c = np.floor(p).astype(np.int64)
        inside = np.all((c >= 0) & (c < np.array(own.shape)), axis=1)
        ids = np.full(ts.shape, -1)
        ids[inside] = own[c[inside, 0], c[inside, 1], c[inside, 2]]
        seq, lens = [], []
        for v in ids:
            if seq and seq[-1] == v:
                lens[-1] += h
            else:
                seq.append(v)
                lens.append(h)
        runs = [(v, L) for v, L in zip(seq, lens) if v >= 0]
        hits = [(v, b - a) for v, a, b in oracle_lib.trace(osc, o, d)]
        hd, rd = dict(hits), dict(runs)
        assert len(rd) == len(runs)       # a convex voxel is entered once
        # grazing segments (a few steps long) are below the march's resolution
        for v, L in hits:
            if L > 8 * h:
                assert v in rd and abs(rd[v] - L) <= 2.5 * h
                checked += 1
        for v, L in runs:
            if L > 8 * h:
                assert v in hd and abs(hd[v] - L) <= 2.5 * h
        common = [v for v, _ in hits if v in rd]
        assert common == [v for v, _ in runs if v in hd]
    assert checked > 20


@pytest.mark.parametrize("seed,K", [(0, 1), (1, 2), (2, 3), (3, 2)])
def test_dda_candidates_equal_brute_force(oracle_lib, seed, K):
    sc = synth.random_multilevel_scene(seed=seed, max_level=K, dims=(6, 5, 4))
    osc = oracle_lib.OracleScene(sc)
    sensors = [
        synth.pinhole(48, 36, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
        synth.fisheye(40, 30, 190.0, synth.camera_pose_looking((0.4, 0.8, 1.0), 1.1)),
        synth.lidar(16, 90, synth.lidar_pose((0.35, 0.55, 1.05), 0.2)),
    ]
    for sen in sensors:
        a = oracle_lib.render(osc, sen, t_min=0.0, brute_force=True, visits_cap=64)
        b = oracle_lib.render(osc, sen, t_min=0.0, brute_force=False, visits_cap=64)
        assert np.array_equal(a["visits"], b["visits"])
        assert np.allclose(a["rgb"], b["rgb"], atol=1e-13)


def test_hits_are_disjoint_and_ordered(oracle_lib):
    sc = synth.random_multilevel_scene(seed=5, max_level=3)
    osc = oracle_lib.OracleScene(sc)
    rng = np.random.default_rng(2)
    for _ in range(50):
        o = np.array(sc.origin) + rng.uniform(-1, 4, size=3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        hits = oracle_lib.trace(osc, o, d)
        segs = [(max(a, 0.0), b) for _, a, b in hits]
        for (a0, b0), (a1, b1) in zip(segs, segs[1:]):
            assert b0 <= a1 + 1e-12       # Sec. III-D: segments do not overlap
            assert a0 < b0


# --------------------------------------------------------------------------
# Invariants and early termination
# --------------------------------------------------------------------------

def test_compositing_invariants(oracle_lib):
    sc = synth.tiny_scene(seed=1)
    osc = oracle_lib.OracleScene(sc)
    cam = synth.pinhole(64, 48, 60.0, np.concatenate([np.eye(3), [[3.2], [3.2], [-8.0]]], 1))
    r = oracle_lib.render(osc, cam, t_min=0.0, want_intensity=True)
    O = r["opacity"]
    assert (O >= 0).all() and (O <= 1).all()
    assert np.allclose(O, 1 - r["t_end"], atol=1e-14)          # sum w = 1 - T_end
    assert (r["rgb"] >= 0).all() and (r["rgb"] <= O[:, None] + 1e-15).all()
    assert (r["intensity"] <= O + 1e-15).all()


def test_early_termination_bound(oracle_lib):
    sc = synth.random_multilevel_scene(seed=3, max_level=2, p_occ=0.9, dims=(6, 5, 4))
    sc.params[:, 3] += 2.0   # denser, so that termination actually happens
    osc = oracle_lib.OracleScene(sc)
    cam = synth.pinhole(48, 36, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    t_min = 1e-3
    a = oracle_lib.render(osc, cam, t_min=0.0)
    b = oracle_lib.render(osc, cam, t_min=t_min)
    assert (b["n_visits"] < a["n_visits"]).any()
    assert np.abs(a["rgb"] - b["rgb"]).max() <= t_min
    assert np.abs(a["opacity"] - b["opacity"]).max() <= t_min
    tmax = 12.0
    assert np.abs(a["depth"] - b["depth"]).max() <= t_min * tmax
    stopped = b["n_visits"] < a["n_visits"]
    assert (b["t_end"][stopped] < t_min).all()


def test_permutation_invariance(oracle_lib):
    sc = synth.random_multilevel_scene(seed=4, max_level=2)
    sc2, perm = synth.shuffle_scene(sc, 9)
    cam = synth.pinhole(48, 36, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    a = oracle_lib.render(oracle_lib.OracleScene(sc), cam, visits_cap=32)
    b = oracle_lib.render(oracle_lib.OracleScene(sc2), cam, visits_cap=32)
    assert np.allclose(a["rgb"], b["rgb"], atol=1e-14)
    mapped = np.where(b["visits"] >= 0, perm[np.maximum(b["visits"], 0)], -1)
    assert np.array_equal(a["visits"], mapped)


# --------------------------------------------------------------------------
# Scene validation (Sec. III-D disjointness)
# --------------------------------------------------------------------------

def test_overlap_and_range_rejected(oracle_lib):
    r = _rec()
    ok = _scene(np.stack([r, r]), cells=((0, 0, 0), (1, 0, 0)), levels=(0, 0), dims=(2, 1, 1))
    assert oracle_lib.OracleScene(ok).status == 0
    dup = _scene(np.stack([r, r]), cells=((0, 0, 0), (0, 0, 0)), levels=(0, 0), dims=(2, 1, 1))
    assert oracle_lib.OracleScene(dup).status == 4
    anc = _scene(np.stack([r, r]), cells=((1, 0, 0), (3, 1, 0)), levels=(0, 1), dims=(2, 1, 1), K=1)
    assert oracle_lib.OracleScene(anc).status == 4
    deep = _scene(np.stack([r, r]), cells=((1, 0, 0), (13, 2, 3)), levels=(0, 3), dims=(2, 1, 1), K=3)
    assert oracle_lib.OracleScene(deep).status == 4
    out = _scene(np.stack([r]), cells=((2, 0, 0),), levels=(0,), dims=(2, 1, 1))
    assert oracle_lib.OracleScene(out).status == 1
    bad_sdf = _scene(_rec(a=-1.0), mode="sdf")
    assert oracle_lib.OracleScene(bad_sdf).status == 1


# --------------------------------------------------------------------------
# Sensors (Fig. 2, Sec. V-C)
# --------------------------------------------------------------------------

def test_pinhole_geometry(oracle_lib):
    pose = synth.camera_pose_looking((1.0, 2.0, 3.0), 0.7)
    cam = synth.pinhole(101, 61, 60.0, pose)
    rays = oracle_lib.gen_rays(cam, [30 * 101 + 50, 0])
    assert np.allclose(rays["d"][0], pose[:, 2], atol=1e-15)   # centre pixel -> optical axis
    assert np.allclose(rays["o"], pose[:, 3])
    # corner pixel: angle to the axis from the pinhole relation
    f = 50.5 / math.tan(math.radians(30))
    ex = math.hypot(50.0, 30.0) / f
    assert math.acos(float(rays["d"][1] @ pose[:, 2])) == pytest.approx(math.atan(ex), rel=1e-12)


def test_fisheye_equidistant(oracle_lib):
    pose = synth.camera_pose_looking((0, 0, 0), 0.0)
    cam = synth.fisheye(200, 120, 190.0, pose)
    f = cam["fx"]
    idx = np.arange(200 * 120)
    rays = oracle_lib.gen_rays(cam, idx)
    u = idx % 200 + 0.5
    v = idx // 200 + 0.5
    r = np.hypot(u - 100, v - 60)
    theta = np.arccos(np.clip(rays["d"] @ pose[:, 2], -1, 1))
    valid = rays["valid"]
    assert np.allclose(theta[valid], (r / f)[valid], atol=1e-12)   # r = f theta
    assert np.array_equal(valid, r / f <= math.radians(95))
    assert (~valid).any() and valid.sum() > 0.5 * len(valid)


def test_panorama_geometry(oracle_lib):
    pose = synth.camera_pose_looking((0, 0, 0), 0.0)
    W, H = 64, 16
    cam = synth.panorama(W, H, pose)
    rays = oracle_lib.gen_rays(cam)
    d = rays["d"].reshape(H, W, 3)
    elev = np.degrees(np.arcsin(d[..., 2]))
    step = 360.0 / W
    assert np.allclose(elev[:, 0], 45.0 - step * (np.arange(H) + 0.5), atol=1e-10)
    az = np.degrees(np.arctan2(d[..., 1], d[..., 0]))   # world heading
    # columns advance by 360/W; the image centre looks along the camera axis (+x)
    daz = np.diff(np.unwrap(np.radians(az[5])))
    assert np.allclose(np.abs(np.degrees(daz)), step, atol=1e-9)
    mid = d[H // 2, W // 2 - 1] + d[H // 2, W // 2]
    assert mid[0] > 0 and abs(mid[1]) < 1e-12


def test_lidar_beams_azimuths_times(oracle_lib):
    p0 = synth.lidar_pose((0.0, 0.0, 1.9), 0.0)
    p1 = synth.lidar_pose((1.0, 0.0, 1.9), 0.02)
    sen = synth.lidar(128, 2048, p0, p1, t0=0.0, t1=0.1)
    idx = np.array([0, 127 * 2048, 512, 1024, 2047])
    rays = oracle_lib.gen_rays(sen, idx)
    el = np.degrees(np.arcsin(rays["d"][:, 2]))
    assert el[0] == pytest.approx(15.0, abs=1e-12)
    assert el[1] == pytest.approx(-25.0, abs=1e-12)
    assert np.allclose(rays["tau"], [0.0, 0.0, 0.025, 0.05, 0.1 * 2047 / 2048], atol=1e-15)
    assert rays["d"][0][1] == 0.0 and rays["d"][0][0] > 0            # azimuth 0 = sensor +x
    assert np.allclose(rays["o"][3], [0.5, 0.0, 1.9], atol=1e-15)      # linear translation
    # column 1024 at tau = 0.05: half the yaw (slerp) plus azimuth 180 degrees
    h = math.degrees(math.atan2(rays["d"][3][1], rays["d"][3][0]))
    assert h == pytest.approx(-180.0 + math.degrees(0.01), abs=1e-9) or \
        h == pytest.approx(180.0 + math.degrees(0.01), abs=1e-9)


def test_rolling_shutter_pose_interpolation(oracle_lib):
    psi = 0.3
    p0 = synth.camera_pose_looking((0.0, 0.0, 1.0), 0.0)
    p1 = synth.camera_pose_looking((2.0, 1.0, 1.0), 2 * psi)
    cam = synth.pinhole(9, 5, 60.0, p0, p1, t0=0.0, t1=0.04, rolling_shutter=True)
    R0, t0 = oracle_lib.pose_at(cam, 0.0)
    R1, t1 = oracle_lib.pose_at(cam, 0.04)
    Rm, tm = oracle_lib.pose_at(cam, 0.02)
    assert np.allclose(R0, p0[:, :3], atol=1e-15) and np.allclose(R1, p1[:, :3], atol=1e-13)
    assert np.allclose(Rm, synth.camera_pose_looking((0, 0, 0), psi)[:, :3], atol=1e-13)
    assert np.allclose(tm, [1.0, 0.5, 1.0], atol=1e-15)
    rays = oracle_lib.gen_rays(cam, [0, 4 * 9])
    assert np.allclose(rays["tau"], [0.0, 0.04])
    assert np.allclose(rays["o"][1], [2.0, 1.0, 1.0])
    glob = synth.pinhole(9, 5, 60.0, p0, p1, t0=0.0, t1=0.04, rolling_shutter=False)
    rg = oracle_lib.gen_rays(glob, [4 * 9])
    assert np.allclose(rg["o"][0], [0.0, 0.0, 1.0]) and rg["tau"][0] == 0.0


# --------------------------------------------------------------------------
# Adjoint vs central finite differences
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["exp", "sdf"])
def test_adjoint_matches_finite_differences(oracle_lib, mode):
    sc = synth.random_multilevel_scene(seed=12, max_level=2, dims=(4, 3, 3), p_occ=0.8,
                                       mode=mode)
    cam = synth.pinhole(12, 9, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    rng = np.random.default_rng(5)
    R = 12 * 9
    g = dict(g_rgb=rng.normal(size=(R, 3)), g_depth=rng.normal(size=R),
             g_opacity=rng.normal(size=R), g_intensity=rng.normal(size=R))
    kw = dict(t_min=0.0, background=(0.3, 0.1, 0.7), want_intensity=True)
    osc = oracle_lib.OracleScene(sc)
    grad = oracle_lib.backward(osc, cam, **g, **kw)

    def loss(params):
        o2 = oracle_lib.OracleScene(sc, params=params)
        r = oracle_lib.render(o2, cam, **kw)
        return float((g["g_rgb"] * r["rgb"]).sum() + (g["g_depth"] * r["depth"]).sum() +
                     (g["g_opacity"] * r["opacity"]).sum() +
                     (g["g_intensity"] * r["intensity"]).sum())

    hit = np.where(np.abs(grad).sum(1) > 0)[0]
    assert len(hit) >= 5
    cols = list(range(0, 25)) + list(range(27, 31)) + ([25, 26] if mode == "sdf" else [])
    picks = [(v, c) for v in rng.choice(hit, size=min(6, len(hit)), replace=False) for c in cols]
    scale = np.abs(grad).max()
    for v, c in picks:
        p = sc.params.astype(np.float64).copy()
        h = 1e-6 * max(1.0, abs(p[v, c]))
        p[v, c] += h
        lp = loss(p)
        p[v, c] -= 2 * h
        lm = loss(p)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[v, c]) <= 1e-6 * max(abs(grad[v, c]), 1e-3 * scale), (v, c, fd, grad[v, c])
    # unused record scalars get no gradient
    assert np.all(grad[:, 31] == 0)
    if mode == "exp":
        assert np.all(grad[:, 25:27] == 0)


def test_dda_candidates_equal_brute_force_deep_octree(oracle_lib):
    """Voxels at every level 0..10: the finest-level walk (2048 cells per axis)
    still enumerates exactly the brute-force hit list."""
    sc = synth.deep_scene(max_level=10, dims=(2, 2, 2), seed=3)
    osc = oracle_lib.OracleScene(sc)
    rng = np.random.default_rng(1)
    tips = [(sc.ijk[v] + 0.5) / 1024.0 for v in np.where(sc.level == 10)[0]]
    for tip in tips:
        for _ in range(16):
            o = np.array(tip) + rng.normal(size=3) * 1.5
            d = np.array(tip) - o + rng.normal(size=3) * 1e-3
            d /= np.linalg.norm(d)
            a = oracle_lib.trace(osc, o, d, brute_force=True)
            b = oracle_lib.trace(osc, o, d, brute_force=False)
            assert [h[0] for h in a] == [h[0] for h in b]


def test_backward_bound_dominates_the_gradient_and_scales_with_it(oracle_lib):
    """orc_backward_bound is a sum of contribution magnitudes, each at least
    the contribution's absolute value: it bounds |gradient| per scalar, is
    zero exactly where no hit contributes, does not depend on the sign of
    the output gradients and scales linearly with their size."""
    for mode in ("exp", "sdf"):
        sc = synth.random_multilevel_scene(seed=12, max_level=2, dims=(4, 3, 3), p_occ=0.8,
                                           mode=mode)
        cam = synth.pinhole(12, 9, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
        R = 12 * 9
        rng = np.random.default_rng(5)
        g = dict(g_rgb=rng.normal(size=(R, 3)), g_depth=rng.normal(size=R),
                 g_opacity=rng.normal(size=R), g_intensity=rng.normal(size=R))
        kw = dict(t_min=1e-3, background=(0.3, 0.1, 0.7), want_intensity=True, brute_force=True)
        osc = oracle_lib.OracleScene(sc)
        grad, bnd = oracle_lib.backward(osc, cam, **g, **kw, bound=True)
        assert np.all(bnd >= np.abs(grad))
        touched = np.abs(grad).sum(1) > 0
        assert np.all(bnd[grad != 0] > 0)
        assert np.all(bnd[~touched] == 0)
        assert np.all(bnd[:, 31] == 0)
        _, b2 = oracle_lib.backward(osc, cam, **{k: -2.0 * v for k, v in g.items()}, **kw,
                                    bound=True)
        assert np.allclose(b2, 2.0 * bnd, rtol=1e-12, atol=0)


def test_set_record_equals_a_scene_built_with_that_record(oracle_lib):
    sc = synth.random_multilevel_scene(seed=7, max_level=1, dims=(4, 3, 3), p_occ=0.8)
    cam = synth.pinhole(16, 12, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    osc = oracle_lib.OracleScene(sc)
    rec = np.random.default_rng(1).normal(size=32)
    osc.set_record(3, rec)
    p = sc.params.astype(np.float64).copy()
    p[3] = rec
    ref = oracle_lib.render(oracle_lib.OracleScene(sc, params=p), cam, t_min=0.0,
                            brute_force=True)
    got = oracle_lib.render(osc, cam, t_min=0.0, brute_force=True)
    for k in ("rgb", "depth", "opacity"):
        assert np.array_equal(got[k], ref[k])
    with pytest.raises(ValueError):
        osc.set_record(sc.n, rec)


def test_conditioned_rays(oracle_lib):
    """A ray through the middle of a row of cells is conditioned; rays along a
    cell plane or through a cell edge are not; and the C check agrees with
    comparing the shrunk and grown visit lists one ray at a time."""
    sc = synth.random_multilevel_scene(seed=2, max_level=1, dims=(4, 4, 4), p_occ=1.0)
    osc = oracle_lib.OracleScene(sc)
    o = np.array(sc.origin, dtype=np.float64)
    s0 = sc.s0
    rows = np.array([
        [*(o + [-1.0, 0.3 * s0, 0.3 * s0]), 1, 0, 0, 0.0, 0.0],   # inside a row of cells
        [*(o + [-1.0, 1.0 * s0, 0.3 * s0]), 1, 0, 0, 0.0, 0.0],   # in the plane y = s0
        [*(o + [-1.0, 2.0 * s0, 2.0 * s0]), 1, 0, 0, 0.0, 0.0],   # along a cell edge
    ])
    sen = synth.explicit_rays(rows, np.float64)
    ok = oracle_lib.conditioned(osc, sen, 1e-6, 1e-6)
    assert ok.tolist() == [True, False, False]
    cam = synth.pinhole(24, 18, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    ok = oracle_lib.conditioned(osc, cam, 1e-4 * s0 / 2, 4e-6)
    rays = oracle_lib.gen_rays(cam)
    for i in range(0, 24 * 18, 7):
        a = oracle_lib.trace_eps(osc, rays["o"][i], rays["d"][i], rays["t_near"][i],
                                 rays["t_far"][i], 1e-4 * s0 / 2, 4e-6, -1)
        b = oracle_lib.trace_eps(osc, rays["o"][i], rays["d"][i], rays["t_near"][i],
                                 rays["t_far"][i], 1e-4 * s0 / 2, 4e-6, +1)
        assert ok[i] == (a == b)
