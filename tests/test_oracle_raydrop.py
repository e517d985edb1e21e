"""Pins of the oracle's raydrop output (Sec. V-C, Table III name LiDAR raydrop;
the paper gives no form): a per-voxel logit rho (record slot 31) composited
like intensity, plus T_end for a ray that leaves the scene.  Checked against
a closed form, the telescoping identity at the logit's limits, and central
differences of the adjoint."""

import math

import numpy as np

import synth


def _slab(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - o) / d
        t2 = (hi - o) / d
    return max(np.nanmax(np.minimum(t1, t2)), 0.0), np.nanmin(np.maximum(t1, t2))


def test_single_constant_voxel_closed_form(oracle_lib):
    rec = np.zeros(32)
    sigma, rho = 1.7, 0.8
    rec[3] = math.log(sigma)
    rec[31] = rho
    sc = synth.single_voxel_scene(rec, s0=1.0, dims=(1, 1, 1))
    osc = oracle_lib.OracleScene(sc)
    cam = synth.pinhole(20, 16, 70.0, synth.camera_pose_looking((-1.7, 0.4, 0.6), 0.2))
    out = oracle_lib.render(osc, cam, t_min=0.0, want_raydrop=True)
    rays = oracle_lib.gen_rays(cam)
    s = 1.0 / (1.0 + math.exp(-rho))
    n_hit = 0
    for i in range(len(out["raydrop"])):
        ta, tb = _slab(rays["o"][i], rays["d"][i], np.zeros(3), np.ones(3))
        L = max(tb - ta, 0.0)
        a = 1.0 - math.exp(-sigma * L)
        assert abs(out["raydrop"][i] - (a * s + (1.0 - a))) < 1e-12, i
        n_hit += L > 0
    assert n_hit > 40


def test_logit_limits_and_range(oracle_lib):
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(5, 4, 3), p_occ=0.6)
    cam = synth.lidar(16, 64, synth.lidar_pose((0.4, 0.5, 0.9), 0.3),
                      synth.lidar_pose((0.6, 0.6, 0.9), 0.4), t0=0.0, t1=0.1)
    rng = np.random.default_rng(0)
    for t_min in (0.0, 1e-4):
        P = np.asarray(sc.params, np.float64).copy()
        P[:, 31] = rng.normal(size=len(P)) * 2.0
        out = oracle_lib.render(oracle_lib.OracleScene(sc, params=P), cam, t_min=t_min,
                                want_raydrop=True)
        assert np.all(out["raydrop"] >= 0.0) and np.all(out["raydrop"] <= 1.0 + 1e-12)
        P[:, 31] = -60.0   # sigmoid ~ 0: only rays that leave the scene drop
        lo = oracle_lib.render(oracle_lib.OracleScene(sc, params=P), cam, t_min=t_min,
                               want_raydrop=True)
        assert np.abs(lo["raydrop"] - lo["t_end"]).max() < 1e-20
        P[:, 31] = 60.0    # sigmoid ~ 1: sum of weights + T_end telescopes to 1
        hi = oracle_lib.render(oracle_lib.OracleScene(sc, params=P), cam, t_min=t_min,
                               want_raydrop=True)
        assert np.abs(hi["raydrop"] - 1.0).max() < 1e-12
        assert (lo["t_end"] < 0.9).mean() > 0.3


def test_raydrop_gradient_matches_finite_differences(oracle_lib):
    sc = synth.random_multilevel_scene(seed=5, max_level=1, dims=(3, 3, 2), p_occ=0.8)
    rng = np.random.default_rng(2)
    P = np.asarray(sc.params, np.float64).copy()
    P[:, 31] = rng.normal(size=len(P))
    cam = synth.lidar(8, 24, synth.lidar_pose((0.2, 0.4, 0.8), 0.1),
                      synth.lidar_pose((0.3, 0.45, 0.8), 0.15), t0=0.0, t1=0.1)
    R = 8 * 24
    g = rng.normal(size=R)
    grad = oracle_lib.backward(oracle_lib.OracleScene(sc, params=P), cam, g_raydrop=g, t_min=0.0)

    def loss(Q):
        return float(g @ oracle_lib.render(oracle_lib.OracleScene(sc, params=Q), cam, t_min=0.0,
                                           want_raydrop=True)["raydrop"])

    touched = np.where(np.abs(grad).sum(axis=1) > 0)[0]
    assert len(touched) > 5
    for v in rng.choice(touched, size=min(6, len(touched)), replace=False):
        for c in (0, 1, 2, 3, 31):
            h = 1e-6
            Qp, Qm = P.copy(), P.copy()
            Qp[v, c] += h
            Qm[v, c] -= h
            fd = (loss(Qp) - loss(Qm)) / (2 * h)
            assert abs(fd - grad[v, c]) <= 1e-6 * max(1.0, abs(fd)), (v, c, fd, grad[v, c])
    # raydrop gradients touch only the density field and the logit
    assert np.all(grad[:, 4:31] == 0)
