"""The rasteriser's front-to-back order, checked on the CPU against exact ray
traces of the oracle.

Tile rasterisation (Sec. III-B, "Tile-based Splatting") composites each tile's
voxels in one sorted order for all of its pixels.  The order used here: level-0
cells by their L1 cell distance from the camera's level-0 cell, then, inside a
cell, octree digits XOR-ed with the camera's side of each split (nearest child
first).  The claim is that for a point camera this order agrees with the
entry order along every ray from it, so the splatted image equals the
ray-cast one.  These tests restate the key and check the claim against the
oracle's exact (FP64, brute-force) hit lists for many rays, scenes and camera
positions, including cameras inside a voxel, outside the grid and on split
planes.
"""

import numpy as np
import pytest

import synth


def camera_order_keys(sc, cam_pos):
    """(L1 distance, digit string) per voxel for a camera at cam_pos."""
    K = sc.max_level
    sfin = sc.s0 / (1 << K)
    e = (np.asarray(cam_pos, dtype=np.float64) - np.asarray(sc.origin)) / sfin
    ei = np.floor(e).astype(np.int64)          # camera's finest cell
    ce = np.floor_divide(ei, 1 << K)           # camera's level-0 cell
    keys = []
    for v in range(len(sc.level)):
        l = int(sc.level[v])
        f = sc.ijk[v].astype(np.int64) << (K - l)
        l1 = int(np.abs((f >> K) - ce).sum())
        dig = 0
        for j in range(1, l + 1):
            dj = 0
            for a in range(3):
                node_lo = (f[a] >> (K - j + 1)) << (K - j + 1)
                mid = node_lo + (1 << (K - j))
                side = 1 if ei[a] >= mid else 0
                dj |= (((f[a] >> (K - j)) & 1) ^ side) << a
            dig |= dj << (3 * (K - j))
        keys.append((l1, dig))
    return keys


def _check(oracle_lib, sc, cam_positions, n_dirs, seed):
    osc = oracle_lib.OracleScene(sc)
    rng = np.random.default_rng(seed)
    checked = 0
    for pos in cam_positions:
        keys = camera_order_keys(sc, pos)
        for _ in range(n_dirs):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            hits = oracle_lib.trace(osc, pos, d, brute_force=True)
            ks = [keys[h[0]] for h in hits]
            assert all(ks[i] < ks[i + 1] for i in range(len(ks) - 1)), (pos, d, hits, ks)
            checked += len(hits) > 1
    return checked


def test_camera_order_matches_ray_order_multilevel(oracle_lib):
    sc = synth.random_multilevel_scene(seed=5, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    lo = np.asarray(sc.origin)
    hi = lo + np.asarray(sc.dims) * sc.s0
    rng = np.random.default_rng(0)
    inside = [lo + rng.random(3) * (hi - lo) for _ in range(6)]
    outside = [lo - 1.0, hi + np.array([0.7, -3.0, 0.4]), np.array([lo[0] - 2, hi[1] + 1, 0.0])]
    # on level-0 split planes and on finer split planes
    plane = [lo + np.array([2 * sc.s0, 1.3, 0.77]), lo + np.array([1.25 * sc.s0, 2 * sc.s0, 0.6])]
    n = _check(oracle_lib, sc, inside + outside + plane, 60, 1)
    assert n > 200


def test_camera_order_matches_ray_order_deep(oracle_lib):
    sc = synth.deep_scene(max_level=6, dims=(2, 2, 2), seed=2)
    rng = np.random.default_rng(3)
    tips = [(sc.ijk[v] + 0.5) / 64.0 for v in np.where(sc.level == 6)[0]]
    cams = [np.array(t) + rng.normal(size=3) * 0.3 for t in tips[:4]] + [np.array([-0.5, 0.3, 2.5])]
    n = _check(oracle_lib, sc, cams, 80, 4)
    assert n > 100


def test_camera_order_matches_ray_order_driving_sample(oracle_lib):
    """The driving scene at reduced size from a street-level camera."""
    sc = synth.driving_scene(60_000, seed=2, ground_extent=30.0, n_actors=20)
    n = _check(oracle_lib, sc, [np.array([0.0, 0.0, 1.7]), np.array([3.1, -2.05, 0.9])], 150, 7)
    assert n > 50


@pytest.mark.parametrize("plant", ["drop_xor", "linf"])
def test_order_check_catches_wrong_keys(oracle_lib, plant):
    """The check above fails for plausible wrong orders (no eye-side flip;
    Chebyshev instead of L1 distance)."""
    sc = synth.random_multilevel_scene(seed=5, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    osc = oracle_lib.OracleScene(sc)
    K = sc.max_level
    sfin = sc.s0 / (1 << K)
    pos = np.asarray(sc.origin) + np.array([1.7, 1.1, 0.9])
    e = np.floor((pos - np.asarray(sc.origin)) / sfin).astype(np.int64)
    ce = e >> K
    keys = []
    for v in range(len(sc.level)):
        l = int(sc.level[v])
        f = sc.ijk[v].astype(np.int64) << (K - l)
        dist = np.abs((f >> K) - ce)
        l1 = int(dist.max() if plant == "linf" else dist.sum())
        dig = 0
        for j in range(1, l + 1):
            dj = 0
            for a in range(3):
                mid = ((f[a] >> (K - j + 1)) << (K - j + 1)) + (1 << (K - j))
                side = 0 if plant == "drop_xor" else (1 if e[a] >= mid else 0)
                dj |= (((f[a] >> (K - j)) & 1) ^ side) << a
            dig |= dj << (3 * (K - j))
        keys.append((l1, dig))
    rng = np.random.default_rng(11)
    bad = 0
    for _ in range(400):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        ks = [keys[h[0]] for h in oracle_lib.trace(osc, pos, d, brute_force=True)]
        bad += any(ks[i] >= ks[i + 1] for i in range(len(ks) - 1))
    assert bad > 0
