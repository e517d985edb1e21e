"""Seeded dynamic actors (Sec. IV-A): voxel sets in their own canonical frame
and synthetic tracks that place them in the world.

Only inputs are drawn here (voxel keys, records, poses); no rendering
arithmetic.
"""

from __future__ import annotations

import math

import numpy as np

from .scenes import SceneData, draw_params


def actor_shell(length: float = 4.4, width: float = 1.9, height: float = 1.6, seed: int = 0,
                mode: str = "exp", params_dtype=np.float32) -> SceneData:
    """A car-sized actor in its canonical frame (x forward, y left, z up, origin
    at the bottom centre of its box): a floor of 0.2 m voxels (level 0) under
    the hollow one-voxel shell of 0.1 m voxels (level 1) of the box above it.
    The grid has 0.2 m cells, K = 1, and is centred on the origin in x and y."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (max(2, int(math.ceil(v / 0.2))) for v in (length, width, height))
    origin = (-0.1 * nx, -0.1 * ny, 0.0)
    fi, fj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    floor = np.stack([fi.ravel(), fj.ravel(), np.zeros(fi.size, np.int64)], axis=1)
    i1, j1, k1 = np.meshgrid(np.arange(2 * nx), np.arange(2 * ny), np.arange(2, 2 * nz),
                             indexing="ij")
    edge = ((i1 == 0) | (i1 == 2 * nx - 1) | (j1 == 0) | (j1 == 2 * ny - 1) | (k1 == 2 * nz - 1))
    shell = np.stack([i1[edge], j1[edge], k1[edge]], axis=1)
    ijk = np.concatenate([floor, shell], axis=0).astype(np.int32)
    level = np.concatenate([np.zeros(floor.shape[0], np.uint8), np.ones(shell.shape[0], np.uint8)])
    params = draw_params(rng, ijk.shape[0], mode, dtype=params_dtype)
    return SceneData(origin, 0.2, (nx, ny, nz), 1, level, ijk, params, mode,
                     f"actor-{nx}x{ny}x{nz}")


def _pose(x, y, z, yaw):
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0, x], [s, c, 0.0, y], [0.0, 0.0, 1.0, z]])


def actor_tracks(n: int, seed: int = 0, t0: float = 0.0, t1: float = 0.1, ground_z: float = 0.2,
                 lanes=(-2.0, 2.0), x_range=(-95.0, 95.0), keep_clear: float = 9.0,
                 speed=(0.0, 15.0), yaw_rate=(-0.3, 0.3), length: float = 5.0):
    """Poses (canonical -> world, 3x4) of n actors at t0 and t1 driving along
    lanes parallel to x (the first lane heading +x, the second -x), spaced so
    that no two boxes of up to `length` metres overlap at t0 or t1, and outside
    |x| < keep_clear (where the sensors sit).  Returns [(pose0, pose1)]."""
    rng = np.random.default_rng(seed)
    dt = t1 - t0
    out = []
    slots = []
    for lane_i, y in enumerate(lanes):
        heading = 0.0 if lane_i % 2 == 0 else math.pi
        x = x_range[0]
        while x < x_range[1]:
            if abs(x) >= keep_clear:
                slots.append((x, y, heading))
            x += length + 2.0 + speed[1] * dt * 2 + rng.uniform(0.5, 6.0)
    if n > len(slots):
        raise ValueError(f"only {len(slots)} actor slots on these lanes")
    pick = rng.choice(len(slots), size=n, replace=False)
    for p in sorted(pick.tolist()):
        x, y, h = slots[p]
        yaw0 = h + rng.uniform(-0.05, 0.05)
        v = rng.uniform(*speed)
        w = rng.uniform(*yaw_rate)
        x1 = x + v * math.cos(yaw0) * dt
        y1 = y + v * math.sin(yaw0) * dt
        out.append((_pose(x, y, ground_z, yaw0), _pose(x1, y1, ground_z, yaw0 + w * dt)))
    return out
