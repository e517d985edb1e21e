"""Seeded sensor descriptors (intrinsics, poses, timing) and ray subsamples.

A descriptor is a plain dict; the CUDA binding and the oracle each marshal it
into their own C struct.  Conventions (both sides implement them):

* world frame z-up;
* camera frame OpenCV (x right, y down, z forward); LiDAR frame x forward,
  y left, z up;
* ``pose0`` / ``pose1``: 3x4 sensor-to-world [R | t] at times ``t0`` / ``t1``.
"""

from __future__ import annotations

import math

import numpy as np

KINDS = {"pinhole": 0, "fisheye": 1, "pano": 2, "lidar": 3, "explicit": 4}


def yaw_matrix(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def camera_pose_looking(position, yaw: float = 0.0) -> np.ndarray:
    """OpenCV camera at ``position`` looking horizontally along heading ``yaw``
    (radians, counter-clockwise from world +x); image 'down' is world -z."""
    f = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.array([0.0, 0.0, -1.0])
    R = np.stack([right, down, f], axis=1)
    return np.concatenate([R, np.asarray(position, float).reshape(3, 1)], axis=1)


def lidar_pose(position, yaw: float = 0.0) -> np.ndarray:
    return np.concatenate([yaw_matrix(yaw), np.asarray(position, float).reshape(3, 1)], axis=1)


def _base(kind, width, height, pose0, pose1=None, t0=0.0, t1=0.0, rolling_shutter=False,
          t_near=0.0, t_far=0.0):
    pose0 = np.asarray(pose0, dtype=np.float64).reshape(3, 4)
    pose1 = pose0.copy() if pose1 is None else np.asarray(pose1, dtype=np.float64).reshape(3, 4)
    return dict(kind=kind, width=int(width), height=int(height), fx=0.0, fy=0.0, cx=0.0,
                cy=0.0, fov=0.0, elev_min=0.0, elev_max=0.0, pose0=pose0, pose1=pose1,
                t0=float(t0), t1=float(t1), rolling_shutter=bool(rolling_shutter),
                t_near=float(t_near), t_far=float(t_far), rays=None)


def pinhole(width, height, hfov_deg, pose0, pose1=None, t0=0.0, t1=0.0,
            rolling_shutter=False, t_near=0.0, t_far=0.0):
    """Pinhole with horizontal FOV ``hfov_deg``; fx = fy = (W/2)/tan(hfov/2),
    principal point at the image centre."""
    s = _base("pinhole", width, height, pose0, pose1, t0, t1, rolling_shutter, t_near, t_far)
    f = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    s.update(fx=f, fy=f, cx=width / 2.0, cy=height / 2.0)
    return s


def fisheye(width, height, fov_deg, pose0, pose1=None, t0=0.0, t1=0.0,
            rolling_shutter=False, t_near=0.0, t_far=0.0):
    """Equidistant fisheye (r = f * theta) whose horizontal FOV is ``fov_deg``:
    f = (W/2) / (fov/2); pixels with theta > fov/2 are invalid."""
    s = _base("fisheye", width, height, pose0, pose1, t0, t1, rolling_shutter, t_near, t_far)
    half = math.radians(fov_deg) / 2.0
    f = (width / 2.0) / half
    s.update(fx=f, fy=f, cx=width / 2.0, cy=height / 2.0, fov=2.0 * half)
    return s


def panorama(width, height, pose0, pose1=None, t0=0.0, t1=0.0, rolling_shutter=False,
             t_near=0.0, t_far=0.0):
    """Equirectangular panorama: 360 degrees of azimuth across the width and
    square angular pixels, so the elevation spans +-(180 deg * H / W)."""
    s = _base("pano", width, height, pose0, pose1, t0, t1, rolling_shutter, t_near, t_far)
    e = math.pi * height / width
    s.update(elev_min=-e, elev_max=e)
    return s


def lidar(beams, azimuths, pose0, pose1=None, t0=0.0, t1=0.1, elev_min_deg=-25.0,
          elev_max_deg=15.0, t_near=0.0, t_far=0.0):
    """Spinning LiDAR: ``beams`` rows with elevations linspace(min, max)
    (row 0 = highest), ``azimuths`` columns spanning 360 degrees, one
    timestamp per column between t0 and t1."""
    s = _base("lidar", azimuths, beams, pose0, pose1, t0, t1, True, t_near, t_far)
    s.update(elev_min=math.radians(elev_min_deg), elev_max=math.radians(elev_max_deg))
    return s


def explicit_rays(rays: np.ndarray, dtype=np.float32):
    """Caller-given rays: (R, 8) rows (ox, oy, oz, dx, dy, dz, t_near, t_far);
    t_far <= 0 means unbounded.  float32 (what the renderer takes) or float64
    (accepted by the oracle only)."""
    rays = np.ascontiguousarray(rays, dtype=dtype).reshape(-1, 8)
    s = _base("explicit", rays.shape[0], 1, np.eye(3, 4))
    s["rays"] = rays
    return s


def n_rays(sensor) -> int:
    return int(sensor["width"]) * int(sensor["height"])


def sample_ray_indices(n_total: int, n_sample: int, seed: int) -> np.ndarray:
    """Seeded sorted subsample of ray indices (without replacement)."""
    rng = np.random.default_rng(seed)
    n_sample = min(n_sample, n_total)
    return np.sort(rng.choice(n_total, size=n_sample, replace=False)).astype(np.int64)
