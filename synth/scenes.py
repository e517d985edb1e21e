"""Seeded sparse-voxel scenes.

A scene is a set of axis-aligned cubic voxels on a multi-level grid: the root
volume is a regular grid of ``dims`` cells of edge ``s0`` (level 0) and a cell
of level l has edge ``s0 / 2**l`` (SaLF Sec. III-A: recursive 8-way
subdivision up to K levels, only non-empty voxels stored).  A voxel is given
by its level and its integer cell coordinates ``ijk`` at that level.

Every voxel carries a 32-scalar parameter record (layout below).  The values
are drawn here; how they are *used* (Eq. 1-6) lives in the oracle and in the
CUDA kernels, never in this module.

Record layout (index: meaning)::

    0:4    W_sigma (Eq. 1) or W_s (Eq. 5): 3 slopes then the bias
    4:13   W_c (Eq. 2), row-major, rows r, g, b; columns x, y, z
    13:25  W_sh (Eq. 2), row-major, rows r, g, b; 4 SH coefficients each
    25     a  (Eq. 6)
    26     b  (Eq. 6)
    27:31  W_int: intensity field, 3 slopes then the bias
    31     padding (0)
"""

from __future__ import annotations

import dataclasses

import numpy as np

RECORD_SCALARS = 32


@dataclasses.dataclass
class SceneData:
    origin: tuple          # world position of the root grid's min corner (m)
    s0: float              # level-0 voxel edge (m)
    dims: tuple            # level-0 grid dimensions (cells)
    max_level: int         # K: deepest subdivision level present in the key space
    level: np.ndarray      # (n,) uint8
    ijk: np.ndarray        # (n, 3) int32, cell coordinates at the voxel's level
    params: np.ndarray     # (n, 32) float32 or float64
    mode: str = "exp"      # "exp" (Eq. 1) or "sdf" (Eq. 5-6)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.level.shape[0])

    def with_params(self, params: np.ndarray) -> "SceneData":
        return dataclasses.replace(self, params=params)


def draw_params(rng: np.random.Generator, n: int, mode: str = "exp",
                dtype=np.float32) -> np.ndarray:
    """Draw n parameter records.

    Geometry, EXP: slopes ~ N(0, 0.25^2), bias ~ N(0, 1), so the density at a
    voxel centre is log-normal(0, 1).  Geometry, SDF: slopes and bias ~
    N(0, 0.5^2).  Colour: W_c ~ N(0, 0.1^2); the constant SH coefficient of
    each channel ~ U[-12, 12] (spreads the colours over most of (0, 1)); the
    other SH coefficients ~ N(0, 0.1^2).  a ~ log-normal(0, 1),
    b ~ U[0.05, 0.5].  Intensity: slopes ~ N(0, 0.1^2), bias ~ U[-4, 4].
    """
    p = np.zeros((n, RECORD_SCALARS), dtype=np.float64)
    if mode == "exp":
        p[:, 0:3] = rng.normal(0.0, 0.25, size=(n, 3))
        p[:, 3] = rng.normal(0.0, 1.0, size=n)
    elif mode == "sdf":
        p[:, 0:4] = rng.normal(0.0, 0.5, size=(n, 4))
    else:
        raise ValueError(mode)
    p[:, 4:13] = rng.normal(0.0, 0.1, size=(n, 9))
    sh = rng.normal(0.0, 0.1, size=(n, 3, 4))
    sh[:, :, 0] = rng.uniform(-12.0, 12.0, size=(n, 3))
    p[:, 13:25] = sh.reshape(n, 12)
    p[:, 25] = np.exp(rng.normal(0.0, 1.0, size=n))
    p[:, 26] = rng.uniform(0.05, 0.5, size=n)
    p[:, 27:30] = rng.normal(0.0, 0.1, size=(n, 3))
    p[:, 30] = rng.uniform(-4.0, 4.0, size=n)
    return p.astype(dtype)


def tiny_scene(seed: int = 1, mode: str = "exp") -> SceneData:
    """4,096 level-0 voxels at distinct random cells of a 64^3 grid, edge 0.1 m."""
    rng = np.random.default_rng(seed)
    dims = (64, 64, 64)
    lin = rng.choice(64 ** 3, size=4096, replace=False)
    k = lin // (64 * 64)
    j = (lin // 64) % 64
    i = lin % 64
    ijk = np.stack([i, j, k], axis=1).astype(np.int32)
    level = np.zeros(4096, dtype=np.uint8)
    params = draw_params(rng, 4096, mode)
    return SceneData((0.0, 0.0, 0.0), 0.1, dims, 0, level, ijk, params, mode,
                     "tiny-4096")


def single_voxel_scene(params: np.ndarray, mode: str = "exp", s0: float = 1.0,
                       dims=(1, 1, 1), cells=((0, 0, 0),), levels=(0,),
                       max_level: int = 0, origin=(0.0, 0.0, 0.0)) -> SceneData:
    """A hand-built scene (used for closed-form checks)."""
    params = np.atleast_2d(np.asarray(params, dtype=np.float64))
    ijk = np.asarray(cells, dtype=np.int32).reshape(-1, 3)
    level = np.asarray(levels, dtype=np.uint8)
    return SceneData(tuple(origin), float(s0), tuple(dims), int(max_level), level,
                     ijk, params, mode, "hand")


def random_multilevel_scene(dims=(6, 5, 4), max_level: int = 2, p_occ: float = 0.45,
                            p_sub: float = 0.35, p_child: float = 0.6, seed: int = 0,
                            s0: float = 0.5, origin=(-1.0, -0.5, 0.25),
                            mode: str = "exp") -> SceneData:
    """Random non-overlapping multi-level voxel set.

    Each level-0 cell is occupied with probability p_occ; an occupied cell at
    level l < K is subdivided with probability p_sub, and then each of its 8
    children is kept (recursively) with probability p_child.  The result is
    disjoint by construction (Sec. III-D).
    """
    rng = np.random.default_rng(seed)
    levels, cells = [], []

    def visit(l, c):
        if l < max_level and rng.random() < p_sub:
            for o in range(8):
                if rng.random() < p_child:
                    ch = (2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + (o >> 2))
                    visit(l + 1, ch)
        else:
            levels.append(l)
            cells.append(c)

    for k in range(dims[2]):
        for j in range(dims[1]):
            for i in range(dims[0]):
                if rng.random() < p_occ:
                    visit(0, (i, j, k))
    n = len(levels)
    params = draw_params(rng, n, mode, dtype=np.float64)
    return SceneData(tuple(origin), float(s0), tuple(dims), int(max_level),
                     np.asarray(levels, dtype=np.uint8),
                     np.asarray(cells, dtype=np.int32).reshape(-1, 3), params, mode,
                     f"multilevel-{seed}")


def deep_scene(max_level: int = 10, dims=(2, 2, 2), seed: int = 0, s0: float = 1.0,
               origin=(0.0, 0.0, 0.0), p_sibling: float = 0.7, mode: str = "exp") -> SceneData:
    """Voxels at every level down to max_level: in each level-0 cell one
    random child is subdivided again at every level (a "spine") and each of
    its 7 siblings is kept as a voxel with probability p_sibling."""
    rng = np.random.default_rng(seed)
    levels, cells = [], []
    for k in range(dims[2]):
        for j in range(dims[1]):
            for i in range(dims[0]):
                c = (i, j, k)
                for l in range(max_level):
                    go = int(rng.integers(8))
                    for o in range(8):
                        ch = (2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + (o >> 2))
                        if o == go:
                            nxt = ch
                        elif rng.random() < p_sibling:
                            levels.append(l + 1)
                            cells.append(ch)
                    c = nxt
                levels.append(max_level)
                cells.append(c)
    n = len(levels)
    params = draw_params(rng, n, mode, dtype=np.float64)
    return SceneData(tuple(origin), float(s0), tuple(dims), int(max_level),
                     np.asarray(levels, dtype=np.uint8),
                     np.asarray(cells, dtype=np.int32).reshape(-1, 3), params, mode,
                     f"deep-{max_level}")


def shuffle_scene(scene: SceneData, seed: int) -> tuple[SceneData, np.ndarray]:
    """Same voxel set in a random input order; returns (scene, perm) with
    new[i] = old[perm[i]]."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(scene.n)
    return dataclasses.replace(scene, level=scene.level[perm], ijk=scene.ijk[perm],
                               params=scene.params[perm]), perm


# --------------------------------------------------------------------------
# Driving-scene-shaped voxel sets
# --------------------------------------------------------------------------

def _shell_cells(i0, j0, k0, nx, ny, nz):
    """Integer cells of the one-voxel-thick hollow shell of an nx*ny*nz box."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    on = ((ii == 0) | (ii == nx - 1) | (jj == 0) | (jj == ny - 1) |
          (kk == 0) | (kk == nz - 1))
    return np.stack([ii[on] + i0, jj[on] + j0, kk[on] + k0], axis=1)


def driving_scene(n_total: int = 2_000_000, seed: int = 2, ground_extent: float = 200.0,
                  ground_layers: int = 1, n_actors: int = 300, mode: str = "exp",
                  keep_clear_radius: float = 8.0, road_half_width: float = 4.0,
                  params_dtype=np.float32) -> SceneData:
    """Synthetic driving scene of exactly n_total voxels.

    Root grid 1024 x 1024 x 128 cells of 0.2 m (204.8 x 204.8 x 25.6 m) with
    min corner (-102.4, -102.4, 0); K = 1 (0.1 m voxels exist).

    * ground: ``ground_layers`` layers of level-0 (0.2 m) voxels over a square
      of side ``ground_extent`` centred on the origin;
    * actors: ``n_actors`` car-sized boxes (L ~ U[3.5, 5], W ~ U[1.7, 2.2],
      H ~ U[1.4, 1.9] m, yaw 0 or 90 degrees) standing on the ground, each the
      hollow one-voxel shell of 0.1 m voxels;
    * poles: vertical 0.1 x 0.1 m columns of height U[3, 8] m, added until the
      total is exactly n_total (the last pole is cut).

    Actors and poles avoid a disc of ``keep_clear_radius`` around the origin
    and a road |y| < ``road_half_width`` along x, where the sensors sit.
    """
    rng = np.random.default_rng(seed)
    dims = (1024, 1024, 128)
    s0 = 0.2
    origin = (-102.4, -102.4, 0.0)
    fine = (2048, 2048, 256)

    ng = int(round(ground_extent / s0))
    g0 = 512 - ng // 2
    gi, gj, gk = np.meshgrid(np.arange(g0, g0 + ng), np.arange(g0, g0 + ng),
                             np.arange(ground_layers), indexing="ij")
    ground = np.stack([gi.ravel(), gj.ravel(), gk.ravel()], axis=1).astype(np.int64)
    if ground.shape[0] > n_total:
        ground = ground[:n_total]
    n_rest = n_total - ground.shape[0]
    half = ground_extent / 2.0 - 3.0
    kbase = 2 * ground_layers  # first level-1 layer above the ground

    def key1(c):
        return (c[:, 0] * fine[1] + c[:, 1]) * fine[2] + c[:, 2]

    def clear(x, y):
        return (x * x + y * y < keep_clear_radius ** 2) | (np.abs(y) < road_half_width)

    actors = []
    placed = 0
    while placed < n_actors:
        L = rng.uniform(3.5, 5.0)
        W = rng.uniform(1.7, 2.2)
        H = rng.uniform(1.4, 1.9)
        x, y = rng.uniform(-half, half, size=2)
        yaw90 = rng.random() < 0.5
        if clear(x, y):
            continue
        nx, ny = int(round(L / 0.1)), int(round(W / 0.1))
        if yaw90:
            nx, ny = ny, nx
        nz = int(round(H / 0.1))
        i0 = int(np.floor((x + 102.4) / 0.1)) - nx // 2
        j0 = int(np.floor((y + 102.4) / 0.1)) - ny // 2
        actors.append(_shell_cells(i0, j0, kbase, nx, ny, nz))
        placed += 1
    act = np.concatenate(actors, axis=0) if actors else np.zeros((0, 3), np.int64)
    _, first = np.unique(key1(act), return_index=True)
    act = act[np.sort(first)]
    if act.shape[0] > n_rest:
        act = act[:n_rest]
    taken = set(key1(act).tolist()) if act.shape[0] < 4_000_000 else None

    poles = []
    need = n_rest - act.shape[0]
    while need > 0:
        x, y = rng.uniform(-half, half, size=2)
        h = rng.uniform(3.0, 8.0)
        if clear(x, y):
            continue
        i = int(np.floor((x + 102.4) / 0.1))
        j = int(np.floor((y + 102.4) / 0.1))
        hc = int(round(h / 0.1))
        col = np.stack([np.full(hc, i), np.full(hc, j), kbase + np.arange(hc)], axis=1)
        kc = key1(col).tolist()
        if any(k in taken for k in kc):
            continue
        col = col[:need]
        taken.update(kc[:need])
        poles.append(col)
        need -= col.shape[0]
    pol = np.concatenate(poles, axis=0) if poles else np.zeros((0, 3), np.int64)

    level = np.concatenate([np.zeros(ground.shape[0], np.uint8),
                            np.ones(act.shape[0] + pol.shape[0], np.uint8)])
    ijk = np.concatenate([ground, act, pol], axis=0).astype(np.int32)
    assert ijk.shape[0] == n_total
    params = draw_params(rng, n_total, mode, dtype=params_dtype)
    return SceneData(origin, s0, dims, 1, level, ijk, params, mode,
                     f"driving-{n_total}")
