"""Span-parallel rays (salf_render_opts.ray_segments): each ray's span in the
voxels' box is cut into K parts walked by K lanes and composited in order
(Eq. 3-4 over consecutive spans), the part in which the ray stops walked
again from the transmittance in front of it.  The outputs must match the
FP64 oracle exactly as whole-ray walks do, for every sensor kind, every K,
and stopping thresholds from never to aggressive (which makes many rays stop
inside a later span)."""

import numpy as np
import pytest

import synth
from tests.parity_util import TOL_C, TOL_D, compare_outputs, gpu_render, oracle_sensitivity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def _sensors():
    return [
        synth.pinhole(61, 45, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
        synth.fisheye(50, 37, 190.0, synth.camera_pose_looking((0.4, 0.8, 1.0), 1.1)),
        synth.panorama(64, 16, synth.camera_pose_looking((0.9, 0.7, 0.95), 0.3)),
        synth.lidar(16, 90, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                    synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1),
        synth.pinhole(33, 29, 60.0, synth.camera_pose_looking((-2.0, 0.2, 1.3), 0.0),
                      synth.camera_pose_looking((-1.6, 0.9, 1.2), 0.5), t0=0.0, t1=0.05,
                      rolling_shutter=True),
    ]


def _edge_rays(sc, seed=3, R=999):
    """Rays starting inside voxels, outside the box, missing it, axis-parallel,
    clipped by t_near / t_far, a ragged count (not a multiple of 32)."""
    rng = np.random.default_rng(seed)
    org = np.array(sc.origin)
    ext = np.array(sc.dims) * sc.s0
    o = org + rng.uniform(-0.5, 1.5, size=(R, 3)) * ext
    d = rng.normal(size=(R, 3))
    d[:50, 1:] = 0.0
    d[50:100, 0] = 0.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tn = np.where(rng.random(R) < 0.3, rng.uniform(0, 1, R), 0.0)
    tf = np.where(rng.random(R) < 0.3, tn + rng.uniform(0.1, 2, R), 0.0)
    tf[100:110] = tn[100:110] + 1e-6  # spans far shorter than a cell
    rays = np.concatenate([o, d, tn[:, None], tf[:, None]], axis=1).astype(np.float32)
    return synth.explicit_rays(rays)


def _check(salf, oracle_lib, sc, sensor, segs, t_min, g=None, osc=None):
    g = g or salf.Scene(sc)
    osc = osc or oracle_lib.OracleScene(sc)
    kw = dict(t_min=t_min, want_intensity=True, background=(0.1, 0.2, 0.3))
    gr = gpu_render(g, sensor, outputs=("rgb", "depth", "opacity", "intensity"),
                    ray_segments=segs, **kw)
    orr = oracle_lib.render(osc, sensor, brute_force=sc.n <= 5000, **kw)
    sens = lambda pos: oracle_sensitivity(oracle_lib, osc, sensor, pos, **kw)
    return compare_outputs(gr, orr, want_intensity=True, t_min=t_min, sensitivity=sens)


@pytest.mark.parametrize("segs", [2, 4, 8])
@pytest.mark.parametrize("t_min", [0.0, 1e-4, 0.05, 0.4])
def test_segments_match_oracle(salf, oracle_lib, segs, t_min):
    sc = synth.random_multilevel_scene(seed=segs, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    g, osc = salf.Scene(sc), oracle_lib.OracleScene(sc)
    for sen in _sensors() + [_edge_rays(sc)]:
        res = _check(salf, oracle_lib, sc, sen, segs, t_min, g, osc)
        assert res["max_c"] <= 1.0, (sen["kind"], res)
    g.check()


def test_segments_dense_scene_stops_inside_spans(salf, oracle_lib):
    """A dense scene (every level-0 cell occupied, a deep octree, densities
    raised e^1.5-fold): most rays stop part-way, often inside a span other
    than the first."""
    sc = synth.random_multilevel_scene(seed=21, max_level=3, dims=(6, 6, 4), p_occ=1.0,
                                       p_sub=0.5, p_child=0.9)
    sc.params[:, 3] += 1.5
    g, osc = salf.Scene(sc), oracle_lib.OracleScene(sc)
    for t_min in (1e-4, 0.02, 0.3):
        op = {}
        for segs in (1, 8):
            sen = synth.lidar(24, 120, synth.lidar_pose((0.5, 0.9, 1.1), 0.1),
                              synth.lidar_pose((0.8, 1.1, 1.1), 0.3), t0=0.0, t1=0.1)
            _check(salf, oracle_lib, sc, sen, segs, t_min, g, osc)
            op[segs] = gpu_render(g, sen, outputs=("opacity",), t_min=t_min, ray_segments=segs)
        # the stopping rule was exercised: many rays end with T below t_min
        assert (op[1]["opacity"] > 1.0 - t_min).mean() > 0.2, t_min


def test_segments_agree_with_whole_rays_driving_lidar(salf):
    """Full 128x2048 LiDAR frame over the 2M-voxel driving scene: every K
    gives the whole-ray outputs up to rounding (termination ties aside)."""
    sc = synth.driving_scene(2_000_000, seed=2)
    g = salf.Scene(sc)
    lid = synth.lidar(128, 2048, synth.lidar_pose((0.0, 0.0, 1.9), 0.0),
                      synth.lidar_pose((1.0, 0.0, 1.9), 0.02), t0=0.0, t1=0.1)
    ref = gpu_render(g, lid, want_intensity=True, ray_segments=1, saved=True,
                     outputs=("rgb", "depth", "opacity", "intensity"))
    for segs in (2, 4, 8):
        got = gpu_render(g, lid, want_intensity=True, ray_segments=segs, saved=True,
                         outputs=("rgb", "depth", "opacity", "intensity"))
        assert np.array_equal(got["valid"], ref["valid"])
        ec = np.maximum(np.abs(got["opacity"] - ref["opacity"]),
                        np.abs(got["intensity"] - ref["intensity"]))
        ed = np.abs(got["depth"] - ref["depth"])
        over = (ec > TOL_C) | (ed > TOL_D)
        # a ray that stops within rounding of t_min may composite one voxel more or less
        assert over.mean() <= 1e-3, (segs, over.sum(), ec.max(), ed.max())
        assert (ec <= 1e-4 + 1e-3).all() and (ed <= TOL_D + 0.1).all(), (segs, ec.max(), ed.max())
        same_count = got["saved"][:, 7] == ref["saved"][:, 7]
        assert same_count.mean() >= 0.999, (segs, same_count.mean())
    g.check()


def test_segment_options(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=5, max_level=1, dims=(4, 4, 3), p_occ=0.6)
    g = salf.Scene(sc)
    lid = synth.lidar(16, 64, synth.lidar_pose((0.3, 0.5, 0.9), 0.0),
                      synth.lidar_pose((0.3, 0.5, 0.9), 0.0))
    for bad in (3, 5, 16, -1):
        with pytest.raises(salf.SalfError) as e:
            g.render(lid, ray_segments=bad)
        assert e.value.status == 1
    # debug outputs walk whole rays whatever the option says
    a = gpu_render(g, lid, ray_segments=8, visits_cap=64, t_min=0.0, outputs=("opacity",))
    b = gpu_render(g, lid, ray_segments=1, visits_cap=64, t_min=0.0, outputs=("opacity",))
    assert np.array_equal(a["visits"], b["visits"]) and np.array_equal(a["opacity"], b["opacity"])
    c = gpu_render(g, lid, ray_segments=4, steps=True, outputs=("opacity",))
    d = gpu_render(g, lid, ray_segments=1, steps=True, outputs=("opacity",))
    assert np.array_equal(c["steps"], d["steps"])
    # host outputs take the option too
    h = g.render_host(lid, ray_segments=4, outputs=("opacity",))
    e = gpu_render(g, lid, ray_segments=4, outputs=("opacity",))
    assert np.array_equal(h["opacity"].numpy(), e["opacity"])
    g.check()
