"""LiDAR raydrop output (record slot 31 logit, composited like intensity plus
T_end for an escaping ray) and its adjoint on the GPU, against the FP64
oracle: every sensor kind and span count, stopping thresholds, host
outputs, the adjoint, and the entry points that refuse it."""

import numpy as np
import pytest

import synth
from tests.parity_util import TOL_C, to_np
from tests.parity_util import conditioned_rays
from tests.test_gpu_backward import grad_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def _scene(seed=4, dense=0.0):
    sc = synth.random_multilevel_scene(seed=seed, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    rng = np.random.default_rng(seed + 100)
    sc.params[:, 31] = rng.normal(size=sc.n) * 1.5
    sc.params[:, 3] += dense
    return sc


def _sensors():
    return [synth.lidar(16, 90, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                        synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1),
            synth.pinhole(48, 36, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
            synth.fisheye(40, 30, 190.0, synth.camera_pose_looking((0.4, 0.8, 1.0), 1.1))]


def _check(g, osc, sen, t_min, segs, want_intensity=True):
    gr = g.render(sen, outputs=("depth", "opacity", "intensity", "raydrop"), t_min=t_min,
                  want_intensity=want_intensity, ray_segments=segs)
    torch.cuda.synchronize()
    o = __import__("oracle").render(osc, sen, t_min=t_min, want_intensity=want_intensity,
                                    want_raydrop=True)
    e = np.abs(to_np(gr["raydrop"]) - o["raydrop"])
    lim = np.full(len(e), TOL_C)
    if t_min > 0:  # one voxel more or less at a stopping tie moves it by at most ~t_min
        lim[o["term_gap"] <= 1e-3] += 2 * t_min
    assert (e <= lim).all(), (sen["kind"], segs, t_min, float(e.max()))
    assert np.array_equal(to_np(gr["valid"]).astype(bool), o["valid"])
    return float(e.max())


@pytest.mark.parametrize("segs", [1, 4, 8])
def test_raydrop_matches_oracle(salf, oracle_lib, segs):
    for dense in (0.0, 1.5):
        sc = _scene(dense=dense)
        g, osc = salf.Scene(sc), oracle_lib.OracleScene(sc)
        for sen in _sensors():
            for t_min in (0.0, 1e-4, 0.05):
                _check(g, osc, sen, t_min, segs)
        g.check()


def test_raydrop_bf16_and_host_outputs(salf, oracle_lib):
    sc = _scene(seed=6)
    q = torch.from_numpy(sc.params).to(torch.bfloat16).double().numpy()
    g = salf.Scene(sc, dtype="bf16")
    osc = oracle_lib.OracleScene(sc, params=q)
    sen = _sensors()[0]
    _check(g, osc, sen, 1e-4, 0)
    dev = g.render(sen, outputs=("raydrop", "depth"), want_intensity=True)
    host = g.render_host(sen, outputs=("raydrop", "depth"), want_intensity=True)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(dev["raydrop"]), host["raydrop"].numpy())
    # the other outputs do not depend on whether raydrop is asked for
    plain = g.render(sen, outputs=("depth",), want_intensity=True)
    assert torch.equal(plain["depth"], dev["depth"])
    g.check()


@pytest.mark.parametrize("mode", ["exp", "sdf"])
def test_raydrop_adjoint_matches_oracle(salf, oracle_lib, mode):
    sc = synth.random_multilevel_scene(seed=12, max_level=2, dims=(5, 4, 3), p_occ=0.8, mode=mode)
    sc.params[:, 31] = np.random.default_rng(3).normal(size=sc.n)
    g = salf.Scene(sc)
    osc = oracle_lib.OracleScene(sc)
    sen = synth.lidar(12, 48, synth.lidar_pose((0.3, 0.5, 0.9), 0.1),
                      synth.lidar_pose((0.6, 0.6, 0.9), 0.3), t0=0.0, t1=0.1)
    R = 12 * 48
    rng = np.random.default_rng(1)
    keep = conditioned_rays(oracle_lib, osc, sen, None, sc)
    gp = rng.normal(size=R).astype(np.float32) * keep
    gd = (rng.normal(size=R) * 0.1).astype(np.float32) * keep
    kw = dict(t_min=0.0, want_intensity=True)
    out = g.render(sen, saved=True, outputs=("raydrop", "depth"), **kw)
    T = lambda a: torch.from_numpy(a).cuda()
    dg = g.backward(sen, out["saved"], d_depth=T(gd), raydrop=out["raydrop"], d_raydrop=T(gp),
                    **kw)
    torch.cuda.synchronize()
    do, bnd = oracle_lib.backward(osc, sen, g_depth=gd.astype(np.float64),
                                  g_raydrop=gp.astype(np.float64), bound=True, **kw)
    assert np.abs(do[:, 31]).max() > 0
    grad_close(dg.cpu().numpy(), do, bnd)
    g.check()


def test_raydrop_refused_where_unsupported(salf):
    import ctypes as C
    from paper_2507_18713_gb300 import _lib as L
    sc = _scene(seed=2)
    g = salf.Scene(sc)
    cam = synth.pinhole(32, 24, 60.0, synth.camera_pose_looking((-2.0, 0.5, 1.0), 0.1))
    with pytest.raises(salf.SalfError) as e:
        g.render_raster(cam, outputs=("rgb", "raydrop"))
    assert e.value.status == 1
    with pytest.raises(salf.SalfError) as e:
        g.render_actors(cam, [], outputs=("rgb", "raydrop"))
    assert e.value.status == 1
    with pytest.raises(salf.SalfError) as e:
        g.render_host_noalloc(cam, outputs=("depth", "raydrop"))
    assert e.value.status == 1
    out = g.render(cam, saved=True, outputs=("rgb",))
    d = torch.zeros((sc.n, 32), device="cuda")
    gp = torch.ones(32 * 24, device="cuda")
    with pytest.raises(salf.SalfError) as e:
        g.backward(cam, out["saved"], d_raydrop=gp, d_params=d)
    assert e.value.status == 1
    g.check()
