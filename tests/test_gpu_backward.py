"""Adjoint kernel (through the C ABI) vs the oracle's analytic gradient (which
is itself pinned to central finite differences on the CPU)."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def grad_close(gg, go, rel=1e-3, floor=1e-4):
    """|gpu - oracle| <= rel |oracle| + floor * max|oracle| (per scalar)."""
    scale = float(np.abs(go).max())
    err = np.abs(gg - go)
    lim = rel * np.abs(go) + floor * scale
    worst = float((err / np.maximum(lim, 1e-30)).max())
    assert (err <= lim).all(), f"worst ratio {worst}, max err {err.max()}, scale {scale}"
    return worst


def _case(salf, oracle_lib, scene, sensor, dtype="f32", t_min=0.0, want_intensity=True,
          background=(0.2, 0.1, 0.4), seed=0, oracle_params=None, idx_only=None):
    g = salf.Scene(scene, dtype=dtype)
    osc = oracle_lib.OracleScene(scene, params=oracle_params)
    R = sensor["width"] * sensor["height"]
    rng = np.random.default_rng(seed)
    gr = rng.normal(size=(R, 3)).astype(np.float32)
    gd = rng.normal(size=R).astype(np.float32) * 0.1
    go = rng.normal(size=R).astype(np.float32)
    gi = rng.normal(size=R).astype(np.float32)
    if idx_only is not None:
        mask = np.zeros(R, bool)
        mask[idx_only] = True
        gr[~mask] = 0
        gd[~mask] = 0
        go[~mask] = 0
        gi[~mask] = 0
    kw = dict(t_min=t_min, background=background, want_intensity=want_intensity)
    out = g.render(sensor, saved=True, outputs=("rgb",), **kw)
    T = lambda a: torch.from_numpy(a).cuda()
    dg = g.backward(sensor, out["saved"], d_rgb=T(gr), d_depth=T(gd), d_opacity=T(go),
                    d_intensity=T(gi), **kw)
    torch.cuda.synchronize()
    g.check()
    idx = idx_only
    sl = (lambda a: a[idx]) if idx is not None else (lambda a: a)
    dor = oracle_lib.backward(osc, sensor, g_rgb=sl(gr).astype(np.float64),
                              g_depth=sl(gd).astype(np.float64), g_opacity=sl(go).astype(np.float64),
                              g_intensity=sl(gi).astype(np.float64), idx=idx,
                              brute_force=scene.n <= 5000, **kw)
    return dg.cpu().numpy(), dor


@pytest.mark.parametrize("mode", ["exp", "sdf"])
def test_backward_matches_oracle(salf, oracle_lib, mode):
    sc = synth.random_multilevel_scene(seed=12, max_level=2, dims=(5, 4, 3), p_occ=0.8, mode=mode)
    sen = synth.pinhole(48, 36, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    dg, do = _case(salf, oracle_lib, sc, sen)
    assert np.abs(do).max() > 0
    grad_close(dg, do)
    assert np.all(dg[:, 31] == 0)


def test_backward_with_early_termination_and_lidar(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(6, 5, 4), p_occ=0.9)
    sc.params[:, 3] += 2.0
    sen = synth.lidar(16, 64, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                      synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1)
    dg, do = _case(salf, oracle_lib, sc, sen, t_min=1e-3)
    grad_close(dg, do, rel=2e-3, floor=5e-4)


def test_backward_bf16(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=5, max_level=1, dims=(5, 4, 3), p_occ=0.8)
    q = torch.from_numpy(sc.params.astype(np.float32)).to(torch.bfloat16).double().numpy()
    sen = synth.pinhole(40, 30, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    dg, do = _case(salf, oracle_lib, sc, sen, dtype="bf16", oracle_params=q)
    grad_close(dg, do)


def test_autograd_function_linear_loss(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(5, 4, 3), p_occ=0.8)
    sen = synth.pinhole(32, 24, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    g = salf.Scene(sc)
    params = torch.tensor(sc.params, dtype=torch.float32, device="cuda", requires_grad=True)
    rng = np.random.default_rng(1)
    wr = rng.normal(size=(32 * 24, 3))
    wd = rng.normal(size=32 * 24) * 0.1
    rgb, depth, opac = salf.RenderFn.apply(params, g, sen, 0.0)
    loss = (rgb * torch.from_numpy(wr).float().cuda()).sum() + \
        (depth * torch.from_numpy(wd).float().cuda()).sum()
    loss.backward()
    do = oracle_lib.backward(oracle_lib.OracleScene(sc), sen, g_rgb=wr, g_depth=wd, t_min=0.0,
                             brute_force=True)
    grad_close(params.grad.cpu().numpy(), do)


def test_training_step_reduces_mse(salf):
    """A few Adam steps through RenderFn lower an image MSE (adjoint sign and
    scale are usable for optimisation)."""
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(5, 4, 3), p_occ=0.8)
    sen = synth.pinhole(32, 24, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    g = salf.Scene(sc, dtype="bf16")
    target = torch.rand(32 * 24, 3, generator=torch.Generator().manual_seed(4)).cuda()
    params = torch.tensor(sc.params, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([params], lr=0.05)
    losses = []
    for _ in range(25):
        opt.zero_grad()
        rgb, _, _ = salf.RenderFn.apply(params, g, sen, 1e-4)
        loss = ((rgb - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert losses[-1] < 0.8 * losses[0], losses


def test_driving_scene_sampled_gradient(salf, oracle_lib):
    """1M-voxel driving scene, BF16 records, 960x640 camera: gradient from a
    sampled subset of rays equals the oracle's for the same rays."""
    sc = synth.driving_scene(1_000_000, seed=4, ground_extent=141.4, n_actors=140)
    q = torch.from_numpy(sc.params.astype(np.float32)).to(torch.bfloat16).double().numpy()
    cam = synth.pinhole(960, 640, 60.0, synth.camera_pose_looking((5.0, 0.0, 1.7), 0.0))
    idx = synth.sample_ray_indices(960 * 640, 8192, 5)
    dg, do = _case(salf, oracle_lib, sc, cam, dtype="bf16", t_min=1e-4, want_intensity=False,
                   background=(0, 0, 0), oracle_params=q, idx_only=idx)
    touched = np.abs(do).sum(1) > 0
    assert touched.sum() > 1000
    grad_close(dg, do, rel=2e-3, floor=5e-4)
