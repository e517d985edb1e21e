"""Adjoint kernel (through the C ABI) vs the oracle's analytic gradient (which
is itself pinned to central finite differences on the CPU), and, on the
training configuration, vs FP64 central differences of the oracle's loss.

The bar, per record scalar j (no global floor):

    |g_gpu - g_oracle| <= 1e-3 |g_oracle| + 1e-6 + K u B_j,   K = 4, u = 2^-24,

where B_j is the oracle's rounding bound for an FP32 evaluation of the same
sum (oracle.backward(..., bound=True)): every contribution's magnitude with
the cancelling sums taken term by term and the hit geometry's FP32
conditioning folded in.  The last term matters where a scalar's exact value
cancels, e.g. the x-slope of a voxel that rays cross face to face along x
(its midpoint sits exactly on the centre plane in FP64, within u t of it in
FP32).  Rays whose visit list or composited count FP32 rounding may change
(oracle.conditioned: the list moves under the visit-list margin; or a
termination test within exp(1e-3) of t_min) get zero output gradient: the
loss is over the well-conditioned rays, chosen by the oracle.
"""

import math

import numpy as np
import pytest

import synth
from tests.parity_util import conditioned_rays

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
K_ROUND = 4.0


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def grad_close(gg, go, bound, rel=1e-3, abs_tol=1e-6, k=K_ROUND):
    """|gpu - oracle| <= rel |oracle| + abs_tol + k u bound, per scalar.
    Returns the worst ratio and how many scalars needed the rounding term."""
    err = np.abs(gg - go)
    base = rel * np.abs(go) + abs_tol
    lim = base + k * U32 * bound
    worst = float((err / lim).max())
    bad = np.argwhere(err > lim)
    msg = ""
    if len(bad):
        v, j = bad[0]
        msg = (f"{len(bad)} scalars out of bound, e.g. voxel {v} slot {j}: gpu {gg[v, j]:.6g} "
               f"oracle {go[v, j]:.6g} bound term {k * U32 * bound[v, j]:.3g}")
    assert len(bad) == 0, msg
    return dict(worst_ratio=worst, n_needing_rounding_term=int((err > base).sum()),
                n_nonzero=int((go != 0).sum()))


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
    idx = np.arange(R) if idx_only is None else np.asarray(idx_only)
    keep = conditioned_rays(oracle_lib, osc, sensor, idx, scene, t_min=t_min)
    mask = np.zeros(R, bool)
    mask[idx[keep]] = True
    for a in (gr, gd, go, gi):
        a[~mask] = 0
    kw = dict(t_min=t_min, background=background, want_intensity=want_intensity)
    out = g.render(sensor, saved=True, outputs=("rgb",), **kw)
    T = lambda a: torch.from_numpy(a).cuda()
    dg = g.backward(sensor, out["saved"], d_rgb=T(gr), d_depth=T(gd), d_opacity=T(go),
                    d_intensity=T(gi), **kw)
    torch.cuda.synchronize()
    g.check()
    f = lambda a: a[idx].astype(np.float64)
    dor, bnd = oracle_lib.backward(osc, sensor, g_rgb=f(gr), g_depth=f(gd), g_opacity=f(go),
                                   g_intensity=f(gi), idx=idx, brute_force=scene.n <= 5000,
                                   bound=True, **kw)
    return dg.cpu().numpy(), dor, bnd, int((~keep).sum())


@pytest.mark.parametrize("mode", ["exp", "sdf"])
def test_backward_matches_oracle(salf, oracle_lib, mode):
    sc = synth.random_multilevel_scene(seed=12, max_level=2, dims=(5, 4, 3), p_occ=0.8, mode=mode)
    sen = synth.pinhole(48, 36, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    dg, do, bnd, n_out = _case(salf, oracle_lib, sc, sen)
    assert np.abs(do).max() > 0 and n_out <= 0.005 * 48 * 36
    print(grad_close(dg, do, bnd), "rays left out", n_out)
    assert np.all(dg[:, 31] == 0)


def test_backward_with_early_termination_and_lidar(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(6, 5, 4), p_occ=0.9)
    sc.params[:, 3] += 2.0
    sen = synth.lidar(16, 64, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                      synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1)
    dg, do, bnd, n_out = _case(salf, oracle_lib, sc, sen, t_min=1e-3)
    assert n_out <= 0.03 * 16 * 64
    print(grad_close(dg, do, bnd), "rays left out", n_out)


def test_backward_bf16(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=5, max_level=1, dims=(5, 4, 3), p_occ=0.8)
    q = torch.from_numpy(sc.params.astype(np.float32)).to(torch.bfloat16).double().numpy()
    sen = synth.pinhole(40, 30, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    dg, do, bnd, _ = _case(salf, oracle_lib, sc, sen, dtype="bf16", oracle_params=q)
    print(grad_close(dg, do, bnd))


def test_autograd_function_linear_loss(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(5, 4, 3), p_occ=0.8)
    sen = synth.pinhole(32, 24, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    osc = oracle_lib.OracleScene(sc)
    keep = conditioned_rays(oracle_lib, osc, sen, None, sc).astype(np.float64)
    g = salf.Scene(sc)
    params = torch.tensor(sc.params, dtype=torch.float32, device="cuda", requires_grad=True)
    rng = np.random.default_rng(1)
    wr = rng.normal(size=(32 * 24, 3)) * keep[:, None]
    wd = rng.normal(size=32 * 24) * 0.1 * keep
    rgb, depth, opac = salf.RenderFn.apply(params, g, sen, 0.0)
    loss = (rgb * torch.from_numpy(wr).float().cuda()).sum() + \
        (depth * torch.from_numpy(wd).float().cuda()).sum()
    loss.backward()
    do, bnd = oracle_lib.backward(osc, sen, g_rgb=wr, g_depth=wd, t_min=0.0, brute_force=True,
                                  bound=True)
    grad_close(params.grad.cpu().numpy(), do, bnd)


def test_scene_params_views(salf):
    """salf_scene_params: the records view is the scene's storage in internal
    order (dev_order maps back to the input); the scene-owned gradient buffer
    receives the same adjoint as a caller buffer."""
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(5, 4, 3), p_occ=0.8)
    sen = synth.pinhole(32, 24, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1))
    g = salf.Scene(sc)
    order = salf.device_view(g.info()["dev_order"], (sc.n,), "<i4").cpu().numpy()
    pv = g.params_view().cpu().numpy()
    assert np.array_equal(pv, sc.params.astype(np.float32)[order])
    out = g.render(sen, saved=True, outputs=("rgb",), t_min=0.0)
    w = torch.from_numpy(np.random.default_rng(2).normal(size=(32 * 24, 3)).astype(np.float32)).cuda()
    mine = g.backward(sen, out["saved"], d_rgb=w, t_min=0.0)
    own = g.grads_view()
    assert float(own.abs().max()) == 0.0  # created zeroed
    g.backward(sen, out["saved"], d_rgb=w, t_min=0.0, d_params="scene")
    g.backward(sen, out["saved"], d_rgb=w, t_min=0.0, d_params="scene")  # accumulates
    torch.cuda.synchronize()
    g.check()
    a, b = own.cpu().numpy(), mine.cpu().numpy()
    assert np.allclose(a, 2 * b, rtol=1e-5, atol=1e-6)


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
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.8 * losses[0], losses


def test_driving_scene_sampled_gradient(salf, oracle_lib):
    """1M-voxel driving scene, BF16 records, 960x640 camera: gradient from a
    sampled subset of rays equals the oracle's for the same rays."""
    sc = synth.driving_scene(1_000_000, seed=4, ground_extent=141.4, n_actors=140)
    q = torch.from_numpy(sc.params.astype(np.float32)).to(torch.bfloat16).double().numpy()
    cam = synth.pinhole(960, 640, 60.0, synth.camera_pose_looking((5.0, 0.0, 1.7), 0.0))
    idx = synth.sample_ray_indices(960 * 640, 8192, 5)
    dg, do, bnd, n_out = _case(salf, oracle_lib, sc, cam, dtype="bf16", t_min=1e-4,
                               want_intensity=False, background=(0, 0, 0), oracle_params=q,
                               idx_only=idx)
    touched = np.abs(do).sum(1) > 0
    assert touched.sum() > 1000
    # the left-out rays: visit lists within the margin of a cell edge or plane
    assert n_out <= 0.02 * len(idx), n_out
    print(grad_close(dg, do, bnd), "rays left out", n_out)


def training_cameras():
    """The 8 training cameras: 960x640, 60 deg, radius 5 m around (0, 0, 1.7),
    yaw k * 45 deg."""
    return [synth.pinhole(960, 640, 60.0, synth.camera_pose_looking(
        (5.0 * math.cos(k * math.pi / 4), 5.0 * math.sin(k * math.pi / 4), 1.7), k * math.pi / 4))
        for k in range(8)]


def test_training_config_finite_differences(salf, oracle_lib):
    """The training configuration: 8 cameras 960x640 around the 1M-voxel scene
    with BF16 records, L = sum over a seeded ray sample S (1,024 rays per
    camera, well-conditioned ones kept) of |rgb - target|^2 with U[0,1]
    targets (seed 4), t_min 1e-4.  For 1,000 voxels visited by S (seed 5) and
    every record scalar Eq. 1-2 use, the GPU adjoint (given the oracle's
    dL/drgb) is compared with FP64 central differences of the oracle's L on
    the dequantised records, each restricted to the rays of S through the
    voxel (no other ray depends on it).  The oracle's analytic gradient is
    checked against the same differences."""
    sc = synth.driving_scene(1_000_000, seed=4, ground_extent=141.4, n_actors=140)
    q = torch.from_numpy(sc.params.astype(np.float32)).to(torch.bfloat16).double().numpy()
    g = salf.Scene(sc, dtype="bf16")
    osc = oracle_lib.OracleScene(sc, params=q)
    cams = training_cameras()
    R = 960 * 640
    t_min = 1e-4
    trng = np.random.default_rng(4)
    targets = [trng.random((R, 3)) for _ in cams]
    cap = 512
    dparams = torch.zeros((sc.n, 32), device="cuda")
    grad_o = np.zeros((sc.n, 32))
    bound = np.zeros((sc.n, 32))
    per_cam = []
    n_left_out = 0
    for k, (cam, tg) in enumerate(zip(cams, targets)):
        idx = synth.sample_ray_indices(R, 1024, 5 + k)
        keep = conditioned_rays(oracle_lib, osc, cam, idx, sc, t_min=t_min)
        n_left_out += int((~keep).sum())
        idx = idx[keep]
        ro = oracle_lib.render(osc, cam, idx=idx, t_min=t_min, visits_cap=cap)
        assert ro["n_visits"].max() <= cap
        d_rgb = 2.0 * (ro["rgb"] - tg[idx])  # dL/drgb of the oracle's render
        full = np.zeros((R, 3), np.float32)
        full[idx] = d_rgb
        out = g.render(cam, saved=True, outputs=("rgb",), t_min=t_min)
        g.backward(cam, out["saved"], d_rgb=torch.from_numpy(full).cuda(), d_params=dparams,
                   t_min=t_min)
        go, bo = oracle_lib.backward(osc, cam, g_rgb=d_rgb, idx=idx, t_min=t_min, bound=True)
        grad_o += go
        bound += bo
        per_cam.append((idx, ro["visits"], tg[idx]))
    torch.cuda.synchronize()
    g.check()
    assert n_left_out <= 0.02 * 8 * 1024, n_left_out
    gg = dparams.cpu().numpy()
    # rays of S through each voxel, per camera
    through: dict = {}
    for k, (idx, vis, _) in enumerate(per_cam):
        for i in range(len(idx)):
            for v in vis[i][vis[i] >= 0]:
                through.setdefault(int(v), {}).setdefault(k, []).append(i)
    visited = np.array(sorted(through))
    picks = np.random.default_rng(5).choice(visited, size=1000, replace=False)
    slots = list(range(25))  # Eq. 1 density and Eq. 2 colour (EXP mode, no intensity)

    def loss(v):
        tot = 0.0
        for k, rows in through[v].items():
            idx, _, tgt = per_cam[k]
            r = oracle_lib.render(osc, cams[k], idx=idx[rows], t_min=t_min)
            tot += float(((r["rgb"] - tgt[rows]) ** 2).sum())
        return tot

    fd = np.zeros((len(picks), 32))
    for n, v in enumerate(picks):
        rec = q[v].copy()
        for j in slots:
            h = 1e-6 * max(1.0, abs(rec[j]))
            p = rec.copy()
            p[j] += h
            osc.set_record(v, p)
            lp = loss(v)
            p[j] = rec[j] - h
            osc.set_record(v, p)
            lm = loss(v)
            fd[n, j] = (lp - lm) / (2 * h)
        osc.set_record(v, rec)
    # the oracle's analytic gradient agrees with its own differences
    oa = grad_o[picks][:, slots]
    assert np.all(np.abs(oa - fd[:, slots]) <= 1e-6 * np.abs(fd[:, slots]) + 1e-7), \
        np.abs(oa - fd[:, slots]).max()
    # the GPU adjoint agrees with the differences within the per-scalar bar
    stats = grad_close(gg[picks][:, slots], fd[:, slots], bound[picks][:, slots])
    assert np.all(gg[picks][:, 25:] == 0)
    print("FD check:", stats, "rays left out", n_left_out, "of", 8 * 1024)


def test_batched_render_split_by_variant_equals_per_sensor_calls(salf):
    """A batch without intensity runs one launch per kernel variant: the static
    pinholes (lean variant), the LiDAR (spans) and the rest (fisheye, explicit
    rays, a rolling-shutter pinhole).  Every sensor's outputs equal its own
    call's bit for bit."""
    sc = synth.random_multilevel_scene(seed=9, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    g = salf.Scene(sc)
    rng = np.random.default_rng(6)
    o = np.array([-2.0, 0.6, 1.0])
    d = rng.normal(size=(200, 3)) * 0.3 + np.array([1.0, 0.0, 0.0])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([np.tile(o, (200, 1)), d, np.zeros((200, 2))], axis=1)
    sensors = [synth.pinhole(64, 48, 70.0, synth.camera_pose_looking((-2.1, 0.5, 1.05), 0.2)),
               synth.fisheye(48, 40, 190.0, synth.camera_pose_looking((-2.0, 0.7, 1.1), 0.3)),
               synth.lidar(16, 128, synth.lidar_pose((0.3, 0.5, 1.0), 0.1),
                           synth.lidar_pose((0.6, 0.6, 1.0), 0.2), t0=0, t1=0.1),
               synth.explicit_rays(rays),
               synth.pinhole(40, 30, 75.0, synth.camera_pose_looking((-2.2, 0.3, 1.2), -0.1)),
               synth.pinhole(40, 30, 75.0, synth.camera_pose_looking((-2.2, 0.3, 1.2), -0.1),
                             synth.camera_pose_looking((-2.1, 0.35, 1.2), -0.05), t0=0.0, t1=0.03,
                             rolling_shutter=True)]
    outs = ("rgb", "depth", "opacity")
    batch = g.render_batch(sensors, outputs=outs, saved=True, t_min=1e-3)
    lone = [g.render(s, outputs=outs, saved=True, t_min=1e-3) for s in sensors]
    torch.cuda.synchronize()
    for b, l, s in zip(batch, lone, sensors):
        for k in outs + ("saved", "valid"):
            assert torch.equal(b[k], l[k]), (s["kind"], k)
    g.check()


def test_batched_render_and_adjoint_equal_per_sensor_calls(salf):
    """salf_render_rays_batch gives each sensor the outputs of its own call bit
    for bit (pinhole, fisheye, LiDAR spans and explicit rays in one batch);
    salf_render_backward_batch gives the sum of the per-sensor adjoints up to
    the order of the atomic sums."""
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    g = salf.Scene(sc, dtype="bf16")
    rng = np.random.default_rng(5)
    o = np.array([-2.0, 0.6, 1.0])
    d = rng.normal(size=(300, 3)) * 0.3 + np.array([1.0, 0.0, 0.0])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([np.tile(o, (300, 1)), d, np.zeros((300, 2))], axis=1)
    sensors = [synth.pinhole(64, 48, 70.0, synth.camera_pose_looking((-2.1, 0.5, 1.05), 0.2)),
               synth.fisheye(48, 40, 190.0, synth.camera_pose_looking((-2.0, 0.7, 1.1), 0.3)),
               synth.lidar(16, 128, synth.lidar_pose((0.3, 0.5, 1.0), 0.1),
                           synth.lidar_pose((0.6, 0.6, 1.0), 0.2), t0=0, t1=0.1),
               synth.explicit_rays(rays),
               synth.pinhole(40, 30, 75.0, synth.camera_pose_looking((-2.2, 0.3, 1.2), -0.1))]
    outs = ("rgb", "depth", "opacity", "intensity")
    kw = dict(t_min=1e-3, want_intensity=True, background=(0.1, 0.2, 0.3))
    batch = g.render_batch(sensors, outputs=outs, saved=True, **kw)
    lone = [g.render(s, outputs=outs, saved=True, **kw) for s in sensors]
    torch.cuda.synchronize()
    for b, l, s in zip(batch, lone, sensors):
        for k in outs + ("saved", "valid"):
            assert torch.equal(b[k], l[k]), (s["kind"], k)
    grads = [torch.from_numpy(rng.normal(size=(s["width"] * s["height"], 3)).astype(np.float32)).cuda()
             for s in sensors]
    gd = [torch.from_numpy(rng.normal(size=s["width"] * s["height"]).astype(np.float32)).cuda()
          for s in sensors]
    one = g.backward_batch(sensors, [b["saved"] for b in batch], d_rgb=grads, d_depth=gd, **kw)
    ref = torch.zeros_like(one)
    for s, b, gr, dd in zip(sensors, batch, grads, gd):
        g.backward(s, b["saved"], d_rgb=gr, d_depth=dd, d_params=ref, **kw)
    torch.cuda.synchronize()
    g.check()
    assert float(ref.abs().max()) > 0
    assert torch.allclose(one, ref, rtol=1e-5, atol=1e-6)


def test_render_batch_fn_matches_render_fn(salf):
    """RenderBatchFn (one launch each way) gives the outputs of RenderFn per
    sensor and the summed gradient."""
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(5, 4, 3), p_occ=0.8)
    g = salf.Scene(sc)
    sensors = [synth.pinhole(32, 24, 70.0, synth.camera_pose_looking((-1.9, 0.25, 0.9), 0.1)),
               synth.pinhole(20, 16, 80.0, synth.camera_pose_looking((-2.0, 0.6, 1.0), -0.2))]
    w = [torch.rand(s["width"] * s["height"], 3, generator=torch.Generator().manual_seed(k)).cuda()
         for k, s in enumerate(sensors)]
    p1 = torch.tensor(sc.params, dtype=torch.float32, device="cuda", requires_grad=True)
    outs = salf.RenderBatchFn.apply(p1, g, sensors, 0.0)
    sum((o * wi).sum() for o, wi in zip(outs[0::3], w)).backward()
    p2 = torch.tensor(sc.params, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = 0.0
    for s, wi, o in zip(sensors, w, outs[0::3]):
        rgb, _, _ = salf.RenderFn.apply(p2, g, s, 0.0)
        assert torch.equal(rgb, o)
        loss = loss + (rgb * wi).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert torch.allclose(p1.grad, p2.grad, rtol=1e-5, atol=1e-6)
