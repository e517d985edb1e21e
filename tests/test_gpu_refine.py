"""Densification and pruning (Sec. III-C) on the GPU vs the oracle: the
per-voxel alpha maxima a render records, the refined voxel list, and renders
of the refined scene."""

import numpy as np
import pytest

import synth
from tests.parity_util import compare_outputs, gpu_render, oracle_sensitivity, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def _inputs(n, seed):
    """Gradients on a 2^-10 grid (their L1 sums are exact in FP32 and FP64)
    and alpha maxima on a 2^-12 grid (none within rounding of 0.001), so that
    both sides take every split / prune decision the same way."""
    rng = np.random.default_rng(seed)
    g = np.round(rng.normal(size=(n, 32)) * rng.uniform(0, 2, size=(n, 1)) * 1024) / 1024
    a = np.floor(rng.uniform(0, 0.01, size=n) * 4096) / 4096
    l1 = np.abs(g[:, 4:13]).sum(axis=1)
    thr = float(np.floor(np.quantile(l1, 0.75) * 1024) + 0.5) / 1024
    return g, a, thr


def test_recorded_alpha_maxima_match_oracle(salf, oracle_lib):
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(6, 5, 4), p_occ=0.6)
    cam = synth.pinhole(64, 48, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    g = salf.Scene(sc)
    ma = torch.zeros(len(sc.level), device="cuda")
    g.render(cam, max_alpha=ma)
    g.render(cam, max_alpha=ma)  # max-accumulated: a second pass changes nothing
    torch.cuda.synchronize()
    ref = np.zeros(len(sc.level))
    oracle_lib.render(oracle_lib.OracleScene(sc), cam, max_alpha=ref)
    got = to_np(ma).astype(np.float64)
    assert (ref > 0).sum() > 50
    err = np.abs(got - ref)
    assert np.percentile(err, 99.5) < 1e-5 and err.max() < 1e-3, err.max()


@pytest.mark.parametrize("seed,K", [(0, 2), (1, 3)])
def test_refined_voxel_list_matches_oracle(salf, oracle_lib, seed, K):
    sc = synth.random_multilevel_scene(seed=seed, max_level=K, dims=(6, 5, 4), p_occ=0.6)
    n = len(sc.level)
    g_np, a_np, thr = _inputs(n, seed)
    gs = salf.Scene(sc)
    params = torch.from_numpy(sc.params.astype(np.float32)).cuda()
    vs, counts = gs.refine(params, torch.from_numpy(g_np.astype(np.float32)).cuda(),
                           torch.from_numpy(a_np.astype(np.float32)).cuda(), thr, 1e-3)
    lv, ij, pr, act = oracle_lib.refine(sc, g_np, a_np, thr, 1e-3)
    assert counts == dict(n_new=len(lv), n_kept=int((act == 0).sum()),
                          n_split=int((act == 1).sum()), n_pruned=int((act == 2).sum()))
    assert counts["n_split"] > 5 and counts["n_pruned"] > 5
    assert np.array_equal(to_np(vs.level), lv) and np.array_equal(to_np(vs.ijk), ij)
    p = to_np(vs.params).astype(np.float64)
    assert np.abs(p - pr).max() <= 1e-5 * max(1.0, np.abs(pr).max())
    # the refined scene builds and renders like the oracle's refined voxel set
    refined = salf.Scene(vs, params=vs.params)
    ref_set = synth.SceneData(sc.origin, sc.s0, sc.dims, sc.max_level, lv, ij, pr.astype(np.float32),
                              sc.mode, "refined")
    osc = oracle_lib.OracleScene(ref_set)
    cam = synth.pinhole(48, 36, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    gr = gpu_render(refined, cam, outputs=("rgb", "depth", "opacity", "intensity"))
    orr = oracle_lib.render(osc, cam)
    compare_outputs(gr, orr, t_min=1e-4,
                    sensitivity=lambda pos: oracle_sensitivity(oracle_lib, osc, cam, pos, t_min=1e-4))
    refined.check()


def test_refine_edge_cases(salf):
    sc = synth.random_multilevel_scene(seed=2, max_level=1, dims=(4, 4, 3), p_occ=0.6)
    n = len(sc.level)
    g = salf.Scene(sc)
    params = torch.from_numpy(sc.params.astype(np.float32)).cuda()
    big = torch.ones((n, 32), device="cuda") * 100.0
    ones = torch.ones(n, device="cuda")
    # nothing to do
    vs, c = g.refine(params, torch.zeros((n, 32), device="cuda"), ones, 1.0, 0.0)
    assert c["n_new"] == n and np.array_equal(to_np(vs.level), sc.level)
    assert np.array_equal(to_np(vs.ijk), sc.ijk)
    assert torch.equal(vs.params, params)
    # everything pruned
    vs, c = g.refine(params, big, ones, 1.0, 2.0)
    assert c["n_new"] == 0 and c["n_pruned"] == n
    # only voxels above the finest level split
    vs, c = g.refine(params, big, ones, 1.0, 0.0)
    coarse = int((sc.level < sc.max_level).sum())
    assert c["n_split"] == coarse and c["n_new"] == n - coarse + 8 * coarse
    # apply without a plan on a fresh scene is refused
    g2 = salf.Scene(sc)
    st = salf.load().salf_scene_refine_apply(g2._h, params.data_ptr(), None, None, None, None)
    assert st == 1  # SALF_ERR_INVALID


@pytest.mark.parametrize("mode", ["exp", "sdf"])
def test_reg_loss_matches_oracle(salf, oracle_lib, mode):
    """L_reg of Eq. 7 and its gradient, GPU vs the oracle's pair sums."""
    sc = synth.random_multilevel_scene(seed=8, max_level=2, dims=(6, 5, 4), p_occ=0.6, mode=mode)
    g = salf.Scene(sc)
    P = np.asarray(sc.params, dtype=np.float32)
    lam = (0.7, 1.3, 0.4)
    loss, grads = g.reg_loss(torch.from_numpy(P).cuda(), *lam)
    torch.cuda.synchronize()
    ref_loss, ref_grad = oracle_lib.reg_loss(sc, P.astype(np.float64), *lam)
    assert len(oracle_lib.face_pairs(sc)) > 200
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss)
    gg = to_np(grads).astype(np.float64)
    assert np.abs(gg - ref_grad).max() <= 1e-4 * max(1.0, np.abs(ref_grad).max())


def test_reg_loss_vanishes_for_global_affine_field(salf):
    sc = synth.random_multilevel_scene(seed=4, max_level=2, dims=(6, 5, 4), p_occ=0.7, mode="sdf")
    rng = np.random.default_rng(3)
    A, c = np.array([0.3, -0.2, 0.5]), 0.1
    P = rng.normal(size=(len(sc.level), 32)).astype(np.float64) * 0.1
    P[:, 25], P[:, 26] = 1.5, 0.3
    for k in range(len(sc.level)):
        e = sc.s0 / (1 << int(sc.level[k]))
        ctr = np.asarray(sc.origin) + (sc.ijk[k] + 0.5) * e
        P[k, :3] = A * (0.5 * e)
        P[k, 3] = A @ ctr + c
    g = salf.Scene(sc)
    loss, _ = g.reg_loss(torch.from_numpy(P.astype(np.float32)).cuda(), 1.0, 1.0, 1.0)
    torch.cuda.synchronize()
    assert abs(float(loss.item())) < 1e-3
