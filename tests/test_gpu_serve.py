"""Serving loop: continuous batching, memory admission, alone-vs-mix equality,
timeouts and host-side fault injection (no GPU fault is ever provoked)."""

import os
import time

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


@pytest.fixture(scope="module")
def scene(salf):
    sc = synth.random_multilevel_scene(seed=1, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    return salf.Scene(sc, dtype="bf16")


def _mix(rng):
    out = []
    for i in range(24):
        k = i % 4
        yaw = rng.uniform(-0.5, 0.5)
        pos = (rng.uniform(-2.5, -1.8), rng.uniform(0.2, 1.0), rng.uniform(0.8, 1.3))
        if k == 0:
            out.append(synth.pinhole(int(rng.integers(20, 90)), int(rng.integers(10, 70)), 70.0,
                                     synth.camera_pose_looking(pos, yaw)))
        elif k == 1:
            out.append(synth.fisheye(64, 48, 190.0, synth.camera_pose_looking(pos, yaw)))
        elif k == 2:
            out.append(synth.lidar(16, 256, synth.lidar_pose((0.3, 0.5, 1.0), yaw),
                                   synth.lidar_pose((0.6, 0.6, 1.0), yaw + 0.1), t0=0, t1=0.1))
        else:
            out.append(synth.panorama(128, 32, synth.camera_pose_looking(pos, yaw)))
    return out


def _lone(scene, sen):
    want_int = sen["kind"] == "lidar"
    out = scene.render(sen, want_intensity=want_int,
                       outputs=("rgb", "depth", "opacity") + (("intensity",) if want_int else ()))
    torch.cuda.synchronize()
    return out


def test_each_result_equals_lone_render(salf, scene):
    rng = np.random.default_rng(0)
    sensors = _mix(rng)
    srv = salf.Server(scene, mem_budget_bytes=64 << 20, n_streams=2)
    tickets = []
    for s in sensors:
        tickets.append(srv.submit(s, want_intensity=s["kind"] == "lidar"))
        time.sleep(0.0005 * rng.random())
    for s, t in zip(sensors, tickets):
        res = srv.fetch(t, timeout_ms=20000)
        assert res is not None
        lone = _lone(scene, s)
        for k in ("depth", "opacity", "valid"):
            assert torch.equal(res[k], lone[k]), (s["kind"], k)
        if s["kind"] != "lidar":
            assert torch.equal(res["rgb"], lone["rgb"]), s["kind"]
        else:
            assert torch.equal(res["intensity"], lone["intensity"])
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == len(sensors) and st["launches"] >= 1
    assert st["requests_launched"] == len(sensors) and st["latency_window"] == len(sensors)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_held_requests_share_launches_and_equal_lone_renders(salf, scene):
    """Requests submitted under a hold start together: requests of one kernel
    class share a launch (two pinholes and explicit rays in one, a fisheye and
    a panorama in another, two LiDARs in a third), so launches carry several
    sensor kinds, and every result equals its lone render bit for bit."""
    rng = np.random.default_rng(3)
    cam = lambda w, h: synth.pinhole(w, h, 70.0, synth.camera_pose_looking((-2.1, 0.5, 1.05), 0.2))
    o = np.array([-2.0, 0.6, 1.0])
    d = rng.normal(size=(500, 3)) * 0.3 + np.array([1.0, 0.0, 0.0])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([np.tile(o, (500, 1)), d, np.zeros((500, 2))], axis=1)
    sensors = [cam(64, 48), synth.fisheye(64, 48, 190.0, synth.camera_pose_looking(
                   (-2.0, 0.7, 1.1), 0.3)),
               synth.lidar(16, 256, synth.lidar_pose((0.3, 0.5, 1.0), 0.1),
                           synth.lidar_pose((0.6, 0.6, 1.0), 0.2), t0=0, t1=0.1),
               synth.explicit_rays(rays), cam(40, 30),
               synth.panorama(128, 32, synth.camera_pose_looking((-1.9, 0.6, 1.0), 0.0)),
               synth.lidar(8, 128, synth.lidar_pose((0.4, 0.5, 1.0), 0.3),
                           synth.lidar_pose((0.5, 0.6, 1.0), 0.3), t0=0, t1=0.1)]
    srv = salf.Server(scene, mem_budget_bytes=64 << 20, n_streams=2)
    srv.hold(True)
    tickets = [srv.submit(s, want_intensity=s["kind"] == "lidar") for s in sensors]
    time.sleep(0.05)
    assert srv.stats()["launches"] == 0   # nothing starts under the hold
    srv.hold(False)
    for s, t in zip(sensors, tickets):
        res = srv.fetch(t, timeout_ms=20000)
        lone = _lone(scene, s)
        keys = ("depth", "opacity", "valid") + (("intensity",) if s["kind"] == "lidar" else ("rgb",))
        for k in keys:
            assert torch.equal(res[k], lone[k]), (s["kind"], k)
        srv.release(t)
    st = srv.stats()
    print(st)
    assert st["launches"] == 3 and st["requests_launched"] == len(sensors)
    assert st["mixed_launches"] == 2 and st["max_batch"] == 3
    srv.close()


def test_admission_by_memory(salf, scene):
    """A budget that fits about two requests: every request still completes,
    in arrival order of admission, and the arena never exceeds the budget."""
    sen = synth.pinhole(128, 96, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.1))
    per = 128 * 96 * (12 + 4 + 4 + 1) + 4 * 256
    budget = int(2.2 * per)
    srv = salf.Server(scene, mem_budget_bytes=budget, n_streams=2)
    ts = [srv.submit(sen) for _ in range(8)]
    done = 0
    for t in ts:
        assert srv.poll(t, timeout_ms=20000) is not None
        srv.release(t)
        done += 1
    st = srv.stats()
    assert done == 8 and st["peak_bytes"] <= budget
    srv.close()


def test_oversize_request_rejected_and_bad_tickets(salf, scene):
    srv = salf.Server(scene, mem_budget_bytes=1 << 16, n_streams=1)
    big = synth.pinhole(512, 512, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.1))
    with pytest.raises(salf.SalfError) as e:
        srv.submit(big)
    assert e.value.status == 1
    with pytest.raises(salf.SalfError) as e:
        srv.release(12345)
    assert e.value.status == 7
    with pytest.raises(salf.SalfError) as e:
        srv.poll(999)
    assert e.value.status == 7
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_poll_timeout_then_completion(salf, scene):
    srv = salf.Server(scene, mem_budget_bytes=256 << 20, n_streams=1)
    sen = synth.pinhole(1024, 768, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.1))
    t = srv.submit(sen)
    first = srv.poll(t, timeout_ms=0)   # usually not done yet; either answer is legal
    res = srv.poll(t, timeout_ms=30000)
    assert res is not None
    assert first is None or first == res
    srv.release(t)
    srv.close()


def test_injected_launch_failure_is_reported_and_isolated(salf, scene, monkeypatch):
    monkeypatch.setenv("SALF_SERVE_FAULT", "launch_fail:1")
    srv = salf.Server(scene, mem_budget_bytes=64 << 20, n_streams=1)
    sen = synth.pinhole(32, 24, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.1))
    t1 = srv.submit(sen)
    with pytest.raises(salf.SalfError) as e:
        srv.poll(t1, timeout_ms=20000)
    assert e.value.status == 3
    srv.release(t1)
    t2 = srv.submit(sen)
    assert srv.poll(t2, timeout_ms=20000) is not None
    srv.release(t2)
    srv.close()


def test_injected_create_oom(salf, scene, monkeypatch):
    monkeypatch.setenv("SALF_SERVE_FAULT", "create_oom")
    with pytest.raises(salf.SalfError) as e:
        salf.Server(scene, mem_budget_bytes=1 << 20)
    assert e.value.status == 2


def test_destroy_with_pending_requests_does_not_hang(salf, scene):
    srv = salf.Server(scene, mem_budget_bytes=1 << 20, n_streams=1)
    sen = synth.pinhole(200, 150, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.1))
    for _ in range(6):
        srv.submit(sen)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30


def test_serving_scene_4m_bf16_parity_and_mix_equality(salf, oracle_lib):
    """The serving configuration at full size: 4,000,000-voxel scene (two ground
    layers, 600 actors), BF16 records.  Sampled outputs of the serving sensor
    kinds match the oracle on the dequantised records; each request's result is
    identical alone and inside a batch."""
    from tests.parity_util import compare_outputs, oracle_sensitivity
    sc = synth.driving_scene(4_000_000, seed=3, ground_layers=2, n_actors=600)
    g = salf.Scene(sc, dtype="bf16")
    q = torch.from_numpy(sc.params).to(torch.bfloat16).double().numpy()
    osc = oracle_lib.OracleScene(sc, params=q)
    sensors = [
        synth.panorama(4096, 1024, synth.camera_pose_looking((0.3, -0.2, 1.7), 0.4)),
        synth.fisheye(1280, 960, 190.0, synth.camera_pose_looking((0.1, 0.2, 1.65), 2.0)),
        synth.lidar(64, 1024, synth.lidar_pose((0.0, 0.1, 1.9), 1.0),
                    synth.lidar_pose((1.0, 0.1, 1.9), 1.02), t0=0.0, t1=0.1),
        synth.pinhole(1920, 1080, 60.0, synth.camera_pose_looking((-0.2, 0.3, 1.72), -1.3)),
    ]
    srv = salf.Server(g, mem_budget_bytes=1 << 30, n_streams=2)
    tickets = [srv.submit(s, want_intensity=s["kind"] == "lidar") for s in sensors]
    for i, (s, t) in enumerate(zip(sensors, tickets)):
        wi = s["kind"] == "lidar"
        res = srv.fetch(t, timeout_ms=60000)
        lone = g.render(s, want_intensity=wi,
                        outputs=("rgb", "depth", "opacity") + (("intensity",) if wi else ()))
        torch.cuda.synchronize()
        for k in ("depth", "opacity", "valid") + (("intensity",) if wi else ("rgb",)):
            assert torch.equal(res[k], lone[k]), (s["kind"], k)
        srv.release(t)
        R = s["width"] * s["height"]
        idx = synth.sample_ray_indices(R, 8192, 40 + i)
        gr = {k: v.cpu().numpy()[idx] for k, v in lone.items() if not k.startswith("_")}
        if "intensity" not in gr:
            gr["intensity"] = np.zeros(len(idx))
        orr = oracle_lib.render(osc, s, idx=idx, want_intensity=wi)
        sens = lambda pos, s=s, idx=idx, wi=wi: oracle_sensitivity(
            oracle_lib, osc, s, idx[pos], t_min=1e-4, want_intensity=wi)
        r = compare_outputs(gr, orr, want_intensity=wi, t_min=1e-4, sensitivity=sens)
        print(s["kind"], r)
    srv.close()
    g.check()
