"""The scene build from device-resident voxels (salf_build_scene with
keys_on_device) against the host build: the same renders and visit lists,
the same errors."""

import time

import numpy as np
import pytest

import synth
from tests.parity_util import to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def _device_set(salf, sc):
    return salf.VoxelSet(sc.origin, sc.s0, sc.dims, sc.max_level,
                         torch.from_numpy(np.asarray(sc.level, np.uint8)).cuda(),
                         torch.from_numpy(np.asarray(sc.ijk, np.int32)).cuda(),
                         torch.from_numpy(np.asarray(sc.params, np.float32)).cuda(), sc.mode)


def _same_renders(a, b, sensors, cap=128):
    for sen in sensors:
        wi = sen["kind"] == "lidar"
        ra = a.render(sen, want_intensity=wi, visits_cap=cap,
                      outputs=("rgb", "depth", "opacity", "intensity"))
        rb = b.render(sen, want_intensity=wi, visits_cap=cap,
                      outputs=("rgb", "depth", "opacity", "intensity"))
        torch.cuda.synchronize()
        for k in ("rgb", "depth", "opacity", "intensity", "valid", "visits", "visit_count"):
            assert torch.equal(ra[k], rb[k]), (sen["kind"], k)


def _sensors_small():
    return [synth.pinhole(61, 45, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
            synth.fisheye(40, 30, 190.0, synth.camera_pose_looking((0.4, 0.8, 1.0), 1.1)),
            synth.lidar(16, 90, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                        synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1)]


@pytest.mark.parametrize("which", ["tiny", "ml1", "ml2", "ml3", "deep", "sdf", "bf16"])
def test_device_build_renders_like_host_build(salf, which):
    dtype = "bf16" if which == "bf16" else "f32"
    if which == "tiny":
        sc = synth.tiny_scene(seed=1)
        sensors = [synth.pinhole(128, 96, 60.0, np.concatenate([np.eye(3), [[3.2], [3.2], [-8.0]]], 1))]
    elif which == "deep":
        sc = synth.deep_scene(max_level=6, dims=(2, 2, 2), seed=2)
        sensors = [synth.pinhole(48, 40, 70.0, synth.camera_pose_looking((-1.5, 0.7, 1.1), 0.3))]
    else:
        K = {"ml1": 1, "ml2": 2, "ml3": 3}.get(which, 2)
        sc = synth.random_multilevel_scene(seed=K, max_level=K, dims=(6, 5, 4), p_occ=0.6,
                                           mode="sdf" if which == "sdf" else "exp")
        sensors = _sensors_small()
    host = salf.Scene(sc, dtype=dtype)
    dev = salf.Scene(_device_set(salf, sc), dtype=dtype)
    assert dev.info()["n_level0_cells"] == host.info()["n_level0_cells"]
    _same_renders(host, dev, sensors)
    dev.check()


def test_device_build_driving_scene(salf):
    sc = synth.driving_scene(2_000_000, seed=2)
    ds = _device_set(salf, sc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    host = salf.Scene(sc)
    t1 = time.perf_counter()
    dev = salf.Scene(ds, params=ds.params)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    print(f"2M-voxel build: host {1e3 * (t1 - t0):.1f} ms, device {1e3 * (t2 - t1):.1f} ms")
    assert dev.info()["n_level0_cells"] == host.info()["n_level0_cells"]
    _same_renders(host, dev, [
        synth.pinhole(480, 270, 60.0, synth.camera_pose_looking((0.0, 0.0, 1.7), 0.0)),
        synth.lidar(32, 512, synth.lidar_pose((0.0, 0.0, 1.9), 0.0),
                    synth.lidar_pose((1.0, 0.0, 1.9), 0.02), t0=0.0, t1=0.1)], cap=256)


def test_device_build_errors_and_empty(salf):
    empty = synth.single_voxel_scene(np.zeros((0, 32)), dims=(3, 2, 2), cells=np.zeros((0, 3)),
                                     levels=())
    g = salf.Scene(_device_set(salf, empty))
    out = g.render(synth.pinhole(17, 9, 60.0, synth.camera_pose_looking((-1, 1, 1), 0.0)))
    assert float(out["opacity"].abs().max()) == 0.0
    rec = np.zeros((2, 32), np.float32)
    # duplicate voxel -> overlap
    dup = synth.single_voxel_scene(rec, dims=(2, 2, 2), cells=[(1, 0, 1), (1, 0, 1)], levels=[0, 0])
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(_device_set(salf, dup))
    assert e.value.status == 4
    # ancestor and descendant -> overlap
    anc = synth.single_voxel_scene(rec, dims=(2, 2, 2), cells=[(1, 1, 0), (3, 2, 1)], levels=[0, 1],
                                   max_level=1)
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(_device_set(salf, anc))
    assert e.value.status == 4
    # outside the grid, level above max_level
    for cells, levels in (([(0, 0, 0), (2, 0, 0)], [0, 0]), ([(0, 0, 0), (1, 1, 1)], [0, 1])):
        bad = synth.single_voxel_scene(rec, dims=(2, 2, 2), cells=cells, levels=levels)
        with pytest.raises(salf.SalfError) as e:
            salf.Scene(_device_set(salf, bad))
        assert e.value.status == 1
    # SDF records need a, b > 0
    sdf = synth.single_voxel_scene(rec[:1], mode="sdf", dims=(2, 2, 2), cells=[(0, 0, 0)], levels=[0])
    with pytest.raises(salf.SalfError) as e:
        salf.Scene(_device_set(salf, sdf))
    assert e.value.status == 1
