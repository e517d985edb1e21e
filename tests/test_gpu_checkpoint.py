"""Scene files (salf_scene_save / salf_scene_load): a saved and reloaded scene
is the same scene -- the same records bit for bit and the same outputs -- for
FP32 and BF16 storage, host- and device-built scenes, and records changed
after the build; malformed files are rejected with SALF_ERR_IO."""

import os

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


def _outputs(g, sen):
    out = g.render(sen, outputs=("rgb", "depth", "opacity"), want_intensity=False)
    torch.cuda.synchronize()
    return {k: out[k].cpu().numpy() for k in ("rgb", "depth", "opacity", "valid")}


def _records(g):
    t = g.params_view()
    if t.dtype != torch.float32:  # BF16 records as their 16-bit patterns
        t = t.view(torch.int16)
    return t.cpu().numpy().copy()


def _header(path):
    with open(path, "rb") as f:
        magic = f.read(8)
        version, dtype, mode, max_level = np.frombuffer(f.read(16), "<i4")
        n = int(np.frombuffer(f.read(8), "<i8")[0])
        geo = np.frombuffer(f.read(32), "<f8")
        dims = np.frombuffer(f.read(16), "<i4")[:3]
        level = np.frombuffer(f.read(n), np.uint8)
        ijk = np.frombuffer(f.read(12 * n), "<i4").reshape(n, 3)
        rest = f.read()
    return dict(magic=magic, version=version, dtype=dtype, mode=mode, max_level=max_level, n=n,
                origin=geo[:3], s0=geo[3], dims=dims, level=level, ijk=ijk, records=rest)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("mode", ["exp", "sdf"])
def test_save_load_round_trip(salf, tmp_path, dtype, mode):
    sc = synth.random_multilevel_scene(seed=3, max_level=2, dims=(6, 5, 4), p_occ=0.5, mode=mode)
    g = salf.Scene(sc, dtype=dtype)
    # records changed after the build are the ones saved
    rng = np.random.default_rng(7)
    p2 = sc.params.astype(np.float64).copy()
    p2[:, 4:25] += rng.normal(0.0, 0.05, size=(sc.n, 21))
    g.update_params(torch.from_numpy(p2.astype(np.float32)).cuda())
    path = str(tmp_path / f"scene_{dtype}_{mode}.salf")
    g.save(path)
    h = _header(path)
    assert h["magic"] == b"SALFSCN1" and h["version"] == 1 and h["n"] == sc.n
    assert h["max_level"] == sc.max_level and tuple(h["dims"]) == tuple(sc.dims)
    assert np.array_equal(h["origin"], np.asarray(sc.origin, float)) and h["s0"] == sc.s0
    # keys in input order
    assert np.array_equal(h["level"], sc.level) and np.array_equal(h["ijk"], sc.ijk)
    # records in input order: FP32 bits, or the BF16 rounding of the FP32 records
    want = torch.from_numpy(p2.astype(np.float32))
    if dtype == "f32":
        got = np.frombuffer(h["records"], "<f4").reshape(sc.n, 32)
        assert np.array_equal(got, want.numpy())
    else:
        got = np.frombuffer(h["records"], "<u2").reshape(sc.n, 32)
        ref = want.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        assert np.array_equal(got, ref)
    g2 = salf.Scene.load(path)
    assert g2.n == g.n and g2.dtype == dtype and g2.mode == mode
    assert g2.geometry == g.geometry
    assert np.array_equal(_records(g2), _records(g))
    for sen in (synth.pinhole(48, 36, 75.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)),
                synth.lidar(16, 90, synth.lidar_pose((0.2, 0.9, 1.05), 0.2),
                            synth.lidar_pose((0.8, 1.0, 1.05), 0.45), t0=0.0, t1=0.1)):
        a, b = _outputs(g, sen), _outputs(g2, sen)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    g2.check()


def test_device_built_scene_round_trip(salf, tmp_path):
    sc = synth.random_multilevel_scene(seed=5, max_level=2, dims=(6, 5, 4), p_occ=0.5)
    dev = salf.VoxelSet(sc.origin, sc.s0, sc.dims, sc.max_level,
                        torch.from_numpy(sc.level).cuda(), torch.from_numpy(sc.ijk).cuda(),
                        torch.from_numpy(sc.params.astype(np.float32)).cuda(), sc.mode)
    g = salf.Scene(dev)
    path = str(tmp_path / "dev.salf")
    g.save(path)
    h = _header(path)
    assert np.array_equal(h["level"], sc.level) and np.array_equal(h["ijk"], sc.ijk)
    g2 = salf.Scene.load(path)
    assert np.array_equal(_records(g2), _records(g))
    sen = synth.pinhole(40, 30, 70.0, synth.camera_pose_looking((-2.0, 0.2, 1.31), 0.0))
    a, b = _outputs(g, sen), _outputs(g2, sen)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_malformed_files_are_rejected(salf, tmp_path):
    from paper_2507_18713_gb300 import _lib as L
    sc = synth.random_multilevel_scene(seed=6, max_level=1, dims=(3, 3, 3), p_occ=0.5)
    g = salf.Scene(sc)
    path = str(tmp_path / "ok.salf")
    g.save(path)
    raw = open(path, "rb").read()
    cases = {"missing": None, "truncated": raw[:-5], "longer": raw + b"\0",
             "magic": b"XALFSCN1" + raw[8:], "empty": b""}
    for name, data in cases.items():
        p = str(tmp_path / f"{name}.salf")
        if data is not None:
            open(p, "wb").write(data)
        with pytest.raises(L.SalfError) as ei:
            salf.Scene.load(p)
        assert ei.value.status == L.ERR_IO, name
    with pytest.raises(L.SalfError) as ei:
        g.save(str(tmp_path / "no_such_dir" / "x.salf"))
    assert ei.value.status == L.ERR_IO
    assert os.path.getsize(path) == len(raw)
