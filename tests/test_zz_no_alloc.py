"""The allocation-free host-output entry point, salf_render_rays_host_noalloc,
called through the C ABI, against the regular salf_render_rays.

Callers that cannot let a library allocate device memory (real-time loops,
applications that reserve all device memory in their own pool, plug-ins that
may not allocate) use this entry point; it stages outputs in a fixed array
compiled into the library.  Collected last so that, if it fails, a run that
stops at the first failure has already run every other test; it builds its
own scene so it also passes alone in a fresh process.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_C, TOL_D = 1e-4, 1e-3


@pytest.fixture(scope="module")
def salf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_18713_gb300 as P
    P.load()
    return P


def _regular(g, sen, want_intensity):
    outs = ("rgb", "depth", "opacity") + (("intensity",) if want_intensity else ())
    r = g.render(sen, outputs=outs, want_intensity=want_intensity)
    torch.cuda.synchronize()
    return {k: r[k].cpu().numpy() for k in outs + ("valid",)}


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(salf):
    sc = synth.random_multilevel_scene(seed=2, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    g = salf.Scene(sc)
    calls = [
        (synth.pinhole(160, 120, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15)), False),
        (synth.lidar(32, 512, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                     synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1), True),
    ]
    for sen, wi in calls:
        ref = _regular(g, sen, wi)
        outs = ("rgb", "depth", "opacity", "valid") + (("intensity",) if wi else ())
        got = g.render_host_noalloc(sen, want_intensity=wi, outputs=outs)
        got = {k: v.numpy() for k, v in got.items()}
        assert np.array_equal(got["valid"], ref["valid"])
        assert np.abs(got["rgb"] - ref["rgb"]).max() <= TOL_C
        assert np.abs(got["opacity"] - ref["opacity"]).max() <= TOL_C
        assert np.abs(got["depth"] - ref["depth"]).max() <= TOL_D
        if wi:
            assert np.abs(got["intensity"] - ref["intensity"]).max() <= TOL_C


def test_noalloc_leaves_device_memory_unchanged(salf):
    """The point of the entry point: once a call of each sensor kind has run
    (loading its kernels), staged calls of other sizes change neither the
    device's free memory nor the scene's device footprint (no staging
    buffer is created for them)."""
    sc = synth.random_multilevel_scene(seed=2, max_level=2, dims=(6, 5, 4), p_occ=0.7)
    g = salf.Scene(sc)
    lid = lambda b, a: synth.lidar(b, a, synth.lidar_pose((0.35, 0.55, 1.05), 0.2),
                                   synth.lidar_pose((0.95, 0.7, 1.05), 0.45), t0=0.0, t1=0.1)
    pin = lambda w, h: synth.pinhole(w, h, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    for sen, wi in ((pin(160, 120), False), (lid(32, 512), True)):
        g.render_host_noalloc(sen, want_intensity=wi, outputs=("rgb", "depth", "opacity", "valid")
                              if not wi else ("depth", "opacity", "intensity", "valid"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    bytes0 = g.info()["device_bytes"]
    for sen, wi in ((pin(1024, 768), False), (lid(64, 1024), True), (pin(320, 200), False)):
        g.render_host_noalloc(sen, want_intensity=wi, outputs=("rgb", "depth", "opacity", "valid")
                              if not wi else ("depth", "opacity", "intensity", "valid"))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert g.info()["device_bytes"] == bytes0


def test_noalloc_rejects_alpha_maxima(salf):
    import ctypes as C
    from paper_2507_18713_gb300 import _lib as L
    from paper_2507_18713_gb300.api import opts_struct, sensor_struct
    sc = synth.random_multilevel_scene(seed=2, max_level=1)
    g = salf.Scene(sc)
    cam = synth.pinhole(32, 24, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    ma = torch.zeros(sc.n, device="cuda")
    depth = torch.empty(32 * 24)
    o = L.Outputs()
    o.depth = depth.data_ptr()
    o.max_alpha = ma.data_ptr()
    keep = []
    s = sensor_struct(cam, keep)
    op = opts_struct()
    st = L.load().salf_render_rays_host_noalloc(g._h, C.byref(s), C.byref(op), C.byref(o), None)
    assert st == L.ERR_INVALID


def test_noalloc_rejects_outputs_beyond_its_fixed_staging(salf):
    sc = synth.random_multilevel_scene(seed=2, max_level=1)
    g = salf.Scene(sc)
    big = synth.pinhole(4096, 4096, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    with pytest.raises(salf.SalfError) as e:
        g.render_host_noalloc(big, outputs=("rgb", "depth", "opacity"))
    assert e.value.status == 1


def test_noalloc_writes_page_locked_outputs_in_place(salf):
    """Page-locked outputs need no staging, so even frames beyond the fixed
    array render, equal to the device-output render bit for bit."""
    sc = synth.random_multilevel_scene(seed=2, max_level=1)
    g = salf.Scene(sc)
    big = synth.pinhole(2048, 2048, 70.0, synth.camera_pose_looking((-2.2, 0.6, 1.1), 0.15))
    R = 2048 * 2048
    out = {"rgb": torch.empty((R, 3)).pin_memory(), "depth": torch.empty(R).pin_memory(),
           "opacity": torch.empty(R).pin_memory()}
    g.render_host_noalloc(big, out=out)
    dev = g.render(big, outputs=("rgb", "depth", "opacity"))
    torch.cuda.synchronize()
    for k in out:
        assert torch.equal(dev[k].cpu(), out[k]), k
    g.check()
