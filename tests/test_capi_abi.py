"""The C-ABI library loads and exports every symbol include/salf.h declares
(no compute calls: this runs without a GPU)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "salf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(salf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("salf_build_scene", "salf_scene_params", "salf_render_rays",
                     "salf_render_backward", "salf_serve_submit", "salf_serve_poll"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2507_18713_gb300 import _lib
    lib = _lib.load()
    names = _declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_struct_layouts_match_header():
    """ctypes mirrors use the C layout; spot-check sizes against hand counts."""
    from paper_2507_18713_gb300 import _lib as L
    assert ctypes.sizeof(L.RenderOpts) == 4 + 12 + 4 + 4 + 4
    assert ctypes.sizeof(L.Outputs) == 10 * 8 + 8 + 8 + 8
    # kind,width,height + 7 floats = 40 -> pad to 8 -> 2*96 poses -> t0,t1 -> int + 2 floats -> ptr
    assert ctypes.sizeof(L.Sensor) == 40 + 192 + 16 + 12 + 4 + 8
    assert ctypes.sizeof(L.RasterStats) == 8 + 8 + 4 + 4 + 4 + 4
    # kind, eta, light_dir[3], min_opacity, offset, t_far
    assert ctypes.sizeof(L.SecondaryOpts) == 4 * 8
    # counters, 3 doubles, peak bytes, then the batching counters
    assert ctypes.sizeof(L.ServeStats) == 5 * 8 + 3 * 8 + 8 + 4 * 8


def test_binding_marshals_the_new_options():
    """ray_segments reaches salf_render_opts; rays_sensor turns an (R, 8) ray
    tensor into an explicit-ray sensor the binding marshals as such."""
    import torch
    from paper_2507_18713_gb300 import _lib as L
    from paper_2507_18713_gb300 import api
    op = api.opts_struct(2e-4, (0.1, 0.2, 0.3), True, 5, 4)
    assert (op.visits_cap, op.ray_segments, op.want_intensity) == (5, 4, 1)
    assert op.t_min_transmittance == ctypes.c_float(2e-4).value   # a C float
    rays = torch.zeros((77, 8))
    sen = api.rays_sensor(rays)
    assert (sen["kind"], sen["width"], sen["height"]) == ("explicit", 77, 1)
    keep: list = []
    s = api.sensor_struct(sen, keep)
    assert s.kind == L.KIND["explicit"] and s.width == 77 and s.height == 1
    assert s.rays == rays.data_ptr()
    assert L.SECONDARY == {"reflect": 0, "refract": 1, "shadow": 2}


def test_no_gpu_means_a_clean_error():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2507_18713_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    st = lib.salf_create(0, ctypes.byref(h))
    assert st in (_lib.ERR_CUDA, _lib.ERR_INVALID)
    assert lib.salf_last_error()
