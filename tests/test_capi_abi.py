"""The C-ABI library loads and exports every symbol include/salf.h declares
(no compute calls: this runs without a GPU)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "salf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(salf_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("salf_build_scene", "salf_render_rays", "salf_render_backward",
                     "salf_serve_submit", "salf_serve_poll"):
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
