"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/lbm.h, the binding carries the same names, and argument
errors are reported before any device work."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import lbm as mod
    mod.library()
    return mod


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lbm_create", "lbm_set_geometry", "lbm_set_fields", "lbm_step", "lbm_get_fields",
                     "lbm_reduce", "lbm_destroy", "lbm_last_error", "lbm_set_stream", "lbm_set_allocator",
                     "lbm_get_state", "lbm_set_state"):
        assert required in names


def test_library_exports_every_declared_symbol(lbm):
    lib = lbm.library()
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_has_same_names(lbm):
    for name in _declared():
        assert callable(getattr(lbm, name, None)), name


def test_create_rejects_bad_arguments(lbm):
    good = dict(tau=(1.0, 1.0), G=-2.2)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_config(0, 4, 4), lbm.make_params([good]))
    assert e.value.status == 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_config(4, 4, 4), lbm.make_params([dict(tau=(0.5, 1.0))]))
    assert e.value.status == 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_config(4, 4, 4, eq_order=2), lbm.make_params([good]))
    assert e.value.status == 1
    for bad in (1, 4, -1):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(lbm.make_config(4, 4, 4, reg_order=bad), lbm.make_params([good]))
        assert e.value.status == 1 and "reg_order" in lbm.lbm_last_error()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_config(4, 4, 4), lbm.make_params([dict(tau=(1.0, 1.0), G=float("nan"))]))
    assert e.value.status == 1
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(lbm.make_config(4, 4, 4), lbm.make_params([dict(tau=(1.0, 1.0), slip=bad)]))
        assert e.value.status == 1


def test_allocator_hook_needs_both(lbm):
    lib = lbm.library()
    assert lib.lbm_set_allocator(lbm._ALLOC_T(lambda n, s: 0), lbm._FREE_T()) == 1
    assert lib.lbm_set_allocator(lbm._ALLOC_T(), lbm._FREE_T()) == 0


def test_structs_match_header(lbm):
    import ctypes
    assert ctypes.sizeof(lbm.lbm_config) == 8 * 4  # 8 ints
    assert ctypes.sizeof(lbm.lbm_instance_params) == 13 * 8


def test_create_rejects_grids_beyond_32_bit_plane_offsets(lbm):
    # 19 planes of 1024 x 1024 x 256 cells overflow the kernels' 32-bit offsets
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_config(1024, 1024, 256), lbm.make_params([dict(tau=(1.0, 1.0), G=-2.2)]))
    assert e.value.status == 1
    assert "cells per instance" in lbm.lbm_last_error()


def test_timing_rejects_null_context(lbm):
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_timing_begin(None, 16)
    assert e.value.status == 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_timing_end(None)
    assert e.value.status == 1


def test_resolved_kernel_null_context(lbm):
    assert lbm.lbm_resolved_kernel(None) == "-1"


def _declared_ws():
    txt = open(os.path.join(ROOT, "include", "ws.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ws_[a-z0-9_]+)\s*\(", txt)))


def test_surrogate_boundary_exported_and_bound(lbm):
    from paper_1711_03254_gb300 import ws
    names = _declared_ws()
    assert "ws_conv3d_fwd" in names and "ws_tc_status" in names
    lib = lbm.library()
    for name in names:
        assert hasattr(lib, name), name
        assert callable(getattr(ws, name, None)), name


def test_surrogate_rejects_bad_arguments_before_launch(lbm):
    # channel counts must be multiples of 16; nothing is launched (no GPU needed)
    from paper_1711_03254_gb300 import ws
    L = ws._lib()
    assert L.ws_conv3d_fwd(None, 16, None, None, None, 16, 0, 1, 1, 1, 1, 16, 16, 3, 0, None) == 1
    p = 1 << 12  # any non-null, 16-byte aligned value: argument checks come first
    assert L.ws_conv3d_fwd(p, 24, p, None, p, 24, 0, 1, 2, 2, 2, 24, 16, 3, 0, None) == 1
    assert L.ws_conv3d_fwd(p, 16, p, None, p, 512, 0, 1, 2, 2, 2, 16, 512, 3, 0, None) == 1


def test_surrogate_forward_kernel_switch(lbm):
    # process-wide choice of the forward kernel; unknown values change nothing
    from paper_1711_03254_gb300 import ws
    L = ws._lib()
    prev = L.ws_conv3d_fwd_algo(2)
    assert prev in (0, 1, 2)
    assert L.ws_conv3d_fwd_algo(5) == -1 and L.ws_conv3d_fwd_algo(-1) == -1
    assert L.ws_conv3d_fwd_algo(4) == 2 and L.ws_conv3d_fwd_algo(3) == 4
    assert L.ws_conv3d_fwd_algo(1) == 3
    assert ws.ws_conv3d_fwd_algo("auto") == "gather"
    with pytest.raises(ValueError):
        ws.ws_conv3d_fwd_algo("fastest")
    L.ws_conv3d_fwd_algo(prev)
    prev = L.ws_conv3d_bwd_weight_algo(2)
    assert L.ws_conv3d_bwd_weight_algo(7) == -1 and L.ws_conv3d_bwd_weight_algo(3) == 2
    assert L.ws_conv3d_bwd_weight_algo(1) == 3
    assert ws.ws_conv3d_bwd_weight_algo("auto") == "gather"
    L.ws_conv3d_bwd_weight_algo(prev)
