"""The C-ABI library builds, loads without a GPU and exports every entry
point include/ro.h and include/ro_mc.h declare (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="ro.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ro_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ro_create", "ro_upload_bricks", "ro_update_residency_octree", "ro_render", "ro_read_requests"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_2309_04393_gb300 import build, ro
    build.build()
    lib = ctypes.CDLL(build.SO)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(ro.EXPORTS) == set(declared_functions())


def test_query_sizes_and_validation_without_gpu():
    from paper_2309_04393_gb300 import ro
    d = ro.make_desc((128, 128, 128), (1, 1, 1), 1, 8, 32, 3, (16, 16, 16), 73)
    s = ro.query_sizes(d)
    assert s.n_bricks == 64 + 8 + 1 and s.n_nodes == 585 and s.depth == 3 and s.channel_stride == 1
    assert s.slot_pitch % 256 == 0 and s.slot_pitch >= 34 ** 3
    assert s.total >= s.cache + s.page_table + s.octree
    d16 = ro.make_desc((4096, 4096, 96), (1, 1, 4), 16, 16, 32, 7, (16, 16, 4), 109275)
    s16 = ro.query_sizes(d16)
    assert s16.n_bricks == 16 * 58708 and s16.n_nodes == 1797717 and s16.channel_stride == 16
    bad = ro.make_desc((128, 128, 128), (1, 1, 1), 1, 8, 32, 3, (12, 16, 16), 73)   # leaf not a power of two
    with pytest.raises(ro.RoError):
        ro.query_sizes(bad)
    bad = ro.make_desc((9000, 16, 16), (1, 1, 1), 1, 8, 32, 1, (16, 16, 16), 8)       # > 256 bricks per axis
    with pytest.raises(ro.RoError):
        ro.query_sizes(bad)
    bad = ro.make_desc((64, 64, 64), (1, 1, 1), 16, 8, 32, 17, (16, 16, 16), 8)       # more than 16 levels
    with pytest.raises(ro.RoError):
        ro.query_sizes(bad)


def test_compensator_header_exports_and_host_checks_without_gpu():
    """include/ro_mc.h: every declared entry point exported, and the calls
    that are host arithmetic or argument checks answer without a device."""
    import ctypes
    from paper_2309_04393_gb300 import build, mc
    build.build()
    lib = ctypes.CDLL(build.SO)
    names = declared_functions("ro_mc.h")
    for name in names:
        assert hasattr(lib, name), name
    assert set(mc.EXPORTS) == set(names)
    L = mc._lib()
    size = ctypes.c_uint64()
    assert L.ro_mc_query_bytes(ctypes.byref(mc.McDesc(0)), ctypes.byref(size)) == 1     # RO_ERR_INVALID_ARG
    assert L.ro_mc_query_bytes(None, ctypes.byref(size)) == 1
    assert L.ro_mc_query_bytes(ctypes.byref(mc.McDesc(1)), None) == 1
    per = []
    for n in (1, 2, 3):
        assert L.ro_mc_query_bytes(ctypes.byref(mc.McDesc(n)), ctypes.byref(size)) == 0
        per.append(size.value)
    # a grid adds three 32-channel activations and three 32-channel gradient
    # buffers (bfloat16), the output gradient and the output (binary32, 34^3
    # voxels); each of the eight regions is rounded up to 256 bytes, so the
    # step differs from that by less than 8 x 256
    grid = 6 * mc.VOXELS * 32 * 2 + 2 * mc.VOXELS * 4
    for a, b in ((per[0], per[1]), (per[1], per[2])):
        assert abs((b - a) - grid) < 8 * 256
    assert all(p % 256 == 0 for p in per)
    assert per[0] > 5 * mc.PARAMS * 4
    h = ctypes.c_void_p()
    # a misaligned arena and a too small one are refused before any device call
    assert L.ro_mc_create(ctypes.byref(mc.McDesc(1)), ctypes.c_void_p(16), per[0], None, ctypes.byref(h)) == 1
    assert L.ro_mc_create(ctypes.byref(mc.McDesc(1)), ctypes.c_void_p(1 << 20), per[0] - 256, None,
                          ctypes.byref(h)) == 3                                         # RO_ERR_CAPACITY
    assert h.value is None
    assert L.ro_mc_destroy(None) == 1
    assert L.ro_mc_apply_gradients(None, ctypes.c_void_p(16), ctypes.c_float(1e-3)) == 1
    assert L.ro_mc_get_moments(None, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 1
