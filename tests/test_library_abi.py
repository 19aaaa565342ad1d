"""The C-ABI library builds, loads without a GPU and exports every entry
point include/ro.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ro.h")).read()
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
