"""Host logic of bench.py (CPU): the code digest that keys the recorded DRAM
traffic of the render kernel ignores comments and white space but not code,
and the guard reports the record only for the workload it was taken on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _digest(tmp_path, text):
    import bench
    p = tmp_path / "k.cu"
    p.write_text(text)
    return bench.code_digest([str(p)])


def test_code_digest_ignores_comments_and_white_space_only(tmp_path):
    base = 'int f(int a) { return a + 1; } // add one\nconst char* s = "a // b /* c */";\n'
    d0 = _digest(tmp_path, base)
    assert _digest(tmp_path, "/* header */\n" + base.replace("// add one", "// plus 1")) == d0
    assert _digest(tmp_path, base.replace("return a + 1;", "return  a+1 ;\n")) == d0
    # code, and comment markers inside a string literal, are code
    assert _digest(tmp_path, base.replace("a + 1", "a + 2")) != d0
    assert _digest(tmp_path, base.replace('"a // b /* c */"', '"a b"')) != d0
    assert _digest(tmp_path, base.replace("int f", "long f")) != d0
    # an escaped quote does not end a literal
    q = 'char c = \'\\\'\'; int x; // note\n'
    assert _digest(tmp_path, q) == _digest(tmp_path, q.replace("// note", "// other"))


def test_traffic_record_only_for_its_workload():
    import bench
    with open(os.path.join(ROOT, "profiles", "render_kernel_cells16_traffic.json")) as fh:
        rec = json.load(fh)
    current = bench.code_digest([os.path.join(ROOT, f) for f in rec["source_files"]])

    class Args:
        workload, image, cache_gib, arc, lod_bias, radius, precision, order = \
            "cells16", None, 8.0, 30.0, None, None, "f32", rec.get("order", 0)

    chan = 3.0e9
    want = int(round(float(rec["dram_bytes_per_channel_sample"]) * chan))
    got = bench.recorded_traffic(Args(), chan)
    assert got == (want if current == rec["code_sha256"] else None)
    # the record's own launch scales back to its own bytes
    own = (int(rec["dram_read_bytes"]) + int(rec["dram_write_bytes"])) / float(rec["channel_samples"])
    assert abs(own - float(rec["dram_bytes_per_channel_sample"])) <= 1e-9 * own
    for field, value in (("precision", "f16"), ("image", "960x540"), ("workload", "views64"), ("cache_gib", 1.5)):
        a = Args()
        setattr(a, field, value)
        assert bench.recorded_traffic(a, chan) is None
