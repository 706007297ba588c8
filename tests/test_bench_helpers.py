"""bench.py's host-side helpers (no GPU): the kernel definitions its DRAM-traffic
table is keyed to can be found and hashed in the sources."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_every_profiled_kernel_is_found_and_hashed():
    b = _bench()
    rows = []
    for line in open(os.path.join(ROOT, "profiles", "dram_traffic.md")):
        parts = [p.strip() for p in line.strip().strip("|").split("|")]
        if len(parts) == 4 and parts[0].startswith("k_"):
            rows.append(parts)
    assert rows
    for name, nbytes, src, sha in rows:
        h = b.kernel_source_sha1(os.path.join(ROOT, src), name)
        assert h is not None and len(h) == 40, name
        assert int(nbytes) > 0


def test_kernel_hash_covers_only_its_own_definition(tmp_path):
    b = _bench()
    src = ("template <class T>\n__global__ void k_a(int n) {\n  if (n) { n += 1; }\n}\n\n"
           "__global__ void k_b(int n) { n += 2; }\n")
    p = tmp_path / "x.cu"
    p.write_text(src)
    ha, hb = b.kernel_source_sha1(str(p), "k_a"), b.kernel_source_sha1(str(p), "k_b")
    p.write_text(src.replace("n += 2", "n += 3"))
    assert b.kernel_source_sha1(str(p), "k_a") == ha  # another kernel changed
    assert b.kernel_source_sha1(str(p), "k_b") != hb
    p.write_text(src.replace("template <class T>", "template <class U>"))
    assert b.kernel_source_sha1(str(p), "k_a") != ha  # its template line is part of it
    assert b.kernel_source_sha1(str(p), "k_missing") is None
