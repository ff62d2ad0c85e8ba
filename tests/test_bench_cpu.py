"""Host-side bookkeeping of bench.py on CPU: the algorithmic byte models and
the rule that ties an ncu DRAM-traffic figure to the code it was taken on.
No GPU involved."""
import json

import bench


def test_code_hash_ignores_comments_but_not_code():
    a = b"int x = 1;  // one\n\n// a comment line\nint y = 2;\n"
    b = b"int x = 1;\n// reworded comment\nint y = 2;   \n"
    c = b"int x = 1;\nint y = 3;\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)


def test_traffic_is_dropped_once_the_kernel_code_changes(tmp_path, monkeypatch):
    files = {"kcore.cu": b"__global__ void k() {}  // v1\n", "dsg_kernels.cuh": b"", "dsg_common.cuh": b""}
    sha = bench.kernel_source_sha("kcore_levels", read=lambda f: files[f])
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(
        {"w": {"kcore_levels": {"bytes": 123, "source_sha": sha, "capture": "test"}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda name, read=None: sha)
    assert bench.dram_traffic("w", "kcore_levels") == 123
    assert bench.dram_traffic("w", "peel_rounds") is None
    assert bench.dram_traffic("other", "kcore_levels") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda name, read=None: "0" * 16)
    assert bench.dram_traffic("w", "kcore_levels") is None


def test_kcore_byte_model_counts_each_atomic_read_and_write():
    n, m = 10, 20
    st = {"rem_scanned": 30, "rem_written": 15, "atomics": 50}
    base = bench.kcore_bytes(n, m, st)
    st2 = dict(st, atomics=51)
    assert bench.kcore_bytes(n, m, st2) - base == 8
    st3 = dict(st, rem_written=16)
    assert bench.kcore_bytes(n, m, st3) - base == 4
