"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every function include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]*?\b(dsg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["dsg_graph_from_csr", "dsg_graph_from_edges", "dsg_graph_free", "dsg_bahmani",
                 "dsg_bahmani_trace", "dsg_kcore", "dsg_status_string", "dsg_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2103_00154_gb300 as dsg
    from paper_2103_00154_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # the binding names every declared function too
    assert set(declared_functions()) <= set(dsg._native.declared_symbols())


def test_host_only_calls_without_gpu():
    import paper_2103_00154_gb300 as dsg
    L = dsg.lib()
    assert L.dsg_status_string(0) == b"ok"
    assert L.dsg_status_string(8) == b"output capacity too small"
    assert b"sm_103a" in L.dsg_version()
    # round bound: ceil(log_{1.1} 1000) + 2 = 73 + 2
    assert dsg.round_bound(1000, 1, 10) == 75
    assert dsg.round_bound(1000, 0, 1) == 1001
    assert dsg.round_bound(0, 1, 10) == 1


def test_argument_errors_are_reported_without_gpu():
    import paper_2103_00154_gb300 as dsg
    from paper_2103_00154_gb300 import _native as N
    L = dsg.lib()
    h = ctypes.c_void_p()
    st = L.dsg_graph_from_csr(1 << 31, None, None, 0, None, ctypes.byref(h))
    assert st == N.DSG_EINVAL and b"2^31" in L.dsg_last_error()
    assert L.dsg_bahmani(None, 1, 10, None, None, None) == N.DSG_EINVAL
    assert L.dsg_kcore(None, None) == N.DSG_EINVAL
    with pytest.raises(dsg.DsgError):
        dsg.set_tuning(block=300)


def test_tuning_setters_accept_their_defaults_without_gpu():
    import paper_2103_00154_gb300 as dsg
    dsg.set_tuning()
    t = dsg.get_tuning()
    assert t["block"] == 512 and t["short_max"] == 32 and t["chunk_len"] == 256
    dsg.set_tuning(block=1024, blocks_per_sm=1, short_max=8, chunk_len=64, hot_deg=5, local_max=0, local_work=0)
    assert dsg.get_tuning()["block"] == 1024
    dsg.set_tuning()


def test_tuning_table_file_round_trip_without_gpu(tmp_path):
    import paper_2103_00154_gb300 as dsg
    path = tmp_path / "tune.json"
    path.write_text('{"dsg_tuning": 1, "entries": [\n'
                    '  {"key": "dev/152|peel|20:24", "block": 1024, "blocks_per_sm": 0, "short_max": 16, '
                    '"chunk_len": 128, "hot_deg": 4096, "local_max": 1024, "local_work": 16384, "ms": 1.0},\n'
                    '  {"key": "dev/152|kcore|20:24", "block": 256, "blocks_per_sm": 0, "short_max": 32, '
                    '"chunk_len": 256, "hot_deg": 0, "local_max": 256, "local_work": 4096, "ms": 2.0},\n'
                    '  {"key": "bad", "block": 300, "blocks_per_sm": 0, "short_max": 32, '
                    '"chunk_len": 256, "hot_deg": 0, "local_max": 256, "local_work": 4096, "ms": 2.0}\n]}\n')
    try:
        dsg.tune_clear()
        assert dsg.tune_entries() == 0
        assert dsg.tune_load(str(path)) == 2          # the entry with an invalid block size is dropped
        assert dsg.tune_entries() == 2
        out = tmp_path / "again.json"
        dsg.tune_save(str(out))
        dsg.tune_clear()
        assert dsg.tune_load(str(out)) == 2
        text = out.read_text()
        assert '"block": 1024' in text and '"local_work": 4096' in text and "bad" not in text
        with pytest.raises(RuntimeError):
            dsg.tune_load(str(tmp_path / "missing.json"))
    finally:
        dsg.tune_clear()
