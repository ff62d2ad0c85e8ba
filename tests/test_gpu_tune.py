"""GPU: the autotuner picks launch parameters per graph-size class without
changing any result, and its table survives a save / load round trip."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402

BLOCKS = {256, 512, 1024}


@pytest.fixture(autouse=True)
def _clean_table():
    dsg.set_tuning()
    dsg.tune_clear()
    yield
    dsg.tune_clear()
    dsg.set_tuning()


def test_autotune_keeps_results_and_round_trips(tmp_path):
    raw = inputs.union(inputs.chung_lu(1 << 15, 1 << 19, 2.1, 32.0, 20000.0, 5), inputs.block(1 << 15, 150, 0.4, 5))
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, 1, 10)
    want_core = oracle.kcore_bz(c)
    g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    try:
        trials = g.autotune(1, 10)
        assert trials >= 2 + 2 * 3
        assert dsg.tune_entries() == 2
        tp, tk = g.tuning("peel"), g.tuning("kcore")
        assert tp["block"] in BLOCKS and tk["block"] in BLOCKS
        for p, q in [(1, 10), (1, 1), (0, 1)]:
            w = oracle.bahmani(c, p, q)
            mask, E, V = g.bahmani(p, q)
            assert (E, V) == (w.E, w.V)
            np.testing.assert_array_equal(mask, w.mask)
        tr = g.bahmani_trace(1, 10)
        assert tr.rounds == want.rounds
        np.testing.assert_array_equal(tr.peel_round, want.peel_round)
        np.testing.assert_array_equal(g.kcore(), want_core)

        path = str(tmp_path / "tune.json")
        dsg.tune_save(path)
        dsg.tune_clear()
        assert dsg.tune_entries() == 0
        assert dsg.tune_load(path) == 2
        assert g.tuning("peel") == tp and g.tuning("kcore") == tk
        np.testing.assert_array_equal(g.kcore(), want_core)
    finally:
        g.close()


def test_tuned_class_does_not_leak_to_other_sizes():
    small = inputs.er_block(2000, 8000, 40, 0.5, 3)
    big = inputs.er_block(40000, 200000, 100, 0.5, 3)
    gs = dsg.Graph.from_edges(small.n, small.src, small.dst)
    gb = dsg.Graph.from_edges(big.n, big.src, big.dst)
    try:
        dsg.set_tuning(block=256, chunk_len=512)
        before = gs.tuning("peel")
        gb.autotune(1, 10, kcore=False)
        assert dsg.tune_entries() == 1
        assert gs.tuning("peel") == before
        assert gs.tuning("kcore")["block"] == 256
        c = oracle.from_raw(small)
        _, E, V = gs.bahmani(1, 10)
        w = oracle.bahmani(c, 1, 10)
        assert (E, V) == (w.E, w.V)
    finally:
        gs.close()
        gb.close()
