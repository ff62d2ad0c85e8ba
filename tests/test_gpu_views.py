"""GPU: views of one graph on separate streams, with capped grids, solve side
by side (peels on one host thread, core numbers on another) and give the same
results as the oracle; a cap never changes a result."""
import threading

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402


@pytest.fixture(autouse=True)
def _default_tuning():
    dsg.set_tuning()
    yield
    dsg.set_tuning()


def test_caps_do_not_change_results():
    raw = inputs.union(inputs.rmat(scale=14, m=1 << 18, seed=31), inputs.block(1 << 14, 100, 0.4, 31))
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, 1, 10)
    want_core = oracle.kcore_bz(c)
    g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    try:
        for cap in (1, 2, 7, 76, 0):
            g.set_max_blocks(cap)
            mask, E, V = g.bahmani(1, 10)
            assert (E, V) == (want.E, want.V), cap
            np.testing.assert_array_equal(mask, want.mask)
            np.testing.assert_array_equal(g.kcore(), want_core)
    finally:
        g.close()


def test_views_solve_side_by_side():
    raw = inputs.union(inputs.chung_lu(1 << 16, 1 << 20, 2.1, 32.0, 20000.0, 33), inputs.block(1 << 16, 150, 0.4, 33))
    c = oracle.from_raw(raw)
    eps = [(1, 1000), (1, 10), (1, 1)]
    want = [oracle.bahmani(c, p, q) for p, q in eps]
    want_core = oracle.kcore_bz(c)
    g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ga, gb = g.view(stream=sa), g.view(stream=sb)
    ga.set_max_blocks(76)
    gb.set_max_blocks(76)
    try:
        for _ in range(3):
            core = {}
            t = threading.Thread(target=lambda: core.setdefault("c", gb.kcore()))
            t.start()
            got = [ga.bahmani(p, q) for p, q in eps]
            t.join()
            np.testing.assert_array_equal(core["c"], want_core)
            for (mask, E, V), w in zip(got, want):
                assert (E, V) == (w.E, w.V)
                np.testing.assert_array_equal(mask, w.mask)
    finally:
        ga.close()
        gb.close()
        g.close()


def test_solve_matches_separate_calls():
    raw = inputs.union(inputs.rmat(scale=15, m=1 << 19, seed=35), inputs.block(1 << 15, 120, 0.4, 35))
    c = oracle.from_raw(raw)
    eps = [(1, 1000), (1, 10), (1, 1), (0, 1)]
    want = [oracle.bahmani(c, p, q) for p, q in eps]
    want_core = oracle.kcore_bz(c)
    g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    try:
        for rep in range(3):
            res, core = g.solve(eps)
            np.testing.assert_array_equal(core, want_core)
            for (mask, E, V), w in zip(res, want):
                assert (E, V) == (w.E, w.V)
                np.testing.assert_array_equal(mask, w.mask)
        # device outputs, and the peels alone
        sets = [torch.empty(raw.n, dtype=torch.uint8, device="cuda") for _ in eps]
        core_d = torch.empty(raw.n, dtype=torch.int32, device="cuda")
        res, _ = g.solve(eps, out_sets=sets, out_core=core_d)
        np.testing.assert_array_equal(core_d.cpu().numpy().view(np.uint32), want_core)
        for s, w in zip(sets, want):
            np.testing.assert_array_equal(s.cpu().numpy(), w.mask)
        res, core = g.solve(eps[:2], want_core=False)
        assert core is None and [(E, V) for _, E, V in res] == [(w.E, w.V) for w in want[:2]]
    finally:
        g.close()
