"""Parity on the benchmark configurations' own inputs (the 10^4-vertex
Erdos-Renyi graph with its planted block, exactly as specified), at the
library defaults and at the launch parameters the autotuner picks for it
(the configuration bench.py times).  Every output against the oracle: CSR
bytes, the peel's set, (|E|, |V|), rounds, per-round |S_r| and |E(S_r)|,
failure rounds, core numbers, densest core and Algorithm 2's second phase."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402


@pytest.fixture(autouse=True)
def _default_tuning():
    dsg.set_tuning()
    dsg.tune_clear()
    yield
    dsg.tune_clear()
    dsg.set_tuning()


def _check_all(g, c, p, q):
    off, adj = g.csr()
    np.testing.assert_array_equal(off, c.off)
    np.testing.assert_array_equal(adj, c.adj)
    want = oracle.bahmani(c, p, q)
    got = g.bahmani_trace(p, q)
    assert (got.rounds, got.best_round, got.E, got.V) == (want.rounds, want.best_round, want.E, want.V)
    np.testing.assert_array_equal(got.hist_S, want.hist_S)
    np.testing.assert_array_equal(got.hist_E, want.hist_E)
    np.testing.assert_array_equal(got.peel_round, want.peel_round)
    np.testing.assert_array_equal(got.mask, want.mask)
    mask, E, V = g.bahmani(p, q)
    assert (E, V) == (want.E, want.V)
    np.testing.assert_array_equal(mask, want.mask)
    core = g.kcore()
    want_core = oracle.kcore_bz(c)
    np.testing.assert_array_equal(core, want_core)
    r = g.cbds()
    kstar, Ek, Vk = oracle.densest_core(c, want_core)
    me, mv, nleg, _ = oracle.cbds_phase2(c, want_core, kstar, Ek, Vk)
    assert (r.k_star, r.E_core, r.V_core, r.E, r.V, r.n_legit) == (kstar, Ek, Vk, me, mv, nleg)


@pytest.mark.parametrize("tuned", [False, True], ids=["defaults", "autotuned"])
def test_er_block_config_exact_input(tuned):
    raw = inputs.er_block(n=10_000, m=50_000, k=100, p=0.5, seed=0)
    c = oracle.from_raw(raw)
    src = torch.from_numpy(raw.src.view(np.int32)).cuda()
    dst = torch.from_numpy(raw.dst.view(np.int32)).cuda()
    g = dsg.Graph.from_edges(raw.n, src, dst, stream=torch.cuda.current_stream())
    if tuned:
        g.autotune(1, 10)
    _check_all(g, c, 1, 10)
    g.close()
    # the same graph from host buffers, as the end-to-end leg of the bench feeds it
    g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    _check_all(g, c, 1, 10)
    g.close()
