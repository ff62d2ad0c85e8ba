"""GPU parity of the peel's thin-tail rounds (lazy candidate lists): on
graphs that peel one thin shell per round for hundreds of rounds, the CUDA
path with lazy rounds on gives the oracle's set, (|E|, |V|), round count,
history and failure rounds, and the same as with lazy rounds off, while
testing fewer vertices; thin and full rounds alternate where shells are
about 1/9 of the vertices, and a paused peel resumes into lazy rounds
again."""
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


def graph(raw):
    return dsg.Graph.from_edges(raw.n, raw.src, raw.dst)


def check_trace(got, want, tag):
    assert got.rounds == want.rounds, tag
    assert got.best_round == want.best_round, tag
    assert (got.E, got.V) == (want.E, want.V), tag
    np.testing.assert_array_equal(got.hist_S, want.hist_S, err_msg=tag)
    np.testing.assert_array_equal(got.hist_E, want.hist_E, err_msg=tag)
    np.testing.assert_array_equal(got.peel_round, want.peel_round, err_msg=tag)
    np.testing.assert_array_equal(got.mask, want.mask, err_msg=tag)


ONIONS = [(1 << 12, 8, 24), (1 << 15, 16, 40), (1 << 17, 24, 60)]


@pytest.mark.parametrize("n,d,core", ONIONS)
@pytest.mark.parametrize("pq", [(1, 1000), (1, 100), (0, 1), (1, 10)])
def test_thin_tail_rounds_match_the_oracle(n, d, core, pq):
    raw = inputs.onion(n, d, core)
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, *pq)
    g = graph(raw)
    got = g.bahmani_trace(*pq)
    check_trace(got, want, f"{raw.name} {pq}")
    dsg.set_tuning(peel_lazy=False)
    full = g.bahmani_trace(*pq)
    check_trace(full, want, f"{raw.name} {pq} lazy off")
    assert full.lazy_rounds == 0
    if pq[0] * 2 * d < pq[1]:
        if d >= 16:
            # a shell of about 1/(d+1) of the vertices per round: most rounds are thin and test
            # only their candidates
            assert got.lazy_rounds > want.rounds // 2, (got.lazy_rounds, want.rounds)
            assert got.tested * 4 < full.tested, (got.tested, full.tested)
        else:
            # shells of about 1/9 of the vertices: thin and full rounds alternate
            assert 0 < got.lazy_rounds < want.rounds, (got.lazy_rounds, want.rounds)


@pytest.mark.parametrize("block", [256, 1024])
def test_thin_tail_rounds_do_not_depend_on_launch_shape(block):
    raw = inputs.onion(1 << 15, 16, 40)
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, 1, 1000)
    dsg.set_tuning(block=block, chunk_len=32, short_max=4)
    check_trace(graph(raw).bahmani_trace(1, 1000), want, f"block {block}")


def test_shells_next_to_denser_parts():
    # an onion next to a denser random block and a clique: the density rises as the
    # shells go and the threshold overtakes the inner shells, which then fail together
    raw = inputs.union(inputs.onion(1 << 14, 12, 30), inputs.block(1 << 12, 200, 0.35, 7),
                       inputs.complete(70))
    c = oracle.from_raw(raw)
    for pq in [(1, 1000), (1, 200), (1, 50)]:
        check_trace(graph(raw).bahmani_trace(*pq), oracle.bahmani(c, *pq), f"mixed {pq}")


def test_paused_peel_resumes_into_lazy_rounds():
    raw = inputs.onion(1 << 15, 16, 40)
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, 1, 1000)
    g = graph(raw)
    st = dsg.PeelState.begin(g, 1, 1000)
    st.advance(7)
    snap = st.snapshot()
    st.close()
    st2 = dsg.PeelState.resume(g, snap)
    st2.advance(13)
    got = st2.finish()
    assert got.rounds == want.rounds
    assert (got.E, got.V) == (want.E, want.V)
    np.testing.assert_array_equal(got.hist_S, want.hist_S)
    np.testing.assert_array_equal(got.hist_E, want.hist_E)
    np.testing.assert_array_equal(got.mask, want.mask)
