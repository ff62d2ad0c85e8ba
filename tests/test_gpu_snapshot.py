"""Snapshot / resume of Algorithm 1 (dsg_peel_*): a peel paused after every
round, written to host memory, freed, and resumed on another handle of the
same graph gives exactly the uninterrupted peel's result and the oracle's:
set, (|E|, |V|), round count and per-round history.  Malformed snapshots are
rejected."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402

GRAPHS = [inputs.er_block(n=3000, m=12000, k=50, p=0.5, seed=8), inputs.rmat(scale=14, m=1 << 18, seed=2),
          inputs.chung_lu(n=1 << 13, m_draws=1 << 17, gamma=2.1, mean=16.0, wmax=3000.0, seed=5), inputs.path(300)]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("pq", [(1, 10), (1, 1000), (0, 1)])
def test_paused_every_round_equals_uninterrupted(gi, pq):
    raw = GRAPHS[gi]
    p, q = pq
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, p, q)
    g1 = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    g2 = dsg.Graph.from_csr(c.n, c.off, c.adj)  # another handle of the same graph
    st = dsg.PeelState.begin(g1, p, q)
    snaps, done, step = 0, False, 0
    while not done:
        snap = st.snapshot()
        st.close()
        st = dsg.PeelState.resume(g2 if step % 2 == 0 else g1, snap)
        r, done = st.advance(1 + step % 3)
        snaps += 1
        step += 1
        assert snaps <= want.rounds + 2
    tr = st.finish()
    assert (tr.rounds, tr.E, tr.V) == (want.rounds, want.E, want.V)
    np.testing.assert_array_equal(tr.hist_S, want.hist_S)
    np.testing.assert_array_equal(tr.hist_E, want.hist_E)
    np.testing.assert_array_equal(tr.mask, want.mask)
    mask, E, V = g1.bahmani(p, q)
    assert (E, V) == (want.E, want.V)
    st.close()
    g1.close()
    g2.close()


def test_snapshot_before_any_round_and_after_the_end():
    raw = GRAPHS[0]
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, 1, 10)
    g = dsg.Graph.from_csr(c.n, c.off, c.adj)
    st = dsg.PeelState.begin(g, 1, 10)
    snap0 = st.snapshot()
    st.advance(0)
    snap_end = st.snapshot()
    st.close()
    for snap in (snap0, snap_end):
        st = dsg.PeelState.resume(g, snap)
        tr = st.finish()
        assert (tr.rounds, tr.E, tr.V) == (want.rounds, want.E, want.V)
        np.testing.assert_array_equal(tr.mask, want.mask)
        st.close()
    g.close()


def test_resume_rejects_malformed_snapshots():
    raw = GRAPHS[0]
    g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    small = inputs.path(500)
    other = dsg.Graph.from_edges(small.n, small.src, small.dst)
    st = dsg.PeelState.begin(g, 1, 10)
    st.advance(2)
    snap = st.snapshot()
    st.close()
    bad_magic = bytearray(snap)
    bad_magic[0] ^= 0xff
    for bad in (bytes(bad_magic), snap[:100], snap[:len(snap) - 4]):
        with pytest.raises(dsg.DsgError) as ei:
            dsg.PeelState.resume(g, bad)
        assert ei.value.status == 1
    with pytest.raises(dsg.DsgError) as ei:
        dsg.PeelState.resume(other, snap)  # a graph of another size
    assert ei.value.status == 1
    g.close()
    other.close()
