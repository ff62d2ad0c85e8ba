"""Batched solve (dsg_batch_solve): every graph of the batch gets exactly
what the oracle (and the one-graph entry points) give it alone -- the peel's
(E, V, R, best round, set) at its own eps, and core numbers where asked."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402


def _mixed_graphs():
    rng = np.random.default_rng(77)
    gs = [inputs.empty(0), inputs.empty(1), inputs.empty(9), inputs.complete(12), inputs.star(300), inputs.path(400),
          inputs.disjoint_cliques([7, 7, 4])]
    for i in range(30):
        n = int(rng.integers(2, 4000))
        g = inputs.random_small(n, float(rng.choice([0.001, 0.004, 0.02])), int(rng.integers(1 << 30)))
        gs.append(inputs.union(g, inputs.block(n, max(2, int(np.sqrt(n))), 0.3, int(rng.integers(1 << 30)))))
    gs += [inputs.rmat(scale=s, m=8 << s, seed=s) for s in (9, 12, 14)]
    gs += [inputs.chung_lu(n=1 << 13, m_draws=1 << 17, gamma=2.3, mean=16.0, wmax=0.0, seed=3)]
    gs += [inputs.batch_graph(i, n_lo=1000, n_hi=20000) for i in range(6)]
    return gs


@pytest.mark.parametrize("device_inputs", [False, True])
def test_batch_matches_oracle_per_graph(device_inputs):
    raws = _mixed_graphs()
    csrs = [oracle.from_raw(r) for r in raws]
    rng = np.random.default_rng(5)
    eps = [[(0, 1), (1, 1000), (1, 100), (1, 10), (1, 1)][int(rng.integers(5))] for _ in raws]
    want_core = (rng.random(len(raws)) < 0.6).astype(np.uint8)
    vb, off, adj = dsg.pack_batch([(c.off, c.adj) for c in csrs], device="cuda" if device_inputs else None)
    solver = dsg.BatchSolver(vb, off, adj, eps, want_core)
    N = solver.N
    out_set = np.zeros(max(N, 1), np.uint8)
    core = np.full(max(N, 1), 0xdeadbeef, np.uint32)
    E, V, R, BR = solver.solve(out_set=out_set, core=core)
    vbh = np.asarray(vb.cpu() if device_inputs else vb).view(np.uint64)
    for g, (c, (p, q)) in enumerate(zip(csrs, eps)):
        want = oracle.bahmani(c, p, q)
        assert (int(E[g]), int(V[g]), int(R[g]), int(BR[g])) == (want.E, want.V, want.rounds, want.best_round), g
        lo, hi = int(vbh[g]), int(vbh[g + 1])
        np.testing.assert_array_equal(out_set[lo:hi], want.mask, err_msg=f"graph {g}")
        if want_core[g]:
            np.testing.assert_array_equal(core[lo:hi], oracle.kcore_bz(c), err_msg=f"graph {g}")
        else:
            assert (core[lo:hi] == 0xdeadbeef).all()


def test_batch_equals_solo_calls_and_device_outputs():
    raws = [inputs.batch_graph(i, n_lo=2000, n_hi=60000) for i in range(8)]
    graphs = [dsg.Graph.from_edges(r.n, r.src, r.dst) for r in raws]
    vb, off, adj = dsg.pack_batch(graphs, device="cuda")
    solver = dsg.BatchSolver(vb, off, adj, [(1, 10)])
    N = solver.N
    out_set = torch.zeros(N, dtype=torch.uint8, device="cuda")
    core = torch.zeros(N, dtype=torch.int32, device="cuda")
    E, V, R, BR = solver.solve(out_set=out_set, core=core)
    vbh = vb.cpu().numpy().view(np.uint64)
    for g, gr in enumerate(graphs):
        mask, e, v = gr.bahmani(1, 10)
        assert (int(E[g]), int(V[g])) == (e, v)
        lo, hi = int(vbh[g]), int(vbh[g + 1])
        np.testing.assert_array_equal(out_set[lo:hi].cpu().numpy(), mask)
        np.testing.assert_array_equal(core[lo:hi].cpu().numpy().view(np.uint32), gr.kcore())


def test_batch_rejects_bad_offsets():
    vb = np.array([0, 3, 2], np.uint64)
    off = np.zeros(4, np.uint64)
    with pytest.raises(dsg.DsgError):
        dsg.BatchSolver(vb, off, np.zeros(1, np.uint32), [(1, 10)]).solve()
    with pytest.raises(dsg.DsgError):
        dsg.BatchSolver(np.array([0, 2], np.uint64), np.zeros(3, np.uint64), np.zeros(1, np.uint32),
                        [(1, 0)]).solve()


def test_batch_with_graphs_above_the_block_share():
    # two large graphs (solved first by the grid-wide kernels) among small ones
    raws = [inputs.rmat(scale=17, m=1 << 21, seed=8), inputs.er_block(n=3000, m=9000, k=30, p=0.5, seed=1),
            inputs.chung_lu(n=1 << 17, m_draws=1 << 20, gamma=2.1, mean=16.0, wmax=20000.0, seed=4),
            inputs.path(50), inputs.empty(3)]
    csrs = [oracle.from_raw(r) for r in raws]
    eps = [(1, 10), (1, 1000), (0, 1), (1, 1), (1, 2)]
    vb, off, adj = dsg.pack_batch([(c.off, c.adj) for c in csrs], device="cuda")
    solver = dsg.BatchSolver(vb, off, adj, eps)
    N = solver.N
    out_set = torch.zeros(N, dtype=torch.uint8, device="cuda")
    core = torch.zeros(N, dtype=torch.int32, device="cuda")
    E, V, R, BR = solver.solve(out_set=out_set, core=core)
    vbh = vb.cpu().numpy().view(np.uint64)
    for g, (c, (p, q)) in enumerate(zip(csrs, eps)):
        want = oracle.bahmani(c, p, q)
        assert (int(E[g]), int(V[g]), int(R[g]), int(BR[g])) == (want.E, want.V, want.rounds, want.best_round), g
        lo, hi = int(vbh[g]), int(vbh[g + 1])
        np.testing.assert_array_equal(out_set[lo:hi].cpu().numpy(), want.mask)
        np.testing.assert_array_equal(core[lo:hi].cpu().numpy().view(np.uint32), oracle.kcore_bz(c))


@pytest.mark.parametrize("split", ["auto", "block_per_graph"])
def test_full_size_batch_members_match_the_oracle(split):
    """Members of the 4,096-graph batch workload at their full sizes -- the
    largest of them (n ~ 10^6) and a seeded sample -- solved together, with
    the default split (the largest go to the grid-wide kernels) and with every
    graph in the block-per-graph launch, as in the full batch: mask, (E, V),
    R, best round and core numbers against the oracle."""
    ns = np.array([inputs.batch_n(i) for i in range(4096)])
    rng = np.random.default_rng(2024)
    members = sorted({int(ns.argmax()), int(ns.argmin())} | set(int(x) for x in rng.choice(4096, 4, replace=False)))
    raws = [inputs.batch_graph(i) for i in members]
    csrs = [oracle.from_raw(r) for r in raws]
    vb, off, adj = dsg.pack_batch([(c.off, c.adj) for c in csrs], device="cuda")
    dsg.set_tuning(batch_split=0 if split == "auto" else 0xffffffff)
    try:
        solver = dsg.BatchSolver(vb, off, adj, [(1, 10)], np.ones(len(raws), np.uint8))
        N = solver.N
        out_set = torch.zeros(N, dtype=torch.uint8, device="cuda")
        core = torch.zeros(N, dtype=torch.int32, device="cuda")
        E, V, R, BR = solver.solve(out_set=out_set, core=core)
    finally:
        dsg.set_tuning()
    vbh = vb.cpu().numpy().view(np.uint64)
    for g, c in enumerate(csrs):
        want = oracle.bahmani(c, 1, 10)
        assert (int(E[g]), int(V[g]), int(R[g]), int(BR[g])) == (want.E, want.V, want.rounds, want.best_round), \
            members[g]
        lo, hi = int(vbh[g]), int(vbh[g + 1])
        np.testing.assert_array_equal(out_set[lo:hi].cpu().numpy(), want.mask, err_msg=str(members[g]))
        np.testing.assert_array_equal(core[lo:hi].cpu().numpy().view(np.uint32), oracle.kcore_bz(c),
                                      err_msg=str(members[g]))
