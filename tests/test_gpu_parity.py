"""GPU parity: every output of the CUDA path through the C ABI equals the CPU
oracle's, bit for bit (nothing here is floating point).

Compared: the canonical CSR of the ingest, the peel's set, (|E|, |V|), round
count, per-round |S_r| and |E(S_r)|, per-vertex failure round, and the core
numbers.  Cases: hand-worked fixtures, closed forms, edge cases (empty,
single vertex, no edges), random graphs with planted blocks spanning many
tiles with ragged tails, hubs whose rows cross the short-row / chunk
boundaries and the ingest's warp / block / merge row classes, all eps of the
test plan, and every launch shape the tuner may pick.
"""
import itertools

import numpy as np
import pytest

import inputs
import oracle
from golden_io import all_fixtures, load

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402

EPS = [(0, 1), (1, 1000), (1, 100), (1, 10), (1, 2), (1, 1), (3, 2)]


@pytest.fixture(autouse=True)
def _default_tuning():
    dsg.set_tuning()
    yield
    dsg.set_tuning()


def gpu_graph(raw):
    return dsg.Graph.from_edges(raw.n, raw.src, raw.dst)


def check_peel(g, c, p, q, tag=""):
    want = oracle.bahmani(c, p, q)
    got = g.bahmani_trace(p, q)
    assert got.rounds == want.rounds, tag
    assert got.best_round == want.best_round, tag
    assert (got.E, got.V) == (want.E, want.V), tag
    np.testing.assert_array_equal(got.hist_S, want.hist_S, err_msg=tag)
    np.testing.assert_array_equal(got.hist_E, want.hist_E, err_msg=tag)
    np.testing.assert_array_equal(got.peel_round, want.peel_round, err_msg=tag)
    np.testing.assert_array_equal(got.mask, want.mask, err_msg=tag)
    mask, E, V = g.bahmani(p, q)
    assert (E, V) == (want.E, want.V), tag
    np.testing.assert_array_equal(mask, want.mask, err_msg=tag)


def check_core(g, c, tag=""):
    np.testing.assert_array_equal(g.kcore(), oracle.kcore_bz(c), err_msg=tag)


def check_csr(g, c, tag=""):
    off, adj = g.csr()
    np.testing.assert_array_equal(off, c.off, err_msg=tag)
    np.testing.assert_array_equal(adj, c.adj, err_msg=tag)


# ----------------------------------------------------------------- fixtures
@pytest.mark.parametrize("name", all_fixtures())
def test_hand_worked(name):
    fx = load(name)
    raw = inputs.from_pairs(fx["n"], fx["pairs"])
    g = gpu_graph(raw)
    got = g.bahmani_trace(fx["p"], fx["q"])
    assert (got.rounds, got.best_round, got.E, got.V) == (fx["rounds"], fx["best_round"], fx["E"], fx["V"])
    np.testing.assert_array_equal(got.hist_S, fx["hist_S"])
    np.testing.assert_array_equal(got.hist_E, fx["hist_E"])
    np.testing.assert_array_equal(got.peel_round, fx["peel_round"])
    np.testing.assert_array_equal(g.kcore(), fx["core"])


# -------------------------------------------------------------- edge cases
@pytest.mark.parametrize("raw", [inputs.empty(0), inputs.empty(1), inputs.empty(7), inputs.complete(1),
                                 inputs.complete(2), inputs.complete(33), inputs.star(1), inputs.star(40),
                                 inputs.path(2), inputs.path(100), inputs.cycle(3), inputs.cycle(64),
                                 inputs.disjoint_cliques([6, 6]), inputs.disjoint_cliques([9, 5, 5]),
                                 inputs.from_pairs(5, [(0, 0), (1, 1), (0, 1), (1, 0), (0, 1)])],
                         ids=lambda r: r.name or "pairs")
def test_edge_cases(raw):
    c = oracle.from_raw(raw)
    g = gpu_graph(raw)
    check_csr(g, c, raw.name)
    for p, q in EPS:
        check_peel(g, c, p, q, f"{raw.name} eps={p}/{q}")
    if raw.n:
        check_core(g, c, raw.name)


def test_empty_graph_outputs():
    g = gpu_graph(inputs.empty(0))
    assert g.n == 0 and g.m == 0
    mask, E, V = g.bahmani(1, 10)
    assert (E, V) == (0, 0)
    tr = g.bahmani_trace(1, 10)
    assert tr.rounds == 0 and list(tr.hist_S) == [0]


# ------------------------------------------------------------ random graphs
def _random_cases():
    rng = np.random.default_rng(2024)
    for i in range(24):
        n = int(rng.integers(2, 3000))
        g = inputs.random_small(n, float(rng.choice([0.001, 0.005, 0.02, 0.08])), int(rng.integers(1 << 30)))
        if i % 2 == 0:
            k = max(2, int(np.sqrt(n)))
            g = inputs.union(g, inputs.block(n, k, 0.5, int(rng.integers(1 << 30))))
        yield g


@pytest.mark.parametrize("pq", EPS)
def test_random_graphs(pq):
    for raw in _random_cases():
        c = oracle.from_raw(raw)
        g = gpu_graph(raw)
        check_peel(g, c, *pq, tag=raw.name)


def test_random_graphs_core_and_csr():
    for raw in _random_cases():
        c = oracle.from_raw(raw)
        g = gpu_graph(raw)
        check_csr(g, c, raw.name)
        check_core(g, c, raw.name)


@pytest.mark.parametrize("scale", [8, 11, 14])
def test_rmat_small(scale):
    raw = inputs.rmat(scale=scale, m=16 << scale, seed=scale)
    c = oracle.from_raw(raw)
    g = gpu_graph(raw)
    check_csr(g, c)
    check_core(g, c)
    for pq in [(1, 1000), (1, 10), (1, 1), (0, 1)]:
        check_peel(g, c, *pq, tag=f"rmat{scale}")


def spread_rows_cases():
    """Graphs whose non-empty rows sit far apart: the edge walker's steps cross
    runs of empty rows of every length (one 32-row window, the 1,024-row
    coarse sample, a widened sample, and steps whose rows are so far apart
    that the pass limit hands them to the plain binary search)."""
    out = []
    for n, gap in [(70_000, 1_100), (300_000, 40_000), (5_000, 37), (1 << 20, 65_537)]:
        ids = np.arange(0, n - 1, gap, dtype=np.int64)
        out.append(inputs.from_pairs(n, np.stack([ids, ids + 1], 1), f"pairs_n{n}_gap{gap}"))
    # stars with 1..60 leaves, centres 5,000 apart, leaves right after each centre
    rng = np.random.default_rng(7)
    pairs = []
    for c0 in range(0, 200_000 - 64, 5_000):
        for t in range(1, int(rng.integers(1, 61)) + 1):
            pairs.append((c0, c0 + t))
    out.append(inputs.from_pairs(200_000, pairs, "far_stars"))
    # one star whose 222 leaves are 900 ids apart: a walker step over the
    # one-entry leaf rows spans ~115,000 rows, past the 64-pass bound of the
    # coarse-sample search, so the plain binary search places the rest
    leaves = np.arange(900, 200_000, 900, dtype=np.int64)
    out.append(inputs.from_pairs(200_000, np.stack([np.zeros_like(leaves), leaves], 1), "far_leaves"))
    return out


@pytest.mark.parametrize("raw", spread_rows_cases(), ids=lambda r: r.name)
def test_rows_spread_far_apart(raw):
    c = oracle.from_raw(raw)
    g = gpu_graph(raw)
    check_csr(g, c, raw.name)
    check_core(g, c, raw.name)
    check_peel(g, c, 1, 10, raw.name)


def test_ingest_row_classes_at_scale():
    # R-MAT scale 17 plus a Chung-Lu graph with 20k-degree hubs: rows land in
    # every sort class (warp 1/2/4/8/16/32 values per lane, block, and giant
    # rows split into 16 value windows), with heavy repetition in the hubs
    for raw in (inputs.rmat(scale=17, m=1 << 21, seed=17),
                inputs.chung_lu(n=1 << 17, m_draws=1 << 21, gamma=2.1, mean=32.0, wmax=40000.0, seed=3)):
        c = oracle.from_raw(raw)
        deg = np.diff(c.off.astype(np.int64))
        g = gpu_graph(raw)
        check_csr(g, c, raw.name)
    assert deg.max() > 8192


def test_small_rows_at_segment_boundaries():
    # rows of 1..40 distinct neighbours, each pair given up to three times in
    # both directions: the small-row sort's 8-, 16- and 32-entry segments
    # (four, two and one row per warp) and the warp rows just above them,
    # with duplicates to drop at every length; the rows of one 32-row group
    # mix all lengths
    rng = np.random.default_rng(41)
    n = 4096
    pairs = []
    for v in range(1024):
        d = 1 + (v * 7) % 40
        nb = rng.choice(np.arange(1024, n), size=d, replace=False)
        for u in nb:
            for _ in range(int(rng.integers(1, 4))):
                pairs.append((v, int(u)) if rng.integers(2) else (int(u), v))
    raw = inputs.from_pairs(n, pairs, "segment-boundaries")
    c = oracle.from_raw(raw)
    deg = np.diff(c.off.astype(np.int64))
    assert {8, 9, 16, 17, 32, 33} <= set(deg[:1024].tolist())
    g = gpu_graph(raw)
    check_csr(g, c, raw.name)
    check_core(g, c, raw.name)
    check_peel(g, c, 1, 10, raw.name)


def test_chung_lu_hubs_cross_every_row_class():
    # hubs of expected degree up to 30000: rows pass 32 (tile/chunk split,
    # warp/block ingest), 256 (several chunks), 4096 and 8192 (merge-path
    # ingest with two or more merge passes)
    raw = inputs.chung_lu(n=1 << 15, m_draws=1 << 20, gamma=2.1, mean=32.0, wmax=30000.0, seed=5)
    c = oracle.from_raw(raw)
    deg = np.diff(c.off.astype(np.int64))
    assert deg.max() > 16384 - 1000 and (deg > 8192).sum() >= 2
    g = gpu_graph(raw)
    check_csr(g, c)
    check_core(g, c)
    for pq in [(1, 1000), (1, 10), (0, 1)]:
        check_peel(g, c, *pq, tag="cl15")


@pytest.mark.parametrize("chunk_len", [32, 100, 256])
def test_128bit_row_loads_match_the_oracle(chunk_len):
    # long rows read as aligned 16-byte groups: chunk bounds and row starts at
    # every residue mod 4 (masked head and tail groups), hub rows over several
    # chunks; and a borrowed adjacency one entry past a 16-byte boundary, where
    # the scan falls back to one entry per lane
    raw = inputs.chung_lu(n=1 << 14, m_draws=1 << 18, gamma=2.1, mean=24.0, wmax=8000.0, seed=11)
    c = oracle.from_raw(raw)
    dsg.set_tuning(short_max=8, chunk_len=chunk_len, peel_vec=True)
    g = gpu_graph(raw)
    for pq in [(1, 1000), (1, 10), (0, 1)]:
        check_peel(g, c, *pq, tag=f"vec chunk {chunk_len}")
    off_d = torch.from_numpy(c.off.view(np.int64)).cuda()
    buf = torch.zeros(c.adj.shape[0] + 4, dtype=torch.int32, device="cuda")
    buf[1:1 + c.adj.shape[0]] = torch.from_numpy(c.adj.view(np.int32)).cuda()
    g2 = dsg.Graph.from_csr(c.n, off_d, buf[1:1 + c.adj.shape[0]])
    check_peel(g2, c, 1, 10, tag=f"vec misaligned chunk {chunk_len}")


def test_star_hubs_straddle_thresholds():
    # stars whose hub degree sits at / around the tile-chunk split and chunk sizes
    pairs, base = [], 0
    for s in [31, 32, 33, 255, 256, 257, 4095, 4096, 4097, 9000]:
        pairs += [(base, base + j) for j in range(1, s + 1)]
        # connect leaves so the hubs do not all fail in round 0
        pairs += [(base + j, base + j + 1) for j in range(1, s, 3)]
        base += s + 1
    raw = inputs.from_pairs(base, pairs)
    c = oracle.from_raw(raw)
    g = gpu_graph(raw)
    check_csr(g, c)
    check_core(g, c)
    for pq in EPS:
        check_peel(g, c, *pq, tag="stars")


def test_giant_rows_split_or_skewed():
    # rows above 8192 raw entries are cut into value ranges by splitters from
    # a sample of the row; a row whose values are mostly one repeated id makes
    # a range above 8192 entries and takes the radix path instead; rows of
    # distinct ids spread evenly, or crowded into a narrow band of ids
    n = 200_000
    rng = np.random.default_rng(41)
    pairs = [np.stack([np.zeros(15000, np.uint32), np.ones(15000, np.uint32)], 1),       # one id 15000 times
             np.stack([np.zeros(6000, np.uint32), rng.integers(2, n, 6000, dtype=np.uint32)], 1),
             np.stack([np.full(40000, 7, np.uint32), rng.integers(0, n, 40000, dtype=np.uint32)], 1),  # spread
             np.stack([np.full(30000, 9, np.uint32), rng.integers(1000, 1400, 30000, dtype=np.uint32)], 1),  # band
             np.stack([np.full(9000, 11, np.uint32), np.arange(20000, 29000, dtype=np.uint32)], 1)]      # sorted run
    arr = np.concatenate(pairs)
    raw = inputs.RawGraph(n, arr[:, 0].copy(), arr[:, 1].copy(), "giant rows")
    c = oracle.from_raw(raw)
    g = gpu_graph(raw)
    check_csr(g, c)
    check_core(g, c)
    check_peel(g, c, 1, 10, tag="giant rows")


def test_long_paths_and_chains():
    # many-sub-round drains: long paths, a ladder and a caterpillar
    raw = inputs.union(inputs.path(5000),
                       inputs.from_pairs(5000, [(i, i + 2) for i in range(0, 4000, 2)]),
                       inputs.from_pairs(5000, [(i, 4500 + i % 400) for i in range(0, 500)]))
    c = oracle.from_raw(raw)
    g = gpu_graph(raw)
    check_core(g, c)
    for pq in [(0, 1), (1, 1000)]:
        check_peel(g, c, *pq, tag="paths")


@pytest.mark.parametrize("block,short_max,chunk_len,bps", [(256, 1, 32, 0), (512, 32, 256, 1), (1024, 4096, 4096, 0),
                                                           (256, 64, 1024, 2), (1024, 8, 32, 1)])
def test_results_do_not_depend_on_launch_shape(block, short_max, chunk_len, bps):
    raw = inputs.union(inputs.rmat(scale=13, m=1 << 17, seed=3), inputs.block(1 << 13, 90, 0.4, 3))
    c = oracle.from_raw(raw)
    dsg.set_tuning(block=block, blocks_per_sm=bps, short_max=short_max, chunk_len=chunk_len)
    g = gpu_graph(raw)
    check_core(g, c)
    for pq in [(1, 100), (1, 2)]:
        check_peel(g, c, *pq, tag=f"tune {block}/{short_max}/{chunk_len}/{bps}")


@pytest.mark.parametrize("hot_deg", [1, 2, 64, 1 << 30])
def test_hub_combining_does_not_change_results(hot_deg):
    # every decrement combined in shared memory (1, 2), hubs only (64), none
    raw = inputs.chung_lu(n=1 << 14, m_draws=1 << 18, gamma=2.1, mean=32.0, wmax=6000.0, seed=9)
    c = oracle.from_raw(raw)
    dsg.set_tuning(hot_deg=hot_deg)
    g = gpu_graph(raw)
    check_core(g, c, f"hot {hot_deg}")
    for pq in [(1, 1000), (1, 10), (0, 1)]:
        check_peel(g, c, *pq, tag=f"hot {hot_deg}")
    r2 = inputs.rmat(scale=13, m=1 << 17, seed=21)
    c2 = oracle.from_raw(r2)
    g2 = gpu_graph(r2)
    check_core(g2, c2, f"rmat hot {hot_deg}")
    check_peel(g2, c2, 1, 10, tag=f"rmat hot {hot_deg}")


def test_long_chains_overflow_the_block_queue():
    # a path of 20000 vertices hanging off a clique: every level-1 vertex joins
    # a chain far longer than one block's local queue
    n = 20000 + 40
    pairs = [(i, i + 1) for i in range(20000 - 1)] + [(20000 + a, 20000 + b) for a in range(40) for b in range(a + 1, 40)]
    pairs += [(19999, 20000)]
    raw = inputs.from_pairs(n, pairs)
    c = oracle.from_raw(raw)
    for block, local_max in ((256, 1024), (1024, 32), (512, 0), (512, 1 << 30)):
        dsg.set_tuning(block=block, local_max=local_max)
        g = gpu_graph(raw)
        check_core(g, c, f"chain {block}/{local_max}")
        r2 = inputs.rmat(scale=12, m=1 << 16, seed=5)
        c2 = oracle.from_raw(r2)
        check_core(gpu_graph(r2), c2, f"rmat chain {block}/{local_max}")


@pytest.mark.parametrize("inline_max,local_work", [(0, 16384), (256, 0), (16384, 1 << 30), (1 << 30, 4096)])
def test_core_numbers_do_not_depend_on_where_rows_are_drained(inline_max, local_work):
    # scan-found rows drained by the finding block or by every warp, cascades
    # in the block or grid-wide: the same core numbers
    for raw in (inputs.chung_lu(n=1 << 14, m_draws=1 << 18, gamma=2.1, mean=32.0, wmax=6000.0, seed=12),
                inputs.union(inputs.rmat(scale=13, m=1 << 17, seed=13), inputs.block(1 << 13, 120, 0.5, 13))):
        c = oracle.from_raw(raw)
        dsg.set_tuning(inline_max=inline_max, local_work=local_work)
        check_core(gpu_graph(raw), c, f"inline {inline_max}/{local_work}")


@pytest.mark.parametrize("tail", [0, 1, 64, 4096, 131072])
def test_core_numbers_do_not_depend_on_where_the_cluster_takes_over(tail):
    # the grid-wide levels hand the remaining graph to the one-cluster tail
    # after the first level with at most `tail` vertices left (0: never):
    # hub-heavy, planted-block and chain graphs, the largest with more
    # remaining vertices than half the cluster's capacity, give the same core
    # numbers wherever the hand-over happens
    graphs = (inputs.chung_lu(n=1 << 17, m_draws=1 << 20, gamma=2.1, mean=16.0, wmax=8000.0, seed=21),
              inputs.union(inputs.rmat(scale=14, m=1 << 18, seed=22), inputs.block(1 << 14, 300, 0.6, 22)),
              inputs.union(inputs.path(5000), inputs.complete(90)))
    for raw in graphs:
        c = oracle.from_raw(raw)
        dsg.set_tuning(kcore_tail=tail)
        check_core(gpu_graph(raw), c, f"tail {tail}")


def test_from_csr_paths():
    raw = inputs.er_block(n=2000, m=9000, k=40, p=0.5, seed=9)
    c = oracle.from_raw(raw)
    # canonical CSR from host, validated
    g = dsg.Graph.from_csr(c.n, c.off, c.adj, flags=dsg.DSG_CSR_VALIDATE)
    check_peel(g, c, 1, 10)
    check_core(g, c)
    # borrowed device CSR
    off_d = torch.from_numpy(c.off.view(np.int64)).cuda()
    adj_d = torch.from_numpy(c.adj.view(np.int32)).cuda()
    g2 = dsg.Graph.from_csr(c.n, off_d, adj_d)
    check_peel(g2, c, 1, 10)
    # a messy CSR canonicalised on the device
    rng = np.random.default_rng(1)
    rows = [[] for _ in range(50)]
    for _ in range(400):
        a, b = int(rng.integers(50)), int(rng.integers(50))
        rows[a].append(b)
    off = np.zeros(51, np.uint64)
    off[1:] = np.cumsum([len(r) for r in rows])
    adj = np.array([x for r in rows for x in r], np.uint32)
    g3 = dsg.Graph.from_csr(50, off, adj, flags=dsg.DSG_CSR_CANONICALIZE)
    src = np.repeat(np.arange(50, dtype=np.uint32), [len(r) for r in rows])
    c3 = oracle.canonical_csr(50, src, adj)
    check_csr(g3, c3)
    check_peel(g3, c3, 1, 10)


def test_validate_rejects_bad_csr():
    bad_cases = [
        (3, [0, 1, 2, 3], [1, 0, 0]),     # odd entry count: 2 -> 0 has no mirror
        (2, [0, 1, 1], [1]),              # one-sided edge
        (2, [0, 2, 3], [1, 1, 0]),        # repeated neighbour
        (2, [0, 1, 2], [0, 1]),           # self loops
        (3, [0, 2, 3, 4], [2, 1, 0, 0]),  # unsorted row
    ]
    for n, off, adj in bad_cases:
        with pytest.raises(dsg.DsgError) as ei:
            dsg.Graph.from_csr(n, np.array(off, np.uint64), np.array(adj, np.uint32), flags=dsg.DSG_CSR_VALIDATE)
        assert ei.value.status == 1


def test_ingest_rejects_out_of_range_ids():
    with pytest.raises(dsg.DsgError) as ei:
        dsg.Graph.from_edges(4, np.array([0, 1, 9], np.uint32), np.array([1, 2, 3], np.uint32))
    assert ei.value.status == 1


def test_device_inputs_and_outputs():
    raw = inputs.er_block(n=5000, m=20000, k=60, p=0.5, seed=2)
    c = oracle.from_raw(raw)
    src = torch.from_numpy(raw.src.view(np.int32)).cuda()
    dst = torch.from_numpy(raw.dst.view(np.int32)).cuda()
    g = dsg.Graph.from_edges(raw.n, src, dst, stream=torch.cuda.current_stream())
    want = oracle.bahmani(c, 1, 10)
    mask_d = torch.empty(raw.n, dtype=torch.uint8, device="cuda")
    _, E, V = g.bahmani(1, 10, out_set=mask_d)
    assert (E, V) == (want.E, want.V)
    np.testing.assert_array_equal(mask_d.cpu().numpy(), want.mask)
    core_d = torch.empty(raw.n, dtype=torch.int32, device="cuda")
    g.kcore(out=core_d)
    np.testing.assert_array_equal(core_d.cpu().numpy().view(np.uint32), oracle.kcore_bz(c))


def test_repeated_calls_identical():
    raw = inputs.rmat(scale=12, m=1 << 16, seed=7)
    g = gpu_graph(raw)
    outs = [g.bahmani_trace(1, 100) for _ in range(5)]
    for o in outs[1:]:
        np.testing.assert_array_equal(o.peel_round, outs[0].peel_round)
        np.testing.assert_array_equal(o.hist_S, outs[0].hist_S)
    cores = [g.kcore() for _ in range(3)]
    for k in cores[1:]:
        np.testing.assert_array_equal(k, cores[0])


def test_trace_history_overflow_reports_but_keeps_scalars():
    raw = inputs.path(50)
    g = gpu_graph(raw)
    with pytest.raises(dsg.DsgError) as ei:
        g.bahmani_trace(0, 1, hist_cap=1)
    assert ei.value.status == 8


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_time_out_cleanly(which):
    # A wait that can never complete (a flag nothing sets; a grid barrier one
    # block skips) must end with DSG_ETIMEOUT, and the context stays usable.
    from paper_2103_00154_gb300 import _native as N
    st = dsg.lib().dsg_debug_wait_timeout(which, 50_000_000)  # 50 ms
    assert st == N.DSG_ETIMEOUT, dsg.lib().dsg_last_error()
    raw = inputs.er_block(n=3000, m=12000, k=50, p=0.5, seed=3)
    check_peel(gpu_graph(raw), oracle.from_raw(raw), 1, 10)
