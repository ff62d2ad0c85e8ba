"""Pins for the CPU oracle against facts that do not come from the oracle.

Closed forms, hand-worked examples (tests/golden/), exact optima by subset
enumeration and by Goldberg's min-cut, a library routine (networkx
core_number), invariants that Algorithm 1 must satisfy, and a second,
independent statement of each computation.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import inputs
import oracle
from golden_io import all_fixtures, load, load_cbds

EPS = [(0, 1), (1, 1000), (1, 100), (1, 10), (1, 2), (1, 1), (3, 2)]


def csr_of(g):
    return oracle.from_raw(g)


# ------------------------------------------------------------------ ingest
def test_canonical_csr_matches_edge_set_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(1, 40))
        m = int(rng.integers(0, 200))
        src = rng.integers(0, n, m).astype(np.uint32)
        dst = rng.integers(0, n, m).astype(np.uint32)
        c = oracle.canonical_csr(n, src, dst)
        want = {v: set() for v in range(n)}
        for a, b in zip(src.tolist(), dst.tolist()):
            if a != b:
                want[a].add(b)
                want[b].add(a)
        assert c.off[0] == 0 and len(c.off) == n + 1
        for v in range(n):
            row = c.adj[int(c.off[v]):int(c.off[v + 1])].tolist()
            assert row == sorted(want[v]), (trial, v)


def test_canonical_csr_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.canonical_csr(3, np.array([0, 5], np.uint32), np.array([1, 1], np.uint32))


# ----------------------------------------------------- hand-worked examples
@pytest.mark.parametrize("name", all_fixtures())
def test_bahmani_hand_worked(name):
    fx = load(name)
    c = csr_of(inputs.from_pairs(fx["n"], fx["pairs"]))
    for fn in (oracle.bahmani, oracle.bahmani_recompute):
        r = fn(c, fx["p"], fx["q"])
        assert r.rounds == fx["rounds"]
        assert r.best_round == fx["best_round"]
        assert (r.E, r.V) == (fx["E"], fx["V"])
        np.testing.assert_array_equal(r.hist_S, fx["hist_S"])
        np.testing.assert_array_equal(r.hist_E, fx["hist_E"])
        np.testing.assert_array_equal(r.peel_round, fx["peel_round"])


@pytest.mark.parametrize("name", all_fixtures())
def test_kcore_hand_worked(name):
    fx = load(name)
    c = csr_of(inputs.from_pairs(fx["n"], fx["pairs"]))
    for fn in (oracle.kcore_bz, oracle.kcore_naive, oracle.kcore_pkc):
        np.testing.assert_array_equal(fn(c), fx["core"])


@pytest.mark.parametrize("name", all_fixtures("cbds_"))
def test_cbds_hand_worked(name):
    fx = load_cbds(name)
    c = csr_of(inputs.from_pairs(fx["n"], fx["pairs"]))
    core = oracle.kcore_bz(c)
    np.testing.assert_array_equal(core, fx["core"])
    dc = oracle.densest_core(c, core)
    assert dc == fx["densest_core"]
    me, mv, nleg, _ = oracle.cbds_phase2(c, core, *dc)
    assert (me, mv, nleg) == fx["phase2"]


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [1, 2, 3, 7, 30])
@pytest.mark.parametrize("pq", EPS)
def test_complete_graph(n, pq):
    # K_n: every degree n-1 equals the average degree 2 rho, so all fail at once.
    c = csr_of(inputs.complete(n))
    r = oracle.bahmani(c, *pq)
    assert r.rounds == 1 and r.best_round == 0
    assert (r.E, r.V) == (n * (n - 1) // 2, n)
    assert r.mask.all()
    assert (oracle.kcore_bz(c) == n - 1).all()


@pytest.mark.parametrize("s", [1, 2, 5, 50])
def test_star(s):
    # K_{1,s}, eps small: round 0 drops the leaves (degree 1 <= 2(1+eps) s/(s+1)),
    # the hub (degree s) survives when s > 2(1+eps)s/(s+1), i.e. s >= 2;
    # the lone hub then fails.  Best = the whole star.
    c = csr_of(inputs.star(s))
    r = oracle.bahmani(c, 1, 100)
    if s >= 2:
        assert r.rounds == 2 and list(r.hist_S) == [s + 1, 1, 0]
    else:
        assert r.rounds == 1
    assert r.best_round == 0 and (r.E, r.V) == (s, s + 1)
    assert (oracle.kcore_bz(c) == 1).all()


@pytest.mark.parametrize("n", [0, 1, 5, 100])
def test_edgeless(n):
    c = csr_of(inputs.empty(n))
    r = oracle.bahmani(c, 1, 10)
    if n == 0:
        assert r.rounds == 0 and (r.E, r.V) == (0, 0)
    else:
        assert r.rounds == 1 and r.best_round == 0 and (r.E, r.V) == (0, n)
    assert (oracle.kcore_bz(c) == 0).all()


@pytest.mark.parametrize("a,b", [(6, 3), (10, 9), (5, 2)])
def test_disjoint_cliques_pick_larger(a, b):
    c = csr_of(inputs.disjoint_cliques([a, b]))
    r = oracle.bahmani(c, 1, 1000)
    assert (r.E, r.V) == (a * (a - 1) // 2, a)
    assert r.mask[:a].all() and not r.mask[a:].any()


def test_two_equal_cliques_keep_round_zero():
    c = csr_of(inputs.disjoint_cliques([6, 6]))
    r = oracle.bahmani(c, 0, 1)
    assert r.rounds == 1 and r.best_round == 0 and (r.E, r.V) == (30, 12)


@pytest.mark.parametrize("n", [3, 4, 10])
def test_cycle_and_path_cores(n):
    assert (oracle.kcore_bz(csr_of(inputs.cycle(n))) == 2).all()
    assert (oracle.kcore_bz(csr_of(inputs.path(n))) == 1).all()
    # cycle, eps = 0: every degree equals 2 rho = 2, "<=" removes all at once
    r = oracle.bahmani(csr_of(inputs.cycle(n)), 0, 1)
    assert r.rounds == 1 and (r.E, r.V) == (n, n)


def test_named_graph_cores():
    # Petersen graph: 3-regular, connected -> all core 3
    outer = [(i, (i + 1) % 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    pet = inputs.from_pairs(10, outer + inner + spokes)
    assert (oracle.kcore_bz(csr_of(pet)) == 3).all()
    # hypercube Q4: 4-regular -> core 4
    q4 = inputs.from_pairs(16, [(v, v ^ (1 << b)) for v in range(16) for b in range(4) if v < v ^ (1 << b)])
    assert (oracle.kcore_bz(csr_of(q4)) == 4).all()
    # complete bipartite K_{3,5}: core min(3,5) = 3
    kb = inputs.from_pairs(8, [(i, 3 + j) for i in range(3) for j in range(5)])
    assert (oracle.kcore_bz(csr_of(kb)) == 3).all()
    # 5x5 grid: every vertex in the 2-core, none in a 3-core
    grid = [(r * 5 + c, r * 5 + c + 1) for r in range(5) for c in range(4)] + \
           [(r * 5 + c, (r + 1) * 5 + c) for r in range(4) for c in range(5)]
    assert (oracle.kcore_bz(csr_of(inputs.from_pairs(25, grid))) == 2).all()


# ---------------------------------------------------- second statements
def _random_graphs(count, seed):
    rng = np.random.default_rng(seed)
    for i in range(count):
        n = int(rng.integers(1, 120))
        p = float(rng.choice([0.02, 0.05, 0.1, 0.3, 0.7]))
        g = inputs.random_small(n, p, int(rng.integers(1 << 30)))
        if i % 3 == 0 and n >= 4:  # plant a dense block
            k = max(2, n // 5)
            g = inputs.union(g, inputs.from_pairs(n, [(a, b) for a in range(k) for b in range(a + 1, k)]))
        yield g


@pytest.mark.parametrize("pq", EPS)
def test_incremental_equals_recompute(pq):
    for g in _random_graphs(60, 11 + pq[0] * 7 + pq[1]):
        c = csr_of(g)
        a = oracle.bahmani(c, *pq)
        b = oracle.bahmani_recompute(c, *pq)
        assert (a.rounds, a.best_round, a.E, a.V) == (b.rounds, b.best_round, b.E, b.V)
        np.testing.assert_array_equal(a.hist_S, b.hist_S)
        np.testing.assert_array_equal(a.hist_E, b.hist_E)
        np.testing.assert_array_equal(a.peel_round, b.peel_round)


def test_kcore_three_statements_agree():
    for g in _random_graphs(80, 3):
        c = csr_of(g)
        bz = oracle.kcore_bz(c)
        np.testing.assert_array_equal(bz, oracle.kcore_naive(c))
        np.testing.assert_array_equal(bz, oracle.kcore_pkc(c))


def test_kcore_matches_networkx():
    nx = pytest.importorskip("networkx")
    for g in list(_random_graphs(40, 99)) + [inputs.er_block(n=3000, m=12000, k=60, p=0.5, seed=4)]:
        c = csr_of(g)
        G = nx.Graph()
        G.add_nodes_from(range(c.n))
        for v in range(c.n):
            for u in c.adj[int(c.off[v]):int(c.off[v + 1])]:
                if u > v:
                    G.add_edge(v, int(u))
        cn = nx.core_number(G)
        want = np.array([cn[v] for v in range(c.n)], np.uint32)
        np.testing.assert_array_equal(oracle.kcore_bz(c), want)


# --------------------------------------------------------------- invariants
def _check_peel_invariants(c, r, p, q):
    n = c.n
    deg0 = np.diff(c.off.astype(np.int64))
    assert r.hist_S[0] == n and r.hist_E[0] == c.m
    assert r.rounds <= oracle.round_bound(n, p, q)
    if n:
        assert r.peel_round.min() >= 1 and r.peel_round.max() == r.rounds
    for t in range(r.rounds + 1):
        alive = r.peel_round > t
        assert int(alive.sum()) == int(r.hist_S[t])
        # E_t = edges induced by S_t (Def. 1), from scratch
        src = np.repeat(np.arange(n), deg0)
        inside = alive[src] & alive[c.adj.astype(np.int64)]
        assert int(inside.sum()) == 2 * int(r.hist_E[t])
    for t in range(r.rounds):
        S, E, S1 = int(r.hist_S[t]), int(r.hist_E[t]), int(r.hist_S[t + 1])
        assert S1 < S  # at least one vertex fails per round
        if E > 0:
            assert (p + q) * S1 < q * S  # geometric shrink
        else:
            assert S1 == 0
    # best = earliest round of maximum density among non-empty sets
    dens = [Fraction(int(r.hist_E[t]), int(r.hist_S[t])) for t in range(r.rounds) if r.hist_S[t] > 0]
    if dens:
        mx = max(dens)
        assert r.best_round == dens.index(mx)
        assert Fraction(r.E, r.V) == mx
        np.testing.assert_array_equal(r.mask, (r.peel_round > r.best_round).astype(np.uint8))


@pytest.mark.parametrize("pq", EPS)
def test_peel_invariants(pq):
    for g in _random_graphs(40, 1000 + pq[1]):
        c = csr_of(g)
        _check_peel_invariants(c, oracle.bahmani(c, *pq), *pq)


def test_peel_invariants_config_small():
    c = csr_of(inputs.er_block())
    for pq in [(1, 10), (1, 1000), (0, 1)]:
        _check_peel_invariants(c, oracle.bahmani(c, *pq), *pq)


def test_kcore_invariants():
    for g in _random_graphs(40, 77):
        c = csr_of(g)
        core = oracle.kcore_bz(c).astype(np.int64)
        deg = np.diff(c.off.astype(np.int64))
        assert (core <= deg).all()
        src = np.repeat(np.arange(c.n), deg)
        dst = c.adj.astype(np.int64)
        for k in range(int(core.max(initial=0)) + 1):
            ins = core >= k
            d_in = np.bincount(src[ins[src] & ins[dst]], minlength=c.n)
            assert (d_in[ins] >= k).all()  # {core >= k} has min degree >= k
        # h-index fixed point: core(v) = largest h with h neighbours of core >= h
        for v in range(c.n):
            nb = np.sort(core[dst[int(c.off[v]):int(c.off[v + 1])]])[::-1]
            h = 0
            while h < len(nb) and nb[h] >= h + 1:
                h += 1
            assert core[v] == h


# ------------------------------------------------------------ exact optima
def _density_brute_python(n, pairs):
    best = Fraction(0)
    for k in range(1, n + 1):
        for sub in itertools.combinations(range(n), k):
            s = set(sub)
            e = sum(1 for a, b in pairs if a in s and b in s)
            best = max(best, Fraction(e, k))
    return best


def test_brute_force_matches_python_enumeration():
    rng = np.random.default_rng(8)
    for _ in range(15):
        n = int(rng.integers(1, 9))
        g = inputs.random_small(n, 0.5, int(rng.integers(1 << 30)))
        c = csr_of(g)
        E, V, _ = oracle.brute_densest(c)
        pairs = list(zip(g.src.tolist(), g.dst.tolist()))
        assert Fraction(E, V) == _density_brute_python(n, pairs)


def test_goldberg_matches_brute_force():
    rng = np.random.default_rng(9)
    for _ in range(60):
        n = int(rng.integers(1, 17))
        g = inputs.random_small(n, float(rng.choice([0.1, 0.3, 0.6])), int(rng.integers(1 << 30)))
        c = csr_of(g)
        Eb, Vb, _ = oracle.brute_densest(c)
        Eg, Vg, mask = oracle.goldberg_densest(c)
        assert Fraction(Eg, Vg) == Fraction(Eb, Vb)
        # the returned set really has that density
        sel = mask.astype(bool)
        deg = np.diff(c.off.astype(np.int64))
        src = np.repeat(np.arange(c.n), deg)
        inside = sel[src] & sel[c.adj.astype(np.int64)]
        assert int(sel.sum()) == Vg and int(inside.sum()) == 2 * Eg


@pytest.mark.parametrize("pq", EPS)
def test_bahmani_bound_brute_force(pq):
    # rho(S~) >= rho* / (2 + 2 eps)  <=>  2 (p+q) E~ V* >= q E* V~
    p, q = pq
    rng = np.random.default_rng(100 + q)
    for _ in range(40):
        n = int(rng.integers(1, 15))
        c = csr_of(inputs.random_small(n, float(rng.choice([0.2, 0.4, 0.7])), int(rng.integers(1 << 30))))
        r = oracle.bahmani(c, p, q)
        Es, Vs, _ = oracle.brute_densest(c)
        if Es == 0:
            continue
        assert 2 * (p + q) * r.E * Vs >= q * Es * r.V


def test_bahmani_and_core_bounds_goldberg():
    # (2+2eps) bound for the peel, and the densest core is a 2-approximation
    for seed, (n, m, k) in enumerate([(400, 1200, 20), (1500, 6000, 40), (3000, 9000, 12)]):
        c = csr_of(inputs.er_block(n=n, m=m, k=k, p=0.5, seed=seed))
        Es, Vs, _ = oracle.goldberg_densest(c)
        for p, q in EPS:
            r = oracle.bahmani(c, p, q)
            assert 2 * (p + q) * r.E * Vs >= q * Es * r.V
        core = oracle.kcore_bz(c)
        kstar, Ek, Vk = oracle.densest_core(c, core)
        assert 2 * Ek * Vs >= Es * Vk
        me, mv, nleg, _ = oracle.cbds_phase2(c, core, kstar, Ek, Vk)
        assert me * Vk >= Ek * mv  # augmentation never lowers the density
        assert me * Vs <= Es * mv  # and never beats the optimum


def test_densest_core_brute_force():
    rng = np.random.default_rng(12)
    for _ in range(30):
        g = inputs.random_small(int(rng.integers(2, 60)), float(rng.choice([0.05, 0.2, 0.5])),
                                int(rng.integers(1 << 30)))
        c = csr_of(g)
        core = oracle.kcore_bz(c).astype(np.int64)
        deg = np.diff(c.off.astype(np.int64))
        src = np.repeat(np.arange(c.n), deg)
        dst = c.adj.astype(np.int64)
        best = None
        for k in range(int(core.max()) + 1):
            ins = core >= k
            V = int(ins.sum())
            E = int((ins[src] & ins[dst]).sum()) // 2
            if V and (best is None or Fraction(E, V) > Fraction(best[1], best[2])):
                best = (k, E, V)
        assert oracle.densest_core(c, core.astype(np.uint32)) == best


def test_cbds_phase2_counts_the_augmented_set():
    # m_e / m_v must be exactly the induced density of (densest core U legit)
    rng = np.random.default_rng(13)
    hits = 0
    for _ in range(60):
        n = int(rng.integers(10, 200))
        g = inputs.union(inputs.random_small(n, 0.05, int(rng.integers(1 << 30))),
                         inputs.from_pairs(n, [(a, b) for a in range(8) for b in range(a + 1, 8)]),
                         inputs.from_pairs(n, [(8 + j, a) for j in range(4) for a in range(5)]))
        c = csr_of(g)
        core = oracle.kcore_bz(c)
        kstar, Ek, Vk = oracle.densest_core(c, core)
        me, mv, nleg, legit = oracle.cbds_phase2(c, core, kstar, Ek, Vk)
        sel = (core >= kstar) | legit.astype(bool)
        deg = np.diff(c.off.astype(np.int64))
        src = np.repeat(np.arange(c.n), deg)
        E = int((sel[src] & sel[c.adj.astype(np.int64)]).sum()) // 2
        assert (me, mv) == (E, int(sel.sum()))
        assert nleg == int(legit.sum())
        # each legit vertex has more edges into the core than the core's density
        for v in np.flatnonzero(legit):
            into = int((core[c.adj[int(c.off[v]):int(c.off[v + 1])]] >= kstar).sum())
            assert into * Vk > Ek and core[v] < kstar
        hits += nleg > 0
    assert hits > 0  # the planted satellites make some cases non-trivial


# ---------------------------------------------------------------- inputs
def test_generators_deterministic_and_threads_invariant():
    lib = inputs._load()
    import ctypes
    for threads in (1, 3, 8):
        src = np.empty(5000, np.uint32)
        dst = np.empty(5000, np.uint32)
        lib.gen_rmat(12, 5000, 0.57, 0.19, 0.19, 1, inputs._p32(src), inputs._p32(dst), threads)
        if threads == 1:
            ref = (src.copy(), dst.copy())
        else:
            np.testing.assert_array_equal(src, ref[0])
            np.testing.assert_array_equal(dst, ref[1])
    e = inputs.er(1000, 5000, 0)
    keys = set()
    for a, b in zip(e.src.tolist(), e.dst.tolist()):
        assert a != b
        keys.add((min(a, b), max(a, b)))
    assert len(keys) == 5000
    g1 = inputs.er_block()
    g2 = inputs.er_block()
    np.testing.assert_array_equal(g1.src, g2.src)


def test_chung_lu_weights_shape():
    w = inputs.chung_lu_weights(1 << 16, 2.1, 32.0, 1000.0)
    assert abs(w.mean() - 32.0) < 1e-6 * 32 and abs(w[0] - 1000.0) < 1e-6 * 1000
    assert (np.diff(w) <= 0).all()


def test_table3_cbds_not_below_the_eps0_peel_on_synthetic_graphs():
    """Table 3 (Sec. 4) reports CBDS-P's density at or above P-Bahmani's at
    eps = 0 on every dataset.  The datasets are not available; the same
    comparison, exact in rationals, on synthetic stand-ins of each family the
    benchmarks use (planted-block Erdos-Renyi, R-MAT, Chung-Lu, batch members).
    It is an observation of the paper, not a theorem; these instances hold it."""
    from fractions import Fraction
    cases = [inputs.er_block(n=3000, m=12000, k=40 + 5 * s, p=0.3 + 0.05 * (s % 5), seed=s) for s in range(6)]
    cases += [inputs.rmat(scale=12 + s % 3, m=(8 + 4 * (s % 3)) << (12 + s % 3), seed=100 + s) for s in range(3)]
    cases += [inputs.chung_lu(n=1 << 12, m_draws=1 << 16, gamma=2.1 + 0.1 * s, mean=16.0, wmax=0.0, seed=200 + s)
              for s in range(3)]
    cases += [inputs.batch_graph(i, n_lo=1000, n_hi=8000) for i in range(4)]
    for raw in cases:
        c = oracle.from_raw(raw)
        peel0 = oracle.bahmani(c, 0, 1)
        core = oracle.kcore_bz(c)
        k, Ek, Vk = oracle.densest_core(c, core)
        me, mv, _, _ = oracle.cbds_phase2(c, core, k, Ek, Vk)
        assert Fraction(me, mv) >= Fraction(peel0.E, peel0.V), raw.name
        assert Fraction(me, mv) >= Fraction(Ek, Vk), raw.name  # phase 2 never loses density (Sec. 3.2)


def test_onion_shells_peel_one_per_round():
    # the nested-shell generator: every vertex of shell i >= 1 has exactly d edges into
    # shell i - 1 and every vertex inside gets at least d + 1 from its outer shell, so at
    # eps < 1/(2d) each round of the peel removes the outermost shell and nothing else
    raw = inputs.onion(1 << 12, 8, 24)
    c = oracle.from_raw(raw)
    deg = np.diff(c.off.astype(np.int64))
    sizes = [24]
    while sum(sizes) < 1 << 12:
        sizes.append(-(-sizes[-1] * 9 // 8))
    assert raw.n == sum(sizes)
    outer = deg[raw.n - sizes[-1]:]
    assert (outer == 8).all()
    inner = deg[24:raw.n - sizes[-1]]
    assert inner.min() >= 2 * 8 + 1
    r = oracle.bahmani(c, 1, 1000)
    assert r.rounds >= len(sizes) - 3
    # round t removes exactly the outermost remaining shell
    for t in range(1, 10):
        assert int(r.hist_S[t - 1] - r.hist_S[t]) == sizes[-t]
