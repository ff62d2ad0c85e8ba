"""GPU parity of the densest k-core (Sec. 3.2) and CBDS-P's second phase
(Algorithm 2) against the oracle: (k*, E_k*, V_k*), (m_e, m_v, #legit), the
result set and the core numbers, bit for bit.  Cases: the hand-worked
fixtures, closed forms, edge cases (no vertex, no edge, ties between equal
cores), random graphs with planted cores and satellites across many tiles,
caller-supplied value arrays on host and device (including values that take
the histogram out of shared memory), and the R-MAT scale-20 graph checked
against the definition."""
import numpy as np
import pytest

import inputs
import oracle
from golden_io import all_fixtures, load_cbds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402


def gpu_graph(raw):
    return dsg.Graph.from_edges(raw.n, raw.src, raw.dst)


def check_all(raw, core=None, tag=""):
    c = oracle.from_raw(raw)
    ocore = oracle.kcore_bz(c) if core is None else np.asarray(core, np.uint32)
    kstar, Ek, Vk = oracle.densest_core(c, ocore)
    me, mv, nleg, legit = oracle.cbds_phase2(c, ocore, kstar, Ek, Vk)
    g = gpu_graph(raw)
    try:
        d = g.densest_core(core=core)
        assert (d.k_star, d.E_core, d.V_core) == (kstar, Ek, Vk), tag
        assert (d.E, d.V, d.n_legit) == (Ek, Vk, 0), tag
        np.testing.assert_array_equal(d.mask, (ocore >= kstar).astype(np.uint8), err_msg=tag)
        r = g.cbds(core=core)
        assert (r.k_star, r.E_core, r.V_core) == (kstar, Ek, Vk), tag
        assert (r.E, r.V, r.n_legit) == (me, mv, nleg), tag
        np.testing.assert_array_equal(r.mask, ((ocore >= kstar) | legit.astype(bool)).astype(np.uint8), err_msg=tag)
        np.testing.assert_array_equal(np.asarray(r.core)[:raw.n], ocore, err_msg=tag)
    finally:
        g.close()
    return (kstar, Ek, Vk), (me, mv, nleg)


@pytest.mark.parametrize("name", all_fixtures("cbds_"))
def test_hand_worked_fixtures(name):
    fx = load_cbds(name)
    dc, p2 = check_all(inputs.from_pairs(fx["n"], fx["pairs"]), tag=name)
    assert dc == fx["densest_core"] and p2 == fx["phase2"]


@pytest.mark.parametrize("raw", [inputs.complete(7), inputs.star(9), inputs.path(12), inputs.cycle(10),
                                 inputs.disjoint_cliques([6, 6]), inputs.disjoint_cliques([9, 5, 3]),
                                 inputs.empty(5), inputs.empty(1)], ids=lambda r: r.name)
def test_closed_forms_and_edges(raw):
    (kstar, Ek, Vk), _ = check_all(raw, tag=raw.name)
    if raw.name == "K7":
        assert (kstar, Ek, Vk) == (0, 21, 7)  # every k-core is all of K7: the smallest k wins
    if raw.name.startswith("empty"):
        assert (kstar, Ek, Vk) == (0, 0, raw.n)
    if raw.name == "cliques(6, 6)":
        assert (kstar, Ek, Vk) == (0, 30, 12)  # equal cores: the smallest k (all of V) wins


def test_no_vertex():
    g = dsg.Graph.from_edges(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    try:
        r = g.cbds()
        assert (r.k_star, r.E_core, r.V_core, r.E, r.V, r.n_legit) == (0, 0, 0, 0, 0, 0)
    finally:
        g.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_with_satellites(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3000, 40000))
    k = int(rng.integers(20, 80))
    base = inputs.er_pairs(n, int(rng.integers(2, 6)) * n, seed)
    core_block = inputs.block(n, k, 0.6, seed)
    # satellites: vertices k..k+s-1 joined to many core vertices and to each other
    s = int(rng.integers(5, 60))
    sat = inputs.from_pairs(n, [(k + i, int(a)) for i in range(s)
                                for a in rng.choice(k, int(rng.integers(k // 4, k // 2)), replace=False)]
                            + [(k + i, k + i + 1) for i in range(s - 1)])
    raw = inputs.union(base, core_block, sat)
    _, (me, mv, nleg) = check_all(raw, tag=f"seed{seed}")


@pytest.mark.parametrize("gen", ["chung_lu", "rmat"])
def test_power_law(gen):
    if gen == "chung_lu":
        raw = inputs.chung_lu(1 << 16, 1 << 20, 2.1, 32.0, 20000.0, 11)
    else:
        raw = inputs.rmat(scale=15, m=1 << 19, seed=4)
    check_all(raw, tag=gen)


@pytest.mark.parametrize("n,gap", [(70_000, 1_100), (1 << 20, 65_537)])
def test_rows_spread_far_apart(n, gap):
    # non-empty rows far apart: the histogram's edge walker crosses long runs
    # of empty rows (coarse samples, widened samples, the pass limit)
    ids = np.arange(0, n - 1, gap, dtype=np.int64)
    pairs = np.concatenate([np.stack([ids, ids + 1], 1), [[1, 2], [2, 3], [1, 3]]])
    check_all(inputs.from_pairs(n, pairs), tag=f"spread n={n} gap={gap}")


def test_leaves_past_the_search_pass_bound():
    # a star with leaves 900 ids apart plus a triangle: the histogram walker's
    # steps over the leaf rows need more than 64 coarse-sample passes
    leaves = np.arange(900, 200_000, 900, dtype=np.int64)
    pairs = np.concatenate([np.stack([np.zeros_like(leaves), leaves], 1), [[1, 2], [2, 3], [1, 3]]])
    check_all(inputs.from_pairs(200_000, pairs), tag="far leaves")


def test_supplied_values_host_device_and_global_histogram():
    raw = inputs.er_block(n=9000, m=40000, k=60, p=0.5, seed=7)
    c = oracle.from_raw(raw)
    deg = np.diff(c.off.astype(np.int64)).astype(np.uint32)
    # the degrees as the "core" values: the densest-core scan and phase 2 are
    # defined for any values below n
    check_all(raw, core=deg, tag="degree values")
    # large values: the histograms leave shared memory (k_max >= 4096)
    rng = np.random.default_rng(3)
    vals = rng.integers(0, 6000, raw.n).astype(np.uint32)
    vals[:60] = 5999
    check_all(raw, core=vals, tag="large values")
    # device-resident values give the same answer
    g = gpu_graph(raw)
    try:
        a = g.cbds(core=vals)
        b = g.cbds(core=torch.from_numpy(vals.view(np.int32)).cuda())
        assert (a.k_star, a.E_core, a.V_core, a.E, a.V, a.n_legit) == (b.k_star, b.E_core, b.V_core, b.E, b.V,
                                                                      b.n_legit)
        bad = vals.copy()
        bad[5] = raw.n
        with pytest.raises(dsg.DsgError):
            g.cbds(core=bad)
    finally:
        g.close()


def test_device_outputs():
    raw = inputs.er_block(n=20000, m=80000, k=80, p=0.5, seed=9)
    g = gpu_graph(raw)
    try:
        host = g.cbds()
        core_d = torch.empty(raw.n, dtype=torch.int32, device="cuda")
        set_d = torch.empty(raw.n, dtype=torch.uint8, device="cuda")
        dev = g.cbds(out_core=core_d, out_set=set_d)
        assert (dev.E, dev.V, dev.n_legit, dev.k_star) == (host.E, host.V, host.n_legit, host.k_star)
        np.testing.assert_array_equal(set_d.cpu().numpy(), host.mask)
        np.testing.assert_array_equal(core_d.cpu().numpy().view(np.uint32), host.core)
    finally:
        g.close()


def test_rmat20_against_the_definition():
    # full-size: (k*, E_k*, V_k*) checked against numpy histograms of the
    # oracle's core numbers, phase 2 against its per-vertex definition
    raw = inputs.rmat(scale=20, m=1 << 24, a=0.57, b=0.19, c=0.19, seed=1)
    c = oracle.from_raw(raw)
    core = oracle.kcore_bz(c)
    g = gpu_graph(raw)
    try:
        r = g.cbds()
    finally:
        g.close()
    np.testing.assert_array_equal(r.core, core)
    deg = np.diff(c.off.astype(np.int64))
    src = np.repeat(np.arange(c.n, dtype=np.int64), deg)
    dst = c.adj.astype(np.int64)
    once = dst > src
    kmax = int(core.max())
    hv = np.bincount(core, minlength=kmax + 1)
    he = np.bincount(np.minimum(core[src[once]], core[dst[once]]), minlength=kmax + 1)
    Vs = np.cumsum(hv[::-1])[::-1]
    Es = np.cumsum(he[::-1])[::-1]
    best = 0
    for k in range(1, kmax + 1):
        if int(Es[k]) * int(Vs[best]) > int(Es[best]) * int(Vs[k]):
            best = k
    assert (r.k_star, r.E_core, r.V_core) == (best, int(Es[best]), int(Vs[best]))
    ks, Ek, Vk = best, int(Es[best]), int(Vs[best])
    inside = core >= ks
    elig = (core.astype(np.int64) * Vk > Ek) & (core < ks)
    cnt = np.bincount(src[inside[dst]], minlength=c.n)
    legit = elig & (cnt * Vk > Ek)
    pairs = int((legit[src] & legit[dst] & once).sum())
    assert r.n_legit == int(legit.sum())
    assert (r.E, r.V) == (Ek + int(cnt[legit].sum()) + pairs, Vk + int(legit.sum()))
    np.testing.assert_array_equal(r.mask, (inside | legit).astype(np.uint8))
