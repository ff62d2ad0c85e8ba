"""Serving loop (dsg_serve_*): results equal the oracle's for every request;
a request gives bit-identical results alone and amid a stream of others;
back-pressure, budget rejection and shutdown with work in flight behave."""
import threading
import time

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402


def _pool(k=24, seed=3):
    rng = np.random.default_rng(seed)
    pool = [inputs.batch_graph(i, n_lo=500, n_hi=40000, threads=1) for i in range(k)]
    pool += [inputs.star(200), inputs.path(300), inputs.empty(5), inputs.complete(20)]
    return pool


def _check(resp, c, p, q, out_set=None, core=None):
    want = oracle.bahmani(c, p, q)
    assert resp["status"] == 0
    assert (resp["E"], resp["V"], resp["rounds"], resp["best_round"]) == (want.E, want.V, want.rounds, want.best_round)
    assert resp["m"] == c.m
    if out_set is not None:
        np.testing.assert_array_equal(out_set[:c.n], want.mask)
    if core is not None:
        np.testing.assert_array_equal(core[:c.n], oracle.kcore_bz(c))


def test_requests_match_the_oracle():
    pool = _pool()
    csrs = [oracle.from_raw(g) for g in pool]
    rng = np.random.default_rng(1)
    with dsg.Server(max_batch=16) as srv:
        tickets = []
        for i in range(60):
            j = int(rng.integers(len(pool)))
            p, q = [(1, 100), (1, 10), (0, 1)][i % 3]
            want_core = i % 2 == 0
            out_set = np.zeros(max(pool[j].n, 1), np.uint8)
            core = np.zeros(max(pool[j].n, 1), np.uint32) if want_core else None
            t = srv.submit(pool[j].n, pool[j].src, pool[j].dst, p, q, want_core, out_set, core)
            assert t is not None
            tickets.append((t, j, p, q, out_set, core))
        for t, j, p, q, out_set, core in tickets:
            _check(srv.wait(t), csrs[j], p, q, out_set, core)
        st = srv.stats()
        assert st["completed"] == 60 and st["p99_us"] >= st["p50_us"] > 0 and st["batches"] >= 1
        assert st["hbm_in_use"] == 0


@pytest.mark.parametrize("big_threads,big_work,batch_work,inflight",
                         [(3, 20000, 0, 2), (1, 1, 0, 4), (2, 0, 50000, 8), (2, 2 ** 64 - 1, 1, 1)])
def test_server_settings_do_not_change_results(big_threads, big_work, batch_work, inflight):
    # requests solved alone by several big-request threads (big_work 1: every
    # one), launches closed by a work cap (1: one graph per launch), many or
    # one launch in flight, no big-request path at all: every result is the
    # oracle's and the time split adds up
    pool = _pool(k=12, seed=5)
    csrs = [oracle.from_raw(g) for g in pool]
    rng = np.random.default_rng(2)
    with dsg.Server(max_batch=8, big_threads=big_threads, big_work=big_work, max_batch_work=batch_work,
                    max_inflight=inflight) as srv:
        tickets = []
        for i in range(30):
            j = int(rng.integers(len(pool)))
            p, q = [(1, 100), (1, 10)][i % 2]
            want_core = i % 3 == 0
            out_set = np.zeros(max(pool[j].n, 1), np.uint8)
            core = np.zeros(max(pool[j].n, 1), np.uint32) if want_core else None
            t = srv.submit(pool[j].n, pool[j].src, pool[j].dst, p, q, want_core, out_set, core)
            assert t is not None
            tickets.append((t, j, p, q, out_set, core))
        for t, j, p, q, out_set, core in tickets:
            _check(srv.wait(t), csrs[j], p, q, out_set, core)
        st = srv.stats()
        assert st["completed"] == 30
        if big_work == 1:
            assert st["big_done"] == 30
        if big_work == 2 ** 64 - 1:
            assert st["big_done"] == 0
        assert st["ingest_busy_s"] > 0
        assert st["big_busy_s"] >= 0 and st["batch_device_s"] >= 0


def test_same_result_alone_and_in_the_mix():
    pool = _pool(k=16, seed=9)
    probe = inputs.batch_graph(3, n_lo=20000, n_hi=60000, threads=1)
    c = oracle.from_raw(probe)
    with dsg.Server(max_batch=32) as srv:
        set_alone = np.zeros(probe.n, np.uint8)
        core_alone = np.zeros(probe.n, np.uint32)
        alone = srv.wait(srv.submit(probe.n, probe.src, probe.dst, 1, 10, True, set_alone, core_alone))
        # the same request amid a Poisson-like stream submitted from another thread
        stop = threading.Event()
        others = []

        def feeder():
            rng = np.random.default_rng(4)
            while not stop.is_set():
                g = pool[int(rng.integers(len(pool)))]
                t = srv.submit(g.n, g.src, g.dst, 1, 100, bool(rng.integers(2)))
                if t is not None:
                    others.append(t)
                time.sleep(float(rng.exponential(0.0005)))

        th = threading.Thread(target=feeder)
        th.start()
        time.sleep(0.05)
        set_mix = np.zeros(probe.n, np.uint8)
        core_mix = np.zeros(probe.n, np.uint32)
        mixed = srv.wait(srv.submit(probe.n, probe.src, probe.dst, 1, 10, True, set_mix, core_mix))
        time.sleep(0.05)
        stop.set()
        th.join()
        for t in others:
            srv.wait(t)
        assert len(others) > 5
    for k in ("E", "V", "rounds", "best_round", "m"):
        assert alone[k] == mixed[k]
    np.testing.assert_array_equal(set_alone, set_mix)
    np.testing.assert_array_equal(core_alone, core_mix)
    _check(alone, c, 1, 10, set_alone, core_alone)


def test_backpressure_budget_and_unknown_ticket():
    g = inputs.er_block(n=2000, m=8000, k=30, p=0.5, seed=2)
    with dsg.Server(max_pending=2, hbm_budget=1 << 20) as srv:
        busy = False
        tickets = []
        for _ in range(200):
            t = srv.submit(g.n, g.src, g.dst, 1, 10)
            if t is None:
                busy = True
                break
            tickets.append(t)
        assert busy  # the queue filled up: DSG_EBUSY
        for t in tickets:
            assert srv.wait(t)["status"] == 0
        big = inputs.rmat(scale=14, m=1 << 18, seed=1)
        with pytest.raises(dsg.DsgError) as ei:
            srv.submit(big.n, big.src, big.dst, 1, 10)  # can never fit the 1 MiB budget
        assert ei.value.status == 1
        with pytest.raises(dsg.DsgError) as ei:
            srv.poll(123456789)
        assert ei.value.status == 7
        assert srv.stats()["rejected"] >= 1


def test_shutdown_with_requests_in_flight():
    pool = _pool(k=8, seed=11)
    srv = dsg.Server(max_batch=4)
    for i in range(40):
        g = pool[i % len(pool)]
        srv.submit(g.n, g.src, g.dst, 1, 10, True)
    srv.close()  # cancels what was not admitted, finishes the rest, frees everything
    # the device is still usable
    c = oracle.from_raw(pool[0])
    gr = dsg.Graph.from_edges(pool[0].n, pool[0].src, pool[0].dst)
    _, E, V = gr.bahmani(1, 10)
    want = oracle.bahmani(c, 1, 10)
    assert (E, V) == (want.E, want.V)


def test_full_size_pool_requests_match_the_oracle_with_sets_and_cores():
    """Requests drawn as in the serving workload (pool graphs of n up to
    2,000,000, seeds 7,000,000 + i; eps 1/100 or 1/10; core numbers on half of
    them), including the largest pool member of the first 256, submitted as a
    burst: every result -- (E, V), rounds, best round, the set and the core
    numbers when asked -- equals the oracle's for that (graph, eps)."""
    ns = np.array([inputs.batch_n(i, seed_base=7_000_000, n_hi=2_000_000) for i in range(256)])
    rng = np.random.default_rng(7)
    picks = sorted({int(ns.argmax())} | set(int(x) for x in rng.choice(256, 5, replace=False)))
    pool = {i: inputs.batch_graph(i, seed_base=7_000_000, n_hi=2_000_000) for i in picks}
    csrs = {i: oracle.from_raw(g) for i, g in pool.items()}
    cache = {}
    with dsg.Server(max_batch=8) as srv:
        tickets = []
        for r in range(12):
            i = picks[r % len(picks)]
            p, q = [(1, 100), (1, 10)][int(rng.integers(2))]
            want_core = bool(rng.random() < 0.5)
            g = pool[i]
            out_set = np.zeros(max(g.n, 1), np.uint8)
            core = np.zeros(max(g.n, 1), np.uint32) if want_core else None
            t = srv.submit(g.n, g.src, g.dst, p, q, want_core, out_set, core)
            assert t is not None
            tickets.append((t, i, p, q, out_set, core))
        for t, i, p, q, out_set, core in tickets:
            resp = srv.wait(t, timeout_s=120)
            key = (i, p, q)
            if key not in cache:
                cache[key] = oracle.bahmani(csrs[i], p, q)
            want = cache[key]
            assert resp["status"] == 0
            assert (resp["E"], resp["V"], resp["rounds"], resp["best_round"]) == \
                (want.E, want.V, want.rounds, want.best_round)
            np.testing.assert_array_equal(out_set[:csrs[i].n], want.mask)
            if core is not None:
                if ("core", i) not in cache:
                    cache[("core", i)] = oracle.kcore_bz(csrs[i])
                np.testing.assert_array_equal(core[:csrs[i].n], cache[("core", i)])
