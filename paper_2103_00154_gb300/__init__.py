"""GB300-native densest-subgraph peeling (arXiv 2103.00154 hot path).

Thin Python face of libdsg (see include/dsg.h).  Names follow the C ABI:

    g = Graph.from_edges(n, src, dst)        # dsg_graph_from_edges (ingest)
    g = Graph.from_csr(n, off, adj)          # dsg_graph_from_csr
    mask, E, V = g.bahmani(p, q)             # dsg_bahmani (Algorithm 1)
    tr = g.bahmani_trace(p, q)               # dsg_bahmani_trace
    core = g.kcore()                         # dsg_kcore (Algorithm 2, phase 1)

Inputs and outputs may be numpy arrays (host) or torch tensors (host or
CUDA).  PyTorch is used only for device memory and streams; all work runs in
libdsg's kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native as N
from ._native import (DSG_CSR_CANONICALIZE, DSG_CSR_VALIDATE, DSG_PTRS_DEVICE, DsgError,  # noqa: F401
                      lib)

__all__ = ["Graph", "Trace", "PeelState", "BatchSolver", "pack_batch", "Server", "DsgError", "lib", "round_bound", "set_tuning", "get_tuning", "set_wait_limit_ns",
           "DSG_CSR_CANONICALIZE", "DSG_CSR_VALIDATE", "DSG_PTRS_DEVICE"]


def round_bound(n: int, p: int, q: int) -> int:
    return int(lib().dsg_round_bound(n, p, q))


def set_tuning(block: int = 512, blocks_per_sm: int = 0, short_max: int = 32, chunk_len: int = 256,
               hot_deg: int = 0, local_max: int = 1024, local_work: int = 16384, inline_max: int = 256,
               kcore_tail: int = 65536, batch_split: int = 0, peel_lazy: bool = True, peel_vec: bool = False):
    N.check(lib().dsg_set_tuning(block, blocks_per_sm, short_max, chunk_len), "set_tuning")
    N.check(lib().dsg_set_hot_degree(hot_deg), "set_hot_degree")
    N.check(lib().dsg_set_local_max(local_max, local_work), "set_local_max")
    N.check(lib().dsg_set_inline_max(inline_max), "set_inline_max")
    N.check(lib().dsg_set_kcore_tail(kcore_tail), "set_kcore_tail")
    N.check(lib().dsg_set_batch_split(batch_split), "set_batch_split")
    N.check(lib().dsg_set_peel_lazy(1 if peel_lazy else 0), "set_peel_lazy")
    N.check(lib().dsg_set_peel_vec(1 if peel_vec else 0), "set_peel_vec")


def get_tuning():
    v = [ctypes.c_uint32() for _ in range(4)]
    N.check(lib().dsg_get_tuning(*[ctypes.byref(x) for x in v]), "get_tuning")
    return dict(zip(("block", "blocks_per_sm", "short_max", "chunk_len"), (x.value for x in v)))


def tune_save(path: str):
    N.check(lib().dsg_tune_save(path.encode()), "tune_save")


def tune_load(path: str) -> int:
    k = ctypes.c_uint32()
    N.check(lib().dsg_tune_load(path.encode(), ctypes.byref(k)), "tune_load")
    return k.value


def tune_clear():
    lib().dsg_tune_clear()


def tune_entries() -> int:
    return int(lib().dsg_tune_entries())


_alloc_hooks = None


def use_torch_allocator(on: bool = True):
    """Route every device buffer the library makes through PyTorch's caching
    allocator (dsg_set_allocator), or back to the library's own pool."""
    global _alloc_hooks
    if not on:
        lib().dsg_set_allocator(N.ALLOC_FN(), N.FREE_FN(), None)
        _alloc_hooks = None
        return
    import torch

    def _alloc(nbytes, ctx, stream):
        try:
            return torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:  # out of memory -> NULL -> DSG_ENOMEM
            return None

    def _free(ptr, ctx, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (N.ALLOC_FN(_alloc), N.FREE_FN(_free))
    lib().dsg_set_allocator(hooks[0], hooks[1], None)
    _alloc_hooks = hooks  # keep the callbacks alive


def set_wait_limit_ns(ns: int):
    lib().dsg_set_wait_limit_ns(int(ns))


@dataclass
class Trace:
    rounds: int
    best_round: int
    E: int
    V: int
    hist_S: np.ndarray
    hist_E: np.ndarray
    peel_round: object
    mask: object
    edges_scanned: int
    decrements: int
    tested: int = 0
    lazy_rounds: int = 0


@dataclass
class Cbds:
    """Densest core (k_star, E_core, V_core) and the result (E, V) with its set;
    for dsg_cbds the result is the densest core grown by Algorithm 2's second
    phase (n_legit vertices added), for dsg_densest_core it is the core itself."""
    k_star: int
    E_core: int
    V_core: int
    E: int
    V: int
    n_legit: int
    mask: object
    core: object


def _u32(x):
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x, np.uint32)
    return x


def _u64(x):
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x, np.uint64)
    return x


class Graph:
    """A device-resident canonical graph (handle to dsg_graph)."""

    def __init__(self, handle, keepalive=()):
        self._h = handle
        self._keep = keepalive  # device arrays borrowed with DSG_PTRS_DEVICE
        n = ctypes.c_uint32()
        m = ctypes.c_uint64()
        N.check(lib().dsg_graph_info(self._h, ctypes.byref(n), ctypes.byref(m)), "graph_info")
        self.n = n.value
        self.m = m.value

    # ------------------------------------------------------------ creation
    @classmethod
    def from_csr(cls, n: int, off, adj, flags: int = 0, stream=None) -> "Graph":
        off, adj = _u64(off), _u32(adj)
        h = ctypes.c_void_p()
        keep = ()
        if N.is_device(off):
            flags |= DSG_PTRS_DEVICE if not (flags & DSG_CSR_CANONICALIZE) else 0
            keep = (off, adj)
        N.check(lib().dsg_graph_from_csr(n, N.ptr(off), N.ptr(adj), flags, N.stream_handle(stream),
                                         ctypes.byref(h)), "graph_from_csr")
        return cls(h, keep)

    @classmethod
    def from_edges(cls, n: int, src, dst, flags: int = 0, stream=None) -> "Graph":
        src, dst = _u32(src), _u32(dst)
        m_raw = int(src.shape[0])
        if int(dst.shape[0]) != m_raw:
            raise ValueError("src and dst differ in length")
        if N.is_device(src):
            flags |= DSG_PTRS_DEVICE
        h = ctypes.c_void_p()
        N.check(lib().dsg_graph_from_edges(n, m_raw, N.ptr(src) if m_raw else None, N.ptr(dst) if m_raw else None,
                                           flags, N.stream_handle(stream), ctypes.byref(h)), "graph_from_edges")
        return cls(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().dsg_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        N.check(lib().dsg_graph_set_stream(self._h, N.stream_handle(stream)), "set_stream")

    # ------------------------------------------------------------ queries
    def csr(self):
        off = np.empty(self.n + 1, np.uint64)
        adj = np.empty(max(2 * self.m, 1), np.uint32)
        N.check(lib().dsg_graph_csr(self._h, N.ptr(off), N.ptr(adj)), "graph_csr")
        return off, adj[:2 * self.m]

    def bahmani(self, p: int, q: int, out_set=None, want_set: bool = True):
        """Algorithm 1 with eps = p/q.  Returns (mask, E, V)."""
        if want_set and out_set is None:
            out_set = np.empty(max(self.n, 1), np.uint8)
        E = ctypes.c_uint64()
        V = ctypes.c_uint64()
        N.check(lib().dsg_bahmani(self._h, p, q, N.ptr(out_set) if want_set else None, ctypes.byref(E),
                                  ctypes.byref(V)), "bahmani")
        if isinstance(out_set, np.ndarray):
            out_set = out_set[:self.n]
        return out_set, E.value, V.value

    def bahmani_trace(self, p: int, q: int, hist_cap: int | None = None, peel_round=None, out_set=None) -> Trace:
        if hist_cap is None:
            hist_cap = round_bound(self.n, p, q) + 1
        hs = np.zeros(max(hist_cap, 1), np.uint64)
        he = np.zeros(max(hist_cap, 1), np.uint64)
        if peel_round is None:
            peel_round = np.zeros(max(self.n, 1), np.uint32)
        if out_set is None:
            out_set = np.zeros(max(self.n, 1), np.uint8)
        t = N.Trace(0, 0, 0, 0, hist_cap, N.ptr(hs), N.ptr(he), N.ptr(peel_round), N.ptr(out_set), 0, 0, 0, 0)
        N.check(lib().dsg_bahmani_trace(self._h, p, q, ctypes.byref(t)), "bahmani_trace")
        R = t.rounds
        if isinstance(peel_round, np.ndarray):
            peel_round = peel_round[:self.n]
        if isinstance(out_set, np.ndarray):
            out_set = out_set[:self.n]
        return Trace(R, t.best_round, t.best_E, t.best_V, hs[:R + 1].copy(), he[:R + 1].copy(), peel_round,
                     out_set, t.edges_scanned, t.decrements, t.tested, t.lazy_rounds)

    def autotune(self, p: int = 1, q: int = 10, peel: bool = True, kcore: bool = True) -> int:
        """Pick launch parameters for this graph's size class (dsg_autotune);
        returns the number of timed solves."""
        t = ctypes.c_uint32()
        N.check(lib().dsg_autotune(self._h, p, q, (1 if peel else 0) | (2 if kcore else 0), ctypes.byref(t)),
                "autotune")
        return t.value

    def _cbds(self, fn, what, core, out_core, out_set, want_set, want_core):
        if want_set and out_set is None:
            out_set = np.empty(max(self.n, 1), np.uint8)
        if want_core and out_core is None and core is None:
            out_core = np.empty(max(self.n, 1), np.uint32)
        r = N.CbdsResult()
        N.check(fn(self._h, N.ptr(_u32(core)), N.ptr(out_core), N.ptr(out_set) if want_set else None,
                   ctypes.byref(r)), what)
        if isinstance(out_set, np.ndarray):
            out_set = out_set[:self.n]
        if isinstance(out_core, np.ndarray):
            out_core = out_core[:self.n]
        return Cbds(r.k_star, r.E_core, r.V_core, r.E, r.V, r.n_legit, out_set if want_set else None,
                    out_core if out_core is not None else core)

    def densest_core(self, core=None, out_core=None, out_set=None, want_set: bool = True,
                     want_core: bool = True) -> Cbds:
        """Densest k-core (Sec. 3.2).  `core` (optional) replaces the core numbers."""
        return self._cbds(lib().dsg_densest_core, "densest_core", core, out_core, out_set, want_set, want_core)

    def cbds(self, core=None, out_core=None, out_set=None, want_set: bool = True, want_core: bool = True) -> Cbds:
        """CBDS-P (Algorithm 2): densest core plus the second phase's legit vertices."""
        return self._cbds(lib().dsg_cbds, "cbds", core, out_core, out_set, want_set, want_core)

    def solve(self, eps, out_sets=None, out_core=None, want_sets: bool = True, want_core: bool = True):
        """dsg_solve: Bahmani peels at every (p, q) in eps plus the core numbers,
        side by side on the GPU.  Returns ([(mask, E, V), ...], core)."""
        k = len(eps)
        pn = (ctypes.c_uint32 * max(k, 1))(*[p for p, _ in eps])
        qn = (ctypes.c_uint32 * max(k, 1))(*[q for _, q in eps])
        if want_sets and out_sets is None:
            out_sets = [np.empty(max(self.n, 1), np.uint8) for _ in range(k)]
        sets = (ctypes.c_void_p * max(k, 1))(*([N.ptr(x) for x in out_sets] if want_sets else [None] * k))
        if want_core and out_core is None:
            out_core = np.empty(max(self.n, 1), np.uint32)
        E = np.zeros(max(k, 1), np.uint64)
        V = np.zeros(max(k, 1), np.uint64)
        N.check(lib().dsg_solve(self._h, k, pn, qn, sets, E.ctypes.data_as(N._U64P), V.ctypes.data_as(N._U64P),
                                N.ptr(out_core) if want_core else None), "solve")
        res = []
        for i in range(k):
            m = out_sets[i] if want_sets else None
            if isinstance(m, np.ndarray):
                m = m[:self.n]
            res.append((m, int(E[i]), int(V[i])))
        if isinstance(out_core, np.ndarray):
            out_core = out_core[:self.n]
        return res, (out_core if want_core else None)

    def view(self, stream=None) -> "Graph":
        """A second handle over this graph's device CSR on `stream` (close it
        before this graph)."""
        h = ctypes.c_void_p()
        N.check(lib().dsg_graph_view(self._h, N.stream_handle(stream), ctypes.byref(h)), "graph_view")
        return Graph(h, keepalive=(self,))

    def set_max_blocks(self, max_blocks: int):
        """Cap the grid of this handle's persistent kernels (0: whole GPU), so
        solves on two handles can share the GPU from two streams."""
        N.check(lib().dsg_graph_set_max_blocks(self._h, int(max_blocks)), "set_max_blocks")

    def tuning(self, kernel: str = "peel") -> dict:
        """Launch parameters a solve of `kernel` ("peel" or "kcore") on this graph uses now."""
        v = (ctypes.c_uint32 * 9)()
        N.check(lib().dsg_tune_lookup(self._h, 0 if kernel == "peel" else 1, v), "tune_lookup")
        return dict(zip(("block", "blocks_per_sm", "short_max", "chunk_len", "hot_deg", "local_max", "local_work",
                         "inline_max", "kcore_tail"), list(v)))

    def kcore(self, out=None):
        """Core numbers (Algorithm 2, first phase)."""
        if out is None:
            out = np.empty(max(self.n, 1), np.uint32)
        N.check(lib().dsg_kcore(self._h, N.ptr(out)), "kcore")
        if isinstance(out, np.ndarray):
            out = out[:self.n]
        return out

    def kcore_counters(self, out=None):
        """Core numbers plus the run's counters: levels, pieces (queued row pieces),
        rem_scanned, rem_written, atomics."""
        if out is None:
            out = np.empty(max(self.n, 1), np.uint32)
        st = np.zeros(5, np.uint64)
        N.check(lib().dsg_kcore_stats(self._h, N.ptr(out), st.ctypes.data_as(N._U64P), 5), "kcore_stats")
        if isinstance(out, np.ndarray):
            out = out[:self.n]
        keys = ("levels", "pieces", "rem_scanned", "rem_written", "atomics")
        return out, {k: int(v) for k, v in zip(keys, st)}


class PeelState:
    """A paused Algorithm 1 peel (dsg_peel_*): advance it some rounds, write a
    snapshot (bytes), resume it from one on a handle of the same graph, or
    finish it.  Finishing gives exactly dsg_bahmani's result."""

    def __init__(self, handle, graph, p: int, q: int):
        self._h = handle
        self._graph = graph  # the graph must outlive the state
        self.p, self.q = p, q

    @classmethod
    def begin(cls, graph: "Graph", p: int, q: int) -> "PeelState":
        h = ctypes.c_void_p()
        N.check(lib().dsg_peel_begin(graph._h, p, q, ctypes.byref(h)), "peel_begin")
        return cls(h, graph, p, q)

    @classmethod
    def resume(cls, graph: "Graph", snap: bytes) -> "PeelState":
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(bytes(snap), len(snap))
        N.check(lib().dsg_peel_resume(graph._h, buf, len(snap), ctypes.byref(h)), "peel_resume")
        hdr = np.frombuffer(bytes(snap)[:128], np.uint64)
        return cls(h, graph, int(hdr[4]), int(hdr[5]))

    def advance(self, max_rounds: int = 0):
        """Run at most max_rounds more rounds (0: to the end); returns (rounds so far, done)."""
        r = ctypes.c_uint64()
        d = ctypes.c_uint32()
        N.check(lib().dsg_peel_advance(self._h, int(max_rounds), ctypes.byref(r), ctypes.byref(d)), "peel_advance")
        return int(r.value), bool(d.value)

    def snapshot(self) -> bytes:
        size = ctypes.c_uint64()
        N.check(lib().dsg_peel_snapshot_size(self._h, ctypes.byref(size)), "peel_snapshot_size")
        buf = ctypes.create_string_buffer(int(size.value))
        N.check(lib().dsg_peel_snapshot(self._h, buf, size.value), "peel_snapshot")
        return buf.raw

    def finish(self, out_set=None, want_set: bool = True) -> Trace:
        n = self._graph.n
        if out_set is None and want_set:
            out_set = np.zeros(max(n, 1), np.uint8)
        cap = round_bound(n, self.p, self.q) + 1
        hs = np.zeros(cap, np.uint64)
        he = np.zeros(cap, np.uint64)
        E, V, R = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        N.check(lib().dsg_peel_finish(self._h, N.ptr(out_set), ctypes.byref(E), ctypes.byref(V), ctypes.byref(R),
                                      N.ptr(hs), N.ptr(he), cap), "peel_finish")
        k = int(R.value) + 1
        mask = out_set[:n] if isinstance(out_set, np.ndarray) else out_set
        return Trace(int(R.value), -1, int(E.value), int(V.value), hs[:k], he[:k], None, mask, 2 * self._graph.m, 0)

    def close(self):
        if self._h:
            lib().dsg_peel_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches
def pack_batch(graphs, device=None):
    """Concatenated CSR of several graphs (dsg_batch layout): returns
    (vtx_base, off, adj) as numpy arrays, or torch tensors on `device` when
    given.  `graphs` are Graph objects or (off, adj) numpy pairs."""
    offs, adjs = [], []
    for g in graphs:
        o, a = g.csr() if isinstance(g, Graph) else g
        offs.append(np.asarray(o, np.uint64))
        adjs.append(np.asarray(a, np.uint32))
    ns = [len(o) - 1 for o in offs]
    vtx_base = np.zeros(len(graphs) + 1, np.uint64)
    vtx_base[1:] = np.cumsum(ns)
    base = 0
    parts = []
    for o in offs:
        parts.append(o[:-1] + np.uint64(base))
        base += int(o[-1])
    parts.append(np.array([base], np.uint64))
    off = np.concatenate(parts) if parts else np.zeros(1, np.uint64)
    adj = np.concatenate(adjs) if adjs else np.zeros(0, np.uint32)
    if device is not None:
        import torch
        return (torch.from_numpy(vtx_base.view(np.int64)).to(device), torch.from_numpy(off.view(np.int64)).to(device),
                torch.from_numpy(adj.view(np.int32) if adj.size else np.zeros(1, np.int32)).to(device))
    return vtx_base, off, adj


class BatchSolver:
    """dsg_batch_solve over a packed batch (see pack_batch)."""

    def __init__(self, vtx_base, off, adj, eps, want_core=None):
        self.vtx_base, self.off, self.adj = vtx_base, off, adj
        self.G = int(vtx_base.shape[0]) - 1
        self.N = int(vtx_base[-1])
        e = np.asarray(eps, np.uint32).reshape(-1, 2)
        if e.shape[0] == 1 and self.G > 1:
            e = np.repeat(e, self.G, axis=0)
        self.p = np.ascontiguousarray(e[:, 0])
        self.q = np.ascontiguousarray(e[:, 1])
        self.want_core = None if want_core is None else np.ascontiguousarray(want_core, np.uint8)

    def _batch(self):
        return N.Batch(self.G, N.ptr(self.vtx_base), N.ptr(self.off), N.ptr(self.adj), N.ptr(self.p), N.ptr(self.q),
                       N.ptr(self.want_core))

    def solve(self, out_set=None, core=None, stream=None, stats=None):
        """(E, V, R, best_round) per graph; stats (numpy uint64[4], optional)
        receives the batch's byte-model counters (see dsg_batch_result)."""
        G = self.G
        E = np.zeros(max(G, 1), np.uint64)
        V = np.zeros(max(G, 1), np.uint64)
        R = np.zeros(max(G, 1), np.uint64)
        BR = np.zeros(max(G, 1), np.uint64)
        b = self._batch()
        r = N.BatchResult(N.ptr(E), N.ptr(V), N.ptr(R), N.ptr(BR), N.ptr(out_set), N.ptr(core), N.ptr(stats))
        N.check(lib().dsg_batch_solve(ctypes.byref(b), ctypes.byref(r), N.stream_handle(stream)), "batch_solve")
        return E[:G], V[:G], R[:G], BR[:G]

    def autotune(self) -> int:
        """dsg_batch_autotune on this batch; returns the number of timed solves."""
        t = ctypes.c_uint32()
        b = self._batch()
        N.check(lib().dsg_batch_autotune(ctypes.byref(b), ctypes.byref(t)), "batch_autotune")
        return int(t.value)


# ------------------------------------------------------------------ serving
class Server:
    """Continuous-batching server (dsg_serve_*).  submit() returns a ticket;
    poll() returns a dict of the request's results or None while pending."""

    def __init__(self, max_batch: int = 0, max_pending: int = 0, hbm_budget: int = 0, max_inflight: int = 0,
                 ingest_threads: int = 0, big_work: int = 0, big_sms: int = 0, max_batch_work: int = 0,
                 big_threads: int = 0):
        cfg = N.ServeConfig(max_batch, max_pending, hbm_budget, max_inflight, ingest_threads, big_work, big_sms,
                            max_batch_work, big_threads)
        h = ctypes.c_void_p()
        N.check(lib().dsg_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "serve_create")
        self._h = h
        self._keep = {}

    def submit(self, n, src, dst, p, q, want_core=False, out_set=None, core=None, borrow=False):
        """Queue a request; None on back-pressure (DSG_EBUSY).  borrow=True:
        src/dst (host, numpy or pinned torch) are read in place and must stay
        unchanged until the request completes."""
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, np.uint32)
            dst = np.ascontiguousarray(dst, np.uint32)
        m_raw = int(src.shape[0])
        r = N.Request(n, m_raw, N.ptr(src), N.ptr(dst), p, q, 1 if want_core else 0,
                      N.DSG_REQ_BORROW if borrow else 0, N.ptr(out_set), N.ptr(core))
        t = ctypes.c_uint64()
        st = lib().dsg_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        if st == N.DSG_EBUSY:
            return None
        N.check(st, "serve_submit")
        self._keep[t.value] = (out_set, core, src, dst)
        return t.value

    def poll(self, ticket, timeout_us: int = 0):
        resp = N.Response()
        st = lib().dsg_serve_poll(self._h, ticket, ctypes.byref(resp), timeout_us)
        if st == N.DSG_EAGAIN:
            return None
        N.check(st, "serve_poll")
        self._keep.pop(ticket, None)
        return {"status": resp.status, "n": resp.n, "m": resp.m, "E": resp.E, "V": resp.V, "rounds": resp.rounds,
                "best_round": resp.best_round, "latency_us": resp.latency_us}

    def wait(self, ticket, timeout_s: float = 60.0):
        import time as _t
        t_end = _t.monotonic() + timeout_s
        while True:
            r = self.poll(ticket, 100_000)
            if r is not None:
                return r
            if _t.monotonic() > t_end:
                raise TimeoutError(f"ticket {ticket} not done after {timeout_s} s")

    def stats(self):
        st = N.ServeStats()
        N.check(lib().dsg_serve_stats(self._h, ctypes.byref(st)), "serve_stats")
        return {f: getattr(st, f) for f, _ in N.ServeStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().dsg_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
