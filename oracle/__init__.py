"""ORACLE -- test infrastructure, not product code.

Python face of ``oracle.c``: a plain serial CPU statement of the densest-
subgraph peel (Algorithm 1), core numbers (Def. 2 / Algorithm 2 first phase),
the densest core and Algorithm 2's second phase, plus exact checkers
(subset enumeration, Goldberg min-cut).  It shares no code with the CUDA
library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline leg may import it.

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

_U8P = ctypes.POINTER(ctypes.c_uint8)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_U64P = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    c = ctypes
    lib.orc_canonical_csr.restype = c.c_int64
    lib.orc_canonical_csr.argtypes = [c.c_uint32, c.c_uint64, _U32P, _U32P, _U64P, _U32P]
    for name in ("orc_bahmani", "orc_bahmani_recompute"):
        f = getattr(lib, name)
        f.restype = c.c_int
        f.argtypes = [c.c_uint32, _U64P, _U32P, c.c_uint64, c.c_uint64, _U32P, _U64P, _U64P, c.c_uint64, _U64P]
    for name in ("orc_kcore_bz", "orc_kcore_naive", "orc_kcore_pkc"):
        f = getattr(lib, name)
        f.restype = c.c_int
        f.argtypes = [c.c_uint32, _U64P, _U32P, _U32P]
    lib.orc_densest_core.restype = c.c_int
    lib.orc_densest_core.argtypes = [c.c_uint32, _U64P, _U32P, _U32P, _U64P]
    lib.orc_brute_densest.restype = c.c_int
    lib.orc_brute_densest.argtypes = [c.c_uint32, _U64P, _U32P, _U64P, _U64P]
    lib.orc_goldberg_densest.restype = c.c_int
    lib.orc_goldberg_densest.argtypes = [c.c_uint32, _U64P, _U32P, _U64P, _U8P]
    lib.orc_cbds_phase2.restype = c.c_int
    lib.orc_cbds_phase2.argtypes = [c.c_uint32, _U64P, _U32P, _U32P, c.c_uint64, c.c_uint64, c.c_uint64, _U64P,
                                    _U8P]
    _lib = lib
    return lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


@dataclass
class CSR:
    n: int
    off: np.ndarray  # uint64[n+1]
    adj: np.ndarray  # uint32[off[n]]

    @property
    def m(self) -> int:
        return int(self.off[-1]) // 2


def canonical_csr(n: int, src: np.ndarray, dst: np.ndarray) -> CSR:
    """Drop loops, dedup, symmetrise, sort rows (Def. 1 simple graph)."""
    lib = _load()
    src = np.ascontiguousarray(src, np.uint32)
    dst = np.ascontiguousarray(dst, np.uint32)
    m_raw = int(src.shape[0])
    off = np.zeros(n + 1, np.uint64)
    adj = np.empty(max(2 * m_raw, 1), np.uint32)
    got = lib.orc_canonical_csr(n, m_raw, _p(src, _U32P), _p(dst, _U32P), _p(off, _U64P), _p(adj, _U32P))
    if got < 0:
        raise ValueError("oracle canonical_csr: vertex id out of range or allocation failure")
    return CSR(n, off, adj[:got].copy())


def from_raw(g) -> CSR:
    return canonical_csr(g.n, g.src, g.dst)


def round_bound(n: int, p: int, q: int) -> int:
    """Upper bound on the number of rounds: with E > 0 a round leaves fewer
    than q/(p+q) of the vertices, so at most ceil(log_{(p+q)/q} n) + 1 rounds
    for p > 0; with p = 0 every round still removes at least one vertex."""
    if n == 0:
        return 0
    if p == 0:
        return n
    return int(math.ceil(math.log(n) / math.log((p + q) / q))) + 2


@dataclass
class PeelResult:
    rounds: int
    best_round: int
    E: int
    V: int
    hist_S: np.ndarray
    hist_E: np.ndarray
    peel_round: np.ndarray
    mask: np.ndarray = field(default=None)


def _bahmani(fn, csr: CSR, p: int, q: int) -> PeelResult:
    lib = _load()
    n = csr.n
    cap = round_bound(n, p, q) + 2
    hs = np.zeros(cap, np.uint64)
    he = np.zeros(cap, np.uint64)
    pr = np.zeros(max(n, 1), np.uint32)
    out = np.zeros(4, np.uint64)
    rc = getattr(lib, fn)(n, _p(csr.off, _U64P), _p(csr.adj, _U32P), p, q, _p(pr, _U32P), _p(hs, _U64P),
                          _p(he, _U64P), cap, _p(out, _U64P))
    if rc != 0:
        raise RuntimeError(f"oracle {fn} failed with {rc}")
    R, br = int(out[0]), int(out[1])
    pr = pr[:n]
    return PeelResult(R, br, int(out[2]), int(out[3]), hs[:R + 1].copy(), he[:R + 1].copy(), pr,
                      (pr > br).astype(np.uint8))


def bahmani(csr: CSR, p: int, q: int) -> PeelResult:
    """Algorithm 1 with eps = p/q (incremental serial statement)."""
    return _bahmani("orc_bahmani", csr, p, q)


def bahmani_recompute(csr: CSR, p: int, q: int) -> PeelResult:
    """Algorithm 1 recomputing induced degrees and |E(S)| every round."""
    return _bahmani("orc_bahmani_recompute", csr, p, q)


def _kcore(fn, csr: CSR) -> np.ndarray:
    lib = _load()
    core = np.zeros(max(csr.n, 1), np.uint32)
    rc = getattr(lib, fn)(csr.n, _p(csr.off, _U64P), _p(csr.adj, _U32P), _p(core, _U32P))
    if rc != 0:
        raise RuntimeError(f"oracle {fn} failed with {rc}")
    return core[:csr.n]


def kcore_bz(csr: CSR) -> np.ndarray:
    return _kcore("orc_kcore_bz", csr)


def kcore_naive(csr: CSR) -> np.ndarray:
    return _kcore("orc_kcore_naive", csr)


def kcore_pkc(csr: CSR) -> np.ndarray:
    return _kcore("orc_kcore_pkc", csr)


def densest_core(csr: CSR, core: np.ndarray):
    """(k*, E_k*, V_k*) of the densest k-core."""
    lib = _load()
    core = np.ascontiguousarray(core, np.uint32)
    out = np.zeros(3, np.uint64)
    lib.orc_densest_core(csr.n, _p(csr.off, _U64P), _p(csr.adj, _U32P), _p(core, _U32P), _p(out, _U64P))
    return int(out[0]), int(out[1]), int(out[2])


def cbds_phase2(csr: CSR, core: np.ndarray, kstar: int, Ek: int, Vk: int):
    """Algorithm 2 second phase: (m_e, m_v, n_legit, legit_mask)."""
    lib = _load()
    core = np.ascontiguousarray(core, np.uint32)
    out = np.zeros(3, np.uint64)
    mask = np.zeros(max(csr.n, 1), np.uint8)
    rc = lib.orc_cbds_phase2(csr.n, _p(csr.off, _U64P), _p(csr.adj, _U32P), _p(core, _U32P), kstar, Ek, Vk,
                             _p(out, _U64P), _p(mask, _U8P))
    if rc != 0:
        raise RuntimeError("oracle cbds_phase2 failed")
    return int(out[0]), int(out[1]), int(out[2]), mask[:csr.n]


def brute_densest(csr: CSR):
    """Exact (E*, V*, mask) by subset enumeration, n <= 24."""
    lib = _load()
    out = np.zeros(2, np.uint64)
    mask = np.zeros(1, np.uint64)
    rc = lib.orc_brute_densest(csr.n, _p(csr.off, _U64P), _p(csr.adj, _U32P), _p(out, _U64P), _p(mask, _U64P))
    if rc != 0:
        raise ValueError("brute_densest: n too large")
    return int(out[0]), int(out[1]), int(mask[0])


def goldberg_densest(csr: CSR):
    """Exact (E*, V*, mask) by Goldberg's min-cut construction."""
    lib = _load()
    out = np.zeros(2, np.uint64)
    mask = np.zeros(max(csr.n, 1), np.uint8)
    rc = lib.orc_goldberg_densest(csr.n, _p(csr.off, _U64P), _p(csr.adj, _U32P), _p(out, _U64P), _p(mask, _U8P))
    if rc != 0:
        raise RuntimeError("goldberg_densest failed")
    return int(out[0]), int(out[1]), mask[:csr.n]
