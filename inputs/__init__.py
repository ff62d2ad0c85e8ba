"""Seeded synthetic graph inputs shared by the oracle, the tests and the bench.

This module produces raw undirected edge pairs (numpy ``uint32`` arrays
``src``/``dst``) and nothing else: it holds none of the densest-subgraph
method's arithmetic.  Self-loops, duplicate pairs and both orientations may
appear; each side canonicalises them with its own ingest step.

The heavy generators live in ``gen.c`` (SplitMix64 counter streams, threaded,
identical bytes for any thread count).  ``build()`` compiles it with gcc.

Workloads (stand-ins for the SNAP social/web graphs of the paper's Table 1,
which are not available here):

* ``er_block``   Erdos-Renyi G(n, m) without replacement plus a planted block
* ``rmat``       R-MAT (a, b, c, d) over 2^scale vertices
* ``chung_lu``   Chung-Lu power law, endpoints drawn proportional to weights
* ``batch_graph`` one member of the uneven batch (ER or Chung-Lu + block)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdsg_inputs.so")
_lib = None

_U32P = ctypes.POINTER(ctypes.c_uint32)
_F64P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (gcc, -O2, no FP contraction)."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                           src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gen_er.restype = ctypes.c_uint64
        lib.gen_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _U32P, _U32P]
        lib.gen_block.restype = ctypes.c_uint64
        lib.gen_block.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, _U32P, _U32P,
                                  ctypes.c_uint64]
        lib.gen_rmat.restype = None
        lib.gen_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_uint64, _U32P, _U32P, ctypes.c_int]
        lib.gen_chung_lu.restype = ctypes.c_int
        lib.gen_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, _U32P, _U32P, ctypes.c_int]
        lib.gen_chung_lu_weights.restype = ctypes.c_int
        lib.gen_chung_lu_weights.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             _F64P]
        lib.gen_er_pairs.restype = None
        lib.gen_er_pairs.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _U32P, _U32P, ctypes.c_int]
        lib.gen_draw.restype = ctypes.c_uint64
        lib.gen_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_U32P)


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


@dataclass
class RawGraph:
    """Raw edge pairs over vertices 0..n-1 (may hold loops and duplicates)."""
    n: int
    src: np.ndarray
    dst: np.ndarray
    name: str = ""

    @property
    def m_raw(self) -> int:
        return int(self.src.shape[0])


def er(n: int, m: int, seed: int) -> RawGraph:
    lib = _load()
    src = np.empty(max(m, 1), np.uint32)
    dst = np.empty(max(m, 1), np.uint32)
    got = lib.gen_er(n, m, seed, _p32(src), _p32(dst))
    return RawGraph(n, src[:got].copy(), dst[:got].copy(), f"er(n={n},m={m},seed={seed})")


def er_pairs(n: int, m: int, seed: int, threads: int | None = None) -> RawGraph:
    """m uniform pairs with replacement (loops and repeats dropped at ingest)."""
    lib = _load()
    src = np.empty(max(m, 1), np.uint32)
    dst = np.empty(max(m, 1), np.uint32)
    lib.gen_er_pairs(n, m, seed, _p32(src), _p32(dst), threads or _threads())
    return RawGraph(n, src[:m], dst[:m], f"er_pairs(n={n},m={m},seed={seed})")


def block(n: int, k: int, p: float, seed: int) -> RawGraph:
    lib = _load()
    cap = k * (k - 1) // 2 if k > 1 else 1
    src = np.empty(max(cap, 1), np.uint32)
    dst = np.empty(max(cap, 1), np.uint32)
    got = lib.gen_block(n, k, p, seed, _p32(src), _p32(dst), cap)
    return RawGraph(n, src[:got].copy(), dst[:got].copy(), f"block(n={n},k={k},p={p},seed={seed})")


def union(*gs: RawGraph) -> RawGraph:
    n = max(g.n for g in gs)
    return RawGraph(n, np.concatenate([g.src for g in gs]), np.concatenate([g.dst for g in gs]),
                    "+".join(g.name for g in gs))


def er_block(n: int = 10_000, m: int = 50_000, k: int = 100, p: float = 0.5, seed: int = 0) -> RawGraph:
    """G(n, m) without replacement plus a planted k-block at edge probability p."""
    g = union(er(n, m, seed), block(n, k, p, seed))
    g.name = f"er_block(n={n},m={m},k={k},p={p},seed={seed})"
    return g


def rmat(scale: int = 20, m: int = 1 << 24, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1) -> RawGraph:
    lib = _load()
    src = np.empty(max(m, 1), np.uint32)
    dst = np.empty(max(m, 1), np.uint32)
    lib.gen_rmat(scale, m, a, b, c, seed, _p32(src), _p32(dst), _threads())
    return RawGraph(1 << scale, src[:m], dst[:m], f"rmat(scale={scale},m={m},seed={seed})")


def chung_lu(n: int = 1 << 24, m_draws: int = 1 << 28, gamma: float = 2.1, mean: float = 32.0,
             wmax: float = 1e5, seed: int = 2, threads: int | None = None) -> RawGraph:
    lib = _load()
    src = np.empty(max(m_draws, 1), np.uint32)
    dst = np.empty(max(m_draws, 1), np.uint32)
    if lib.gen_chung_lu(n, m_draws, gamma, mean, wmax, seed, _p32(src), _p32(dst), threads or _threads()) != 0:
        raise MemoryError("chung_lu: host allocation failed")
    return RawGraph(n, src[:m_draws], dst[:m_draws], f"chung_lu(n={n},m={m_draws},gamma={gamma},seed={seed})")


def chung_lu_weights(n: int, gamma: float, mean: float, wmax: float) -> np.ndarray:
    lib = _load()
    w = np.empty(max(n, 1), np.float64)
    lib.gen_chung_lu_weights(n, gamma, mean, wmax, w.ctypes.data_as(_F64P))
    return w[:n]


def batch_n(i: int, seed_base: int = 1000, n_lo: int = 1_000, n_hi: int = 1_000_000) -> int:
    """Vertex count of batch member i (log-uniform in [n_lo, n_hi]), without generating it."""
    lib = _load()
    u = (lib.gen_draw(seed_base + i, 7, 0) >> 11) * 2.0 ** -53
    n = int(math.floor(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
    return max(n_lo, min(n_hi, n))


def batch_graph(i: int, seed_base: int = 1000, n_lo: int = 1_000, n_hi: int = 1_000_000,
                threads: int | None = None) -> RawGraph:
    """Member i of the uneven batch: n log-uniform in [n_lo, n_hi]; even i is
    Erdos-Renyi with mean degree 8 (4n uniform pairs), odd i is Chung-Lu
    (exponent 2.3, mean degree 16, structural cut-off sqrt(16 n)); each gets a
    planted block of floor(sqrt(n)) vertices at edge probability 0.3."""
    seed = seed_base + i
    n = batch_n(i, seed_base, n_lo, n_hi)
    k = int(math.isqrt(n))
    if i % 2 == 0:
        base = er_pairs(n, 4 * n, seed, threads)
    else:
        base = chung_lu(n, 8 * n, 2.3, 16.0, 0.0, seed, threads)
    g = union(base, block(n, k, 0.3, seed))
    g.name = f"batch[{i}](n={n},{'er' if i % 2 == 0 else 'cl'})"
    return g


# ----------------------------------------------------------------- small shapes
def from_pairs(n: int, pairs, name: str = "") -> RawGraph:
    arr = np.asarray(list(pairs), dtype=np.uint32).reshape(-1, 2)
    return RawGraph(n, arr[:, 0].copy(), arr[:, 1].copy(), name)


def complete(n: int) -> RawGraph:
    return from_pairs(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def star(s: int) -> RawGraph:
    return from_pairs(s + 1, [(0, j) for j in range(1, s + 1)], f"star{s}")


def path(n: int) -> RawGraph:
    return from_pairs(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def cycle(n: int) -> RawGraph:
    return from_pairs(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def disjoint_cliques(sizes) -> RawGraph:
    pairs, base = [], 0
    for s in sizes:
        pairs += [(base + i, base + j) for i in range(s) for j in range(i + 1, s)]
        base += s
    return from_pairs(base, pairs, f"cliques{tuple(sizes)}")


def empty(n: int) -> RawGraph:
    return RawGraph(n, np.zeros(0, np.uint32), np.zeros(0, np.uint32), f"empty{n}")


def random_small(n: int, p: float, seed: int) -> RawGraph:
    """Dense-ish random graph for brute-force checks; numpy RNG is fine here."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    return RawGraph(n, iu[keep].astype(np.uint32), ju[keep].astype(np.uint32), f"gnp({n},{p},{seed})")


def onion(n: int = 1 << 20, d: int = 64, core: int = 160) -> RawGraph:
    """Nested shells around a clique: shell 0 is K_core; every vertex of shell
    i >= 1 has d edges into shell i - 1, spread evenly (vertex j of the shell
    to vertices (j d + t) mod |shell i-1|, t < d), and each shell is
    ceil((d+1)/d) times the one inside it, so every inner vertex gets at
    least d + 1 edges from outside.  Shells are added until at least n
    vertices exist.  Deterministic (no seed).  With eps < 1/(2d) a round of
    the (2+2eps) peel removes exactly the outermost shell (degree d, while
    every vertex inside has at least 2d + 1 until its outer shell is gone),
    so the peel takes about one round per shell: a long tail of rounds that
    each remove a few percent of the survivors."""
    sizes = [core]
    while sum(sizes) < n:
        sizes.append(-(-sizes[-1] * (d + 1) // d))
    base = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    iu, ju = np.triu_indices(core, 1)
    src, dst = [iu.astype(np.uint32)], [ju.astype(np.uint32)]
    for i in range(1, len(sizes)):
        j = np.repeat(np.arange(sizes[i], dtype=np.int64), d)
        t = np.tile(np.arange(d, dtype=np.int64), sizes[i])
        src.append((base[i] + j).astype(np.uint32))
        dst.append((base[i - 1] + (j * d + t) % sizes[i - 1]).astype(np.uint32))
    return RawGraph(int(base[-1]), np.concatenate(src), np.concatenate(dst),
                    f"onion(n={n},d={d},core={core},shells={len(sizes)})")
