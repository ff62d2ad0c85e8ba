"""ctypes binding of libdsg (include/dsg.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
arrays / torch tensors into pointers and status codes into exceptions.  It
never falls back to anything else: if libdsg.so is missing or fails to load,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

c = ctypes
_U8P = c.POINTER(c.c_uint8)
_U32P = c.POINTER(c.c_uint32)
_U64P = c.POINTER(c.c_uint64)
_VP = c.c_void_p

DSG_OK, DSG_EINVAL, DSG_ENOMEM, DSG_ECUDA, DSG_ETIMEOUT, DSG_EBUSY, DSG_EAGAIN, DSG_ENOTFOUND, DSG_EOVERFLOW = range(9)
DSG_CSR_CANONICALIZE = 0x1
DSG_CSR_VALIDATE = 0x2
DSG_PTRS_DEVICE = 0x4
DSG_REQ_BORROW = 0x1


class DsgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Trace(c.Structure):
    _fields_ = [("rounds", c.c_uint64), ("best_round", c.c_uint64), ("best_E", c.c_uint64),
                ("best_V", c.c_uint64), ("hist_cap", c.c_uint64), ("hist_S", _VP), ("hist_E", _VP),
                ("peel_round", _VP), ("out_set", _VP), ("edges_scanned", c.c_uint64), ("decrements", c.c_uint64),
                ("tested", c.c_uint64), ("lazy_rounds", c.c_uint64)]


class Batch(c.Structure):
    _fields_ = [("num_graphs", c.c_uint32), ("vtx_base", _VP), ("off", _VP), ("adj", _VP), ("eps_num", _VP),
                ("eps_den", _VP), ("want_core", _VP)]


class BatchResult(c.Structure):
    _fields_ = [("E", _VP), ("V", _VP), ("rounds", _VP), ("best_round", _VP), ("out_set", _VP), ("core", _VP),
                ("stats", _VP)]


class ServeConfig(c.Structure):
    _fields_ = [("max_batch", c.c_uint32), ("max_pending", c.c_uint32), ("hbm_budget", c.c_uint64),
                ("max_inflight", c.c_uint32), ("ingest_threads", c.c_uint32), ("big_work", c.c_uint64),
                ("big_sms", c.c_uint32), ("max_batch_work", c.c_uint64), ("big_threads", c.c_uint32)]


class Request(c.Structure):
    _fields_ = [("n", c.c_uint32), ("m_raw", c.c_uint64), ("src", _VP), ("dst", _VP), ("eps_num", c.c_uint32),
                ("eps_den", c.c_uint32), ("want_core", c.c_uint32), ("flags", c.c_uint32), ("out_set", _VP),
                ("core", _VP)]


class Response(c.Structure):
    _fields_ = [("status", c.c_int), ("n", c.c_uint32), ("m", c.c_uint64), ("E", c.c_uint64), ("V", c.c_uint64),
                ("rounds", c.c_uint64), ("best_round", c.c_uint64), ("latency_us", c.c_double)]


class ServeStats(c.Structure):
    _fields_ = [("submitted", c.c_uint64), ("admitted", c.c_uint64), ("completed", c.c_uint64),
                ("rejected", c.c_uint64), ("pending", c.c_uint64), ("in_flight", c.c_uint64),
                ("batches", c.c_uint64), ("hbm_in_use", c.c_uint64), ("hbm_budget", c.c_uint64),
                ("p50_us", c.c_double), ("p99_us", c.c_double), ("graphs_per_s", c.c_double),
                ("uptime_s", c.c_double), ("big_done", c.c_uint64), ("ingest_busy_s", c.c_double),
                ("big_busy_s", c.c_double), ("batch_device_s", c.c_double)]


class CbdsResult(c.Structure):
    _fields_ = [("k_star", c.c_uint64), ("E_core", c.c_uint64), ("V_core", c.c_uint64), ("E", c.c_uint64),
                ("V", c.c_uint64), ("n_legit", c.c_uint64)]


ALLOC_FN = c.CFUNCTYPE(c.c_void_p, c.c_size_t, c.c_void_p, c.c_void_p)
FREE_FN = c.CFUNCTYPE(None, c.c_void_p, c.c_void_p, c.c_void_p)

_LIB = None

# (name, restype, argtypes)
_SIGS = [
    ("dsg_graph_from_csr", c.c_int, [c.c_uint32, _VP, _VP, c.c_uint32, _VP, c.POINTER(_VP)]),
    ("dsg_graph_from_edges", c.c_int, [c.c_uint32, c.c_uint64, _VP, _VP, c.c_uint32, _VP, c.POINTER(_VP)]),
    ("dsg_graph_info", c.c_int, [_VP, _U32P, _U64P]),
    ("dsg_graph_csr", c.c_int, [_VP, _VP, _VP]),
    ("dsg_graph_set_stream", c.c_int, [_VP, _VP]),
    ("dsg_graph_free", None, [_VP]),
    ("dsg_bahmani", c.c_int, [_VP, c.c_uint32, c.c_uint32, _VP, _U64P, _U64P]),
    ("dsg_bahmani_trace", c.c_int, [_VP, c.c_uint32, c.c_uint32, c.POINTER(Trace)]),
    ("dsg_round_bound", c.c_uint64, [c.c_uint32, c.c_uint32, c.c_uint32]),
    ("dsg_bahmani_noalloc", c.c_int, [c.c_uint32, _VP, _VP, c.c_uint32, c.c_uint32, _VP, _U64P, _U64P, _VP]),
    ("dsg_peel_begin", c.c_int, [_VP, c.c_uint32, c.c_uint32, c.POINTER(_VP)]),
    ("dsg_peel_advance", c.c_int, [_VP, c.c_uint32, _U64P, _U32P]),
    ("dsg_peel_snapshot_size", c.c_int, [_VP, _U64P]),
    ("dsg_peel_snapshot", c.c_int, [_VP, _VP, c.c_uint64]),
    ("dsg_peel_resume", c.c_int, [_VP, _VP, c.c_uint64, c.POINTER(_VP)]),
    ("dsg_peel_finish", c.c_int, [_VP, _VP, _U64P, _U64P, _U64P, _VP, _VP, c.c_uint64]),
    ("dsg_peel_free", None, [_VP]),
    ("dsg_kcore", c.c_int, [_VP, _VP]),
    ("dsg_densest_core", c.c_int, [_VP, _VP, _VP, _VP, c.POINTER(CbdsResult)]),
    ("dsg_cbds", c.c_int, [_VP, _VP, _VP, _VP, c.POINTER(CbdsResult)]),
    ("dsg_batch_solve", c.c_int, [c.POINTER(Batch), c.POINTER(BatchResult), _VP]),
    ("dsg_batch_autotune", c.c_int, [c.POINTER(Batch), _U32P]),
    ("dsg_serve_create", c.c_int, [c.POINTER(ServeConfig), c.POINTER(_VP)]),
    ("dsg_serve_submit", c.c_int, [_VP, c.POINTER(Request), _U64P]),
    ("dsg_serve_poll", c.c_int, [_VP, c.c_uint64, c.POINTER(Response), c.c_uint32]),
    ("dsg_serve_stats", c.c_int, [_VP, c.POINTER(ServeStats)]),
    ("dsg_serve_destroy", None, [_VP]),
    ("dsg_kcore_stats", c.c_int, [_VP, _VP, _U64P, c.c_uint32]),
    ("dsg_set_tuning", c.c_int, [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32]),
    ("dsg_get_tuning", c.c_int, [_U32P, _U32P, _U32P, _U32P]),
    ("dsg_set_hot_degree", c.c_int, [c.c_uint32]),
    ("dsg_set_local_max", c.c_int, [c.c_uint32, c.c_uint32]),
    ("dsg_set_wait_limit_ns", None, [c.c_uint64]),
    ("dsg_autotune", c.c_int, [_VP, c.c_uint32, c.c_uint32, c.c_uint32, _U32P]),
    ("dsg_tune_save", c.c_int, [c.c_char_p]),
    ("dsg_tune_load", c.c_int, [c.c_char_p, _U32P]),
    ("dsg_tune_clear", None, []),
    ("dsg_tune_entries", c.c_uint32, []),
    ("dsg_tune_lookup", c.c_int, [_VP, c.c_uint32, _U32P]),
    ("dsg_graph_set_max_blocks", c.c_int, [_VP, c.c_uint32]),
    ("dsg_graph_view", c.c_int, [_VP, _VP, c.POINTER(_VP)]),
    ("dsg_solve", c.c_int, [_VP, c.c_uint32, _U32P, _U32P, c.POINTER(_VP), _U64P, _U64P, _VP]),
    ("dsg_set_inline_max", c.c_int, [c.c_uint32]),
    ("dsg_set_kcore_tail", c.c_int, [c.c_uint32]),
    ("dsg_set_batch_split", c.c_int, [c.c_uint32]),
    ("dsg_set_peel_lazy", c.c_int, [c.c_uint32]),
    ("dsg_set_peel_vec", c.c_int, [c.c_uint32]),
    ("dsg_set_allocator", None, [ALLOC_FN, FREE_FN, _VP]),
    ("dsg_debug_wait_timeout", c.c_int, [c.c_uint32, c.c_uint64]),
    ("dsg_debug_peel_trace", c.c_int, [_VP, c.c_uint32, c.c_uint32, _U64P, c.c_uint64, _U64P]),
    ("dsg_debug_kcore_trace", c.c_int, [_VP, _U64P, c.c_uint64, _U64P]),
    ("dsg_launch_count", c.c_ulonglong, []),
    ("dsg_profile_enable", None, [c.c_int]),
    ("dsg_profile_reset", None, []),
    ("dsg_profile_report", c.c_int, [c.c_char_p, c.c_size_t]),
    ("dsg_status_string", c.c_char_p, [c.c_int]),
    ("dsg_last_error", c.c_char_p, []),
    ("dsg_version", c.c_char_p, []),
]


def lib_path() -> str:
    return _build.lib_file()


def lib():
    """Load libdsg.so (building it first if sources are newer)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libdsg.so not found at {path}")
        L = c.CDLL(path)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def declared_symbols():
    return [s[0] for s in _SIGS]


def check(status: int, what: str = ""):
    if status != DSG_OK:
        L = lib()
        msg = L.dsg_last_error().decode(errors="replace") or L.dsg_status_string(status).decode()
        raise DsgError(status, f"{what}: {msg}" if what else msg)


def ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def is_device(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def stream_handle(stream):
    """cudaStream_t of a torch.cuda.Stream (or an int handle); None -> default."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def profile_report() -> dict:
    """{kernel: (launches, total_ms)} of the launches timed so far."""
    buf = c.create_string_buffer(1 << 16)
    lib().dsg_profile_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, k, ms = line.split()
        out[name] = (int(k), float(ms))
    return out
