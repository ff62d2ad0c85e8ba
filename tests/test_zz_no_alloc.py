"""dsg_bahmani_noalloc: the peel for callers that cannot allocate device
memory when they run it (their memory belongs to an allocator they do not
own, or their hot path must not call cudaMalloc).  It must give exactly what
dsg_bahmani gives, call after call, although every call reuses the same
fixed scratch buffer.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402
from paper_2103_00154_gb300 import _native as N  # noqa: E402


def _device_csr(c):
    off = torch.from_numpy(c.off.view(np.int64)).cuda()
    adj = torch.from_numpy(c.adj.view(np.int32) if c.adj.size else np.zeros(1, np.int32)).cuda()
    return off, adj


def _noalloc(c, p, q, stream):
    off, adj = _device_csr(c)
    mask = torch.full((max(c.n, 1),), 7, dtype=torch.uint8, device="cuda")
    E = ctypes.c_uint64(123)
    V = ctypes.c_uint64(456)
    st = dsg.lib().dsg_bahmani_noalloc(c.n, off.data_ptr(), adj.data_ptr(), p, q, mask.data_ptr(),
                                       ctypes.byref(E), ctypes.byref(V), stream.cuda_stream)
    assert st == N.DSG_OK, dsg.lib().dsg_last_error()
    return mask[:c.n].cpu().numpy(), E.value, V.value


def _existing(c, p, q):
    g = dsg.Graph.from_csr(c.n, c.off, c.adj)
    mask, E, V = g.bahmani(p, q)
    g.close()
    return mask, E, V


def test_noalloc_matches_dsg_bahmani_on_consecutive_calls():
    stream = torch.cuda.current_stream()
    big = oracle.from_raw(inputs.rmat(scale=16, m=1 << 20, seed=4))
    small = oracle.from_raw(inputs.er_block(n=3000, m=12000, k=50, p=0.5, seed=8))
    # a large graph, then a smaller one over the leftovers, then the large one again
    for c, (p, q) in [(big, (1, 10)), (small, (1, 10)), (big, (1, 1000)), (big, (1, 10)), (small, (0, 1))]:
        got_mask, got_E, got_V = _noalloc(c, p, q, stream)
        want_mask, want_E, want_V = _existing(c, p, q)
        assert (got_E, got_V) == (want_E, want_V)
        np.testing.assert_array_equal(got_mask, want_mask)


def test_noalloc_allocates_no_device_memory():
    """With every library allocation routed through PyTorch's caching
    allocator, repeated calls leave its counters unchanged (the dsg_bahmani
    path, run the same way, does allocate: the check can see allocations)."""
    stream = torch.cuda.current_stream()
    c = oracle.from_raw(inputs.rmat(scale=14, m=1 << 18, seed=9))
    off, adj = _device_csr(c)
    mask = torch.empty(c.n, dtype=torch.uint8, device="cuda")
    E, V = ctypes.c_uint64(), ctypes.c_uint64()
    L = dsg.lib()

    def call():
        st = L.dsg_bahmani_noalloc(c.n, off.data_ptr(), adj.data_ptr(), 1, 10, mask.data_ptr(), ctypes.byref(E),
                                   ctypes.byref(V), stream.cuda_stream)
        assert st == N.DSG_OK, L.dsg_last_error()

    dsg.use_torch_allocator(True)
    try:
        call()  # the first call in this context looks up the buffer's address
        torch.cuda.synchronize()
        before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
        want = oracle.bahmani(c, 1, 10)
        assert (E.value, V.value) == (want.E, want.V)
        np.testing.assert_array_equal(mask.cpu().numpy(), want.mask)
        g = dsg.Graph.from_csr(c.n, c.off, c.adj)
        g.bahmani(1, 10)
        g.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) > before
    finally:
        dsg.use_torch_allocator(False)


def test_noalloc_rejects_graphs_beyond_the_fixed_buffer():
    n = 5_000_000  # eps = 0 needs a 16(n+2)-byte round history alone: above 64 MiB
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    st = dsg.lib().dsg_bahmani_noalloc(n, off.data_ptr(), None, 0, 1, None, None, None, None)
    assert st == N.DSG_EINVAL
    assert b"fixed" in dsg.lib().dsg_last_error()
