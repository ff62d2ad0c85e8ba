"""GPU: with PyTorch's caching allocator installed through dsg_set_allocator
every device buffer of the library comes from torch, and results stay equal
to the oracle; switching back to the built-in pool keeps working."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2103_00154_gb300 as dsg  # noqa: E402


def test_torch_allocator_round_trip():
    raw = inputs.er_block(n=30000, m=150000, k=90, p=0.5, seed=21)
    c = oracle.from_raw(raw)
    want = oracle.bahmani(c, 1, 10)
    want_core = oracle.kcore_bz(c)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    dsg.use_torch_allocator(True)
    try:
        g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
        # the graph's CSR (u64 offsets, u32 adjacency) lives in torch's pool now
        assert torch.cuda.memory_allocated() - before >= 8 * (g.n + 1) + 4 * 2 * g.m
        mask, E, V = g.bahmani(1, 10)
        assert (E, V) == (want.E, want.V)
        np.testing.assert_array_equal(mask, want.mask)
        np.testing.assert_array_equal(g.kcore(), want_core)
        r = g.cbds()
        kstar, Ek, Vk = oracle.densest_core(c, want_core)
        assert (r.k_star, r.E_core, r.V_core) == (kstar, Ek, Vk)
        g.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before  # every buffer went back
    finally:
        dsg.use_torch_allocator(False)
    g = dsg.Graph.from_edges(raw.n, raw.src, raw.dst)
    try:
        np.testing.assert_array_equal(g.kcore(), want_core)
    finally:
        g.close()
