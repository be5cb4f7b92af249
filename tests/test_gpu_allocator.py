"""The library's device memory through PyTorch's caching allocator
(tp_set_allocator, installed by use_torch_allocator): results equal the
oracle's, the memory is visibly torch's, and buffers made under one
allocator are released through it after the hook changed."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402


@pytest.fixture
def torch_alloc():
    tp.use_torch_allocator()
    try:
        yield
    finally:
        tp.use_default_allocator()


@pytest.mark.parametrize("kind,k", [("rgg", 16), ("rmat", 32)])
def test_partition_with_torch_allocator_equals_oracle(torch_alloc, kind, k):
    xadj, adj = synth.rgg2d(1 << 16, 16.0, 3) if kind == "rgg" else synth.rmat(15, 16, seed=2)
    want, wst = oracle.partition(oracle.Graph(xadj, adj), k, 0.03, oracle.Params(seed=1))
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    g = tp.graph_from_csr(xadj, adj)
    assert torch.cuda.memory_allocated() > base  # the graph lives in torch's pool
    for gg in (g.compress(), g):
        part, st = tp.partition(gg, k, 0.03, tp.default_params(seed=1))
        assert np.array_equal(part.cpu().numpy(), want)
        assert st["cut"] == wst["cut"] and st["level_n"] == wst["level_n"]
    assert torch.cuda.max_memory_allocated() > base + 8 * len(adj)


def test_buffers_are_released_through_the_allocator_that_made_them():
    xadj, adj = synth.gnm(4000, 30000, 5)
    want, _ = oracle.partition(oracle.Graph(xadj, adj), 8, 0.03, oracle.Params(seed=2))
    g_default = tp.graph_from_csr(xadj, adj)  # library allocator
    tp.use_torch_allocator()
    try:
        g_torch = tp.graph_from_csr(xadj, adj)  # torch's pool
        part, _ = tp.partition(g_default, 8, 0.03, tp.default_params(seed=2))
        assert np.array_equal(part.cpu().numpy(), want)
        del g_default  # freed with cudaFreeAsync although the hook is torch's
    finally:
        tp.use_default_allocator()
    part, _ = tp.partition(g_torch, 8, 0.03, tp.default_params(seed=2))
    assert np.array_equal(part.cpu().numpy(), want)
    before = torch.cuda.memory_allocated()
    del g_torch  # returned to torch's pool although the hook is the default again
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() < before
