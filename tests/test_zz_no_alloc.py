"""tp_metrics_static: the partition metrics without device allocation.

Callers that cannot allocate device memory when they need the metrics (code
under CUDA stream capture, services with a fixed device-memory footprint,
callers without an allocator) use this entry point; its scratch is a fixed
array inside the library. It must give exactly what the allocating
tp_metrics gives, call after call, since every call reuses (and must clear)
the same array. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402

TP_ERR_BUDGET = 6
STATIC_MAX_BLOCKS = 16383


def _static_metrics(g, part, k):
    cut = ctypes.c_int64(-1)
    B = np.full(k, -1, np.int64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = tp.lib().tp_metrics_static(g.handle, ctypes.c_void_p(part.data_ptr()), k,
                                    ctypes.byref(cut), ctypes.c_void_p(B.ctypes.data), stream)
    return rc, cut.value, B


def test_metrics_static_matches_allocating_metrics_twice_in_a_row():
    xadj, adj = synth.rgg2d(50000, 16.0, 7)
    csr = tp.graph_from_csr(xadj, adj)
    rng = np.random.default_rng(3)
    for g in (csr, csr.compress()):
        for k in (5, 1000):
            for _ in range(2):  # the second call must not see the first call's sums
                part = torch.from_numpy(rng.integers(0, k, size=len(xadj) - 1).astype(np.int32)).cuda()
                want_cut, want_B = tp.metrics(g, part, k)
                rc, cut, B = _static_metrics(g, part, k)
                assert rc == 0
                assert cut == want_cut
                assert np.array_equal(B, want_B)


def test_metrics_static_rejects_k_beyond_its_scratch():
    xadj, adj = synth.gnm(1000, 4000, 2)
    g = tp.graph_from_csr(xadj, adj)
    part = torch.zeros(1000, dtype=torch.int32, device="cuda")
    rc, _, _ = _static_metrics(g, part, STATIC_MAX_BLOCKS)
    assert rc == 0
    rc, _, _ = _static_metrics(g, part, STATIC_MAX_BLOCKS + 1)
    assert rc == TP_ERR_BUDGET
