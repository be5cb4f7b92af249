"""GB300 (sm_103a) multilevel graph partitioner after "Tera-Scale Multilevel
Graph Partitioning" (TeraPart): deterministic size-constrained label
propagation over CSR or gap+VarInt compressed graphs, contraction, initial
bisection and LP refinement, all in CUDA kernels behind the C-ABI of
include/terapart.h.

This module marshals arguments only. PyTorch provides device memory and
streams; numpy arrays are accepted as host inputs.
"""
import ctypes
import threading

import numpy as np

from ._lib import ProfileEntry, Params, Request, RequestInfo, Stats, TpError, check, lib

__all__ = ["Graph", "Params", "Stats", "TpError", "default_params", "graph_from_csr",
           "graph_from_compressed", "partition", "lp_cluster", "lp_subround", "contract",
           "initial_partition", "lp_refine", "rebalance", "metrics", "launch_count",
           "profile_enable", "profile_read", "PROFILE_FAMILIES", "partition_batch", "Server",
           "footprint_bytes", "use_torch_allocator", "use_default_allocator", "set_allocator",
           "graph_from_stream_ex"]

PROFILE_FAMILIES = ("rate_small", "rate_mid", "rate_big", "rate_huge", "approve", "rate_lane")


def _torch():
    import torch

    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(x):
    """Device pointer of a CUDA tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return ctypes.c_void_p(x.ctypes.data)
    assert x.is_contiguous()
    return ctypes.c_void_p(x.data_ptr())


# Device-memory hook (tp_set_allocator): alloc(bytes, stream, ctx) -> pointer,
# free(pointer, bytes, stream, ctx).
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_hook = None  # the installed callbacks, kept alive while the library may call them


def set_allocator(alloc, free):
    """Installs Python callables as the library's device allocator:
    alloc(nbytes, stream_handle) -> int pointer (0 or an exception: out of
    memory), free(pointer, nbytes, stream_handle). None, None restores the
    library's default (cudaMallocAsync / cudaFreeAsync). Process-wide; set it
    while no library call is running."""
    global _hook
    if alloc is None and free is None:
        check(lib().tp_set_allocator(None, None, None), "tp_set_allocator")
        _hook = None
        return

    def _a(nbytes, stream, ctx):
        try:
            return alloc(int(nbytes), int(stream or 0)) or None
        except Exception:
            return None

    def _f(ptr, nbytes, stream, ctx):
        free(int(ptr or 0), int(nbytes), int(stream or 0))

    hook = (ALLOC_FN(_a), FREE_FN(_f))
    check(lib().tp_set_allocator(ctypes.cast(hook[0], ctypes.c_void_p),
                                 ctypes.cast(hook[1], ctypes.c_void_p), None), "tp_set_allocator")
    _hook = hook


def use_torch_allocator():
    """Routes every device allocation of the library through PyTorch's
    caching allocator (on the stream the library allocates on), so the
    partitioner shares torch's memory pool instead of allocating beside it."""
    torch = _torch()

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    set_allocator(alloc, free)


def use_default_allocator():
    """Restores the library's own stream-ordered allocator."""
    set_allocator(None, None)


def default_params(**overrides) -> Params:
    p = Params()
    lib().tp_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Graph:
    """Owning handle of a device-resident graph (CSR or compressed)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle) if not isinstance(handle, ctypes.c_void_p) else handle

    @property
    def handle(self):
        return self._h

    def info(self):
        n, m2, comp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        nb, sb = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().tp_graph_info(self._h, ctypes.byref(n), ctypes.byref(m2), ctypes.byref(comp),
                                  ctypes.byref(nb), ctypes.byref(sb)), "tp_graph_info")
        return {"n": n.value, "m2": m2.value, "compressed": bool(comp.value), "bytes": nb.value,
                "stream_bytes": sb.value}

    @property
    def n(self):
        return self.info()["n"]

    def compress(self, stream=None) -> "Graph":
        out = ctypes.c_void_p()
        check(lib().tp_graph_compress(self._h, _stream(stream), ctypes.byref(out)),
              "tp_graph_compress")
        return Graph(out)

    def decompress(self, stream=None) -> "Graph":
        out = ctypes.c_void_p()
        check(lib().tp_graph_decompress(self._h, _stream(stream), ctypes.byref(out)),
              "tp_graph_decompress")
        return Graph(out)

    def export_csr(self, stream=None):
        torch = _torch()
        inf = self.info()
        n, m2 = inf["n"], inf["m2"]
        xadj = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        adj = torch.empty(max(m2, 1), dtype=torch.int32, device="cuda")
        vw = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        ew = torch.empty(max(m2, 1), dtype=torch.int64, device="cuda")
        check(lib().tp_graph_export_csr(self._h, _ptr(xadj), _ptr(adj), _ptr(vw), _ptr(ew),
                                        _stream(stream)), "tp_graph_export_csr")
        return xadj, adj[:m2], vw[:n], ew[:m2]

    def export_compressed(self, stream=None):
        torch = _torch()
        inf = self.info()
        n, nbytes = inf["n"], inf["stream_bytes"]
        data = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        check(lib().tp_graph_export_compressed(self._h, _ptr(data), _ptr(off), _stream(stream)),
              "tp_graph_export_compressed")
        return data[:nbytes], off

    def encode_ex(self, intervals=True, weights=False, stream=None):
        """(bytes uint8 CUDA tensor, offsets int64 CUDA tensor holding u64) of
        this CSR graph in the interval + edge-weight format (tp_encode_ex)."""
        torch = _torch()
        n = self.n
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        nb = ctypes.c_uint64()
        check(lib().tp_encode_ex(self._h, int(intervals), int(weights), _ptr(off), None,
                                 ctypes.byref(nb), _stream(stream)), "tp_encode_ex")
        data = torch.empty(max(nb.value, 1), dtype=torch.uint8, device="cuda")
        check(lib().tp_encode_ex(self._h, int(intervals), int(weights), _ptr(off), _ptr(data),
                                 ctypes.byref(nb), _stream(stream)), "tp_encode_ex")
        return data[: nb.value], off

    def check(self, stream=None):
        check(lib().tp_graph_check(self._h, _stream(stream)), "tp_graph_check")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().tp_graph_destroy(h)
            except Exception:
                pass
            self._h = ctypes.c_void_p()


def _is_host(x):
    return isinstance(x, np.ndarray) or getattr(getattr(x, "device", None), "type", "") == "cpu"


def graph_from_csr(xadj, adj, vw=None, ew=None, stream=None) -> Graph:
    """xadj int64[n+1], adj int32[2m]: numpy arrays or CPU tensors (copied in
    from host memory, pinned tensors asynchronously) or CUDA tensors."""
    host = _is_host(xadj)
    if isinstance(xadj, np.ndarray):
        xadj = np.ascontiguousarray(xadj, np.int64)
        adj = np.ascontiguousarray(adj, np.int32)
        vw = None if vw is None else np.ascontiguousarray(vw, np.int64)
        ew = None if ew is None else np.ascontiguousarray(ew, np.int64)
    out = ctypes.c_void_p()
    check(lib().tp_graph_from_csr(len(xadj) - 1, _ptr(xadj), _ptr(adj), _ptr(vw), _ptr(ew),
                                  int(host), _stream(stream), ctypes.byref(out)),
          "tp_graph_from_csr")
    return Graph(out)


def graph_from_compressed(n, data, off, stream=None) -> Graph:
    host = isinstance(data, np.ndarray)
    if host:
        data = np.ascontiguousarray(data, np.uint8)
        off = np.ascontiguousarray(off, np.uint64)
    out = ctypes.c_void_p()
    nbytes = len(data) if host else data.numel()
    check(lib().tp_graph_from_compressed(n, nbytes, _ptr(data), _ptr(off), int(host),
                                         _stream(stream), ctypes.byref(out)),
          "tp_graph_from_compressed")
    return Graph(out)


def lp_subround(g: Graph, label, lw, cap, round_key, S, s, stream=None):
    """One synchronous LP sub-round in place on label (int32 CUDA) and lw (int64 CUDA)."""
    check(lib().tp_lp_subround(g.handle, _ptr(label), _ptr(lw), lw.numel(), cap, round_key, S, s,
                               _stream(stream)), "tp_lp_subround")


def lp_cluster(g: Graph, max_cluster_weight, params=None, level=0, stream=None):
    torch = _torch()
    p = params or default_params()
    C = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    check(lib().tp_lp_cluster(g.handle, max_cluster_weight, ctypes.byref(p), level, _ptr(C),
                              _stream(stream)), "tp_lp_cluster")
    return C[: g.n]


def contract(g: Graph, C, stream=None):
    torch = _torch()
    out = ctypes.c_void_p()
    mp = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    check(lib().tp_contract(g.handle, _ptr(C), _stream(stream), ctypes.byref(out), _ptr(mp)),
          "tp_contract")
    return Graph(out), mp[: g.n]


def initial_partition(g: Graph, k, l_max, params=None, stream=None):
    torch = _torch()
    p = params or default_params()
    part = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    check(lib().tp_initial_partition(g.handle, k, l_max, ctypes.byref(p), _ptr(part),
                                     _stream(stream)), "tp_initial_partition")
    return part[: g.n]


def lp_refine(g: Graph, k, l_max, part, params=None, level=0, stream=None):
    p = params or default_params()
    check(lib().tp_lp_refine(g.handle, k, l_max, ctypes.byref(p), level, _ptr(part),
                             _stream(stream)), "tp_lp_refine")
    return part


def rebalance(g: Graph, k, l_max, part, stream=None):
    ok = ctypes.c_int()
    check(lib().tp_rebalance(g.handle, k, l_max, _ptr(part), ctypes.byref(ok), _stream(stream)),
          "tp_rebalance")
    return bool(ok.value)


def metrics(g: Graph, part, k, stream=None):
    cut = ctypes.c_int64()
    B = np.zeros(k, np.int64)
    check(lib().tp_metrics(g.handle, _ptr(part), k, ctypes.byref(cut), _ptr(B), _stream(stream)),
          "tp_metrics")
    return cut.value, B


def stats_dict(st: Stats):
    L = st.levels
    return {"cut": st.cut, "max_block_weight": st.max_block_weight, "l_max": st.l_max,
            "u_max": st.u_max, "imbalance": st.imbalance, "levels": L,
            "balanced": bool(st.balanced), "level_n": list(st.level_n[:L]),
            "level_m2": list(st.level_m2[:L]), "ms_coarsen": st.ms_coarsen,
            "ms_initial": st.ms_initial, "ms_uncoarsen": st.ms_uncoarsen,
            "ms_lp_level0": st.ms_lp_level0, "peak_bytes": st.peak_bytes}


def partition(g: Graph, k, eps=0.03, params=None, out=None, stream=None):
    """Full multilevel partition. Returns (part int32 CUDA tensor, stats dict)."""
    torch = _torch()
    p = params or default_params()
    n = g.n
    part = out if out is not None else torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    st = Stats()
    check(lib().tp_partition(g.handle, k, eps, ctypes.byref(p), _ptr(part), ctypes.byref(st),
                             _stream(stream)), "tp_partition")
    return part[:n], stats_dict(st)



def partition_batch(graphs, ks, eps=0.03, params=None, concurrency=1, outs=None):
    """Batched mode: partitions independent graphs together (tp_partition_batch),
    one union graph per level; concurrency bounds how many unions (groups of a
    very large batch) run at once.

    Each result equals partition(graphs[i], ks[i], eps, params). Returns a list
    of (part int32 CUDA tensor, stats dict) in input order; raises on the first
    failing graph.
    """
    torch = _torch()
    p = params or default_params()
    cnt = len(graphs)
    if len(ks) != cnt:
        raise ValueError("one k per graph")
    parts = outs if outs is not None else [
        torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda") for g in graphs]
    handles = (ctypes.c_void_p * max(cnt, 1))(*[g.handle for g in graphs])
    karr = (ctypes.c_int32 * max(cnt, 1))(*[int(k) for k in ks])
    parr = (ctypes.c_void_p * max(cnt, 1))(*[_ptr(t) for t in parts])
    st = (Stats * max(cnt, 1))()
    status = (ctypes.c_int * max(cnt, 1))()
    torch.cuda.synchronize()  # inputs written on other streams are complete
    check(lib().tp_partition_batch(cnt, handles, karr, eps, ctypes.byref(p), parr, st, status,
                                   concurrency), "tp_partition_batch")
    return [(parts[i][: graphs[i].n], stats_dict(st[i])) for i in range(cnt)]


def graph_from_stream_ex(n, data, off, intervals=True, weighted=False, stream=None) -> Graph:
    """CSR graph decoded from an interval + edge-weight stream (device tensors;
    tp_graph_from_stream_ex)."""
    out = ctypes.c_void_p()
    check(lib().tp_graph_from_stream_ex(int(n), int(data.numel()), _ptr(data), _ptr(off),
                                        int(intervals), int(weighted), _stream(stream),
                                        ctypes.byref(out)), "tp_graph_from_stream_ex")
    return Graph(out)


def footprint_bytes(n, m2, k, upload=True, compress=False) -> int:
    """Device memory budget one served request is charged (tp_footprint_bytes)."""
    return lib().tp_footprint_bytes(n, m2, k, int(upload), int(compress))


class Server:
    """Serving with continuous batching (tp_server_*): requests are admitted in
    FIFO order as workers and device-memory budget free up, and run
    concurrently; each result equals partition() of that graph alone."""

    def __init__(self, budget_bytes, workers=8, params=None):
        self._p = params or default_params()
        h = ctypes.c_void_p()
        check(lib().tp_server_create(int(budget_bytes), workers, ctypes.byref(self._p),
                                     ctypes.byref(h)), "tp_server_create")
        self._h = h
        self._pending = {}
        self._lock = threading.Lock()

    def submit(self, k, eps=0.03, xadj=None, adj=None, graph=None, compress=False):
        """Queues a request on a host CSR (xadj, adj numpy) or a resident Graph;
        returns a ticket."""
        if graph is not None:
            n = graph.n
            req = Request(graph.handle, 0, None, None, 0, int(k), float(eps), None)
            keep = ()
        else:
            xadj = np.ascontiguousarray(xadj, dtype=np.int64)
            adj = np.ascontiguousarray(adj, dtype=np.int32)
            n = len(xadj) - 1
            req = Request(None, n, xadj.ctypes.data, adj.ctypes.data, int(compress), int(k),
                          float(eps), None)
            keep = (xadj, adj)
        part = np.empty(max(n, 1), dtype=np.int32)
        req.part = part.ctypes.data
        t = ctypes.c_uint64()
        check(lib().tp_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)),
              "tp_server_submit")
        with self._lock:
            self._pending[t.value] = (part, n, keep, graph)
        return t.value

    def wait(self, ticket):
        """(partition numpy int32, stats dict, info dict) of a submitted request."""
        with self._lock:  # a ticket is waited once
            entry = self._pending.pop(ticket, None)
        if entry is None:
            raise TpError(1, "tp_server_wait (unknown or already waited ticket)")
        part, n, _, _ = entry
        st, info = Stats(), RequestInfo()
        check(lib().tp_server_wait(self._h, ticket, ctypes.byref(st), ctypes.byref(info)),
              "tp_server_wait")
        return part[:n], stats_dict(st), {f: getattr(info, f) for f, _ in RequestInfo._fields_}

    def peak_in_use(self):
        return lib().tp_server_peak_in_use(self._h)

    def close(self):
        if self._h:
            lib().tp_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return lib().tp_launch_count()


def profile_enable(on: bool = True):
    lib().tp_profile_enable(int(on))


def profile_read(stream=None):
    """Per-family {launches, ms, bytes} of the profiled level-0 LP launches (clears them)."""
    arr = (ProfileEntry * len(PROFILE_FAMILIES))()
    k = lib().tp_profile_read(arr, len(arr), _stream(stream))
    if k < 0:
        raise TpError(3, "tp_profile_read")
    return {PROFILE_FAMILIES[i]: {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes}
            for i in range(k)}
