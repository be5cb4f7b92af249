"""ctypes declarations of the C-ABI in include/terapart.h.

Argument marshalling only: every step of the partitioner runs in the CUDA
library. Loading fails loudly when the library has not been built; there is
no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libterapart.so")

i32, i64, u64, vp, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
P = ctypes.POINTER

STATUS = {0: "ok", 1: "invalid", 2: "oom", 3: "cuda", 4: "corrupt", 5: "timeout", 6: "budget"}


class TpError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")


class Params(ctypes.Structure):
    _fields_ = [("seed", u64), ("cluster_rounds", i32), ("refine_rounds", i32),
                ("sub_rounds", i32), ("c_lim", i32), ("ip_attempts", i32), ("two_hop", i32),
                ("max_levels", i32), ("tier_lane", i32), ("tier_small", i32), ("tier_mid", i32),
                ("warps_per_block", i32), ("use_graphs", i32), ("graph_n", i32),
                ("table_slack", i32)]


class Stats(ctypes.Structure):
    _fields_ = [("cut", i64), ("max_block_weight", i64), ("l_max", i64), ("u_max", i64),
                ("imbalance", ctypes.c_double), ("levels", i32), ("balanced", i32),
                ("level_n", i64 * 64), ("level_m2", i64 * 64), ("ms_coarsen", ctypes.c_double),
                ("ms_initial", ctypes.c_double), ("ms_uncoarsen", ctypes.c_double),
                ("ms_lp_level0", ctypes.c_double), ("peak_bytes", i64)]


class Request(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("n", i64), ("xadj", ctypes.c_void_p),
                ("adj", ctypes.c_void_p), ("compress", i32), ("k", i32), ("eps", ctypes.c_double),
                ("part", ctypes.c_void_p)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("queued_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("footprint_bytes", i64), ("peak_bytes", i64),
                ("retries", i32)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("family", i32), ("launches", i64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


SIGNATURES = {
    "tp_params_default": (None, [P(Params)]),
    "tp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tp_set_allocator": (ctypes.c_int, [vp, vp, vp]),
    "tp_graph_from_csr": (ctypes.c_int, [i64, vp, vp, vp, vp, ctypes.c_int, vp, P(vp)]),
    "tp_graph_compress": (ctypes.c_int, [vp, vp, P(vp)]),
    "tp_graph_from_compressed": (ctypes.c_int, [i64, u64, vp, vp, ctypes.c_int, vp, P(vp)]),
    "tp_graph_decompress": (ctypes.c_int, [vp, vp, P(vp)]),
    "tp_encode_ex": (ctypes.c_int, [vp, i32, i32, vp, vp, P(u64), vp]),
    "tp_graph_from_stream_ex": (ctypes.c_int, [i64, u64, vp, vp, i32, i32, vp, P(vp)]),
    "tp_graph_info": (ctypes.c_int, [vp, P(i64), P(i64), P(ctypes.c_int), P(sz), P(sz)]),
    "tp_graph_export_csr": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
    "tp_graph_export_compressed": (ctypes.c_int, [vp, vp, vp, vp]),
    "tp_graph_check": (ctypes.c_int, [vp, vp]),
    "tp_graph_destroy": (None, [vp]),
    "tp_lp_subround": (ctypes.c_int, [vp, vp, vp, i64, i64, u64, i32, i32, vp]),
    "tp_lp_cluster": (ctypes.c_int, [vp, i64, P(Params), i32, vp, vp]),
    "tp_contract": (ctypes.c_int, [vp, vp, vp, P(vp), vp]),
    "tp_initial_partition": (ctypes.c_int, [vp, i32, i64, P(Params), vp, vp]),
    "tp_lp_refine": (ctypes.c_int, [vp, i32, i64, P(Params), i32, vp, vp]),
    "tp_rebalance": (ctypes.c_int, [vp, i32, i64, vp, P(ctypes.c_int), vp]),
    "tp_metrics": (ctypes.c_int, [vp, vp, i32, P(i64), vp, vp]),
    "tp_metrics_static": (ctypes.c_int, [vp, vp, i32, P(i64), vp, vp]),
    "tp_partition": (ctypes.c_int, [vp, i32, ctypes.c_double, P(Params), vp, P(Stats), vp]),
    "tp_partition_batch": (ctypes.c_int, [i32, P(vp), P(i32), ctypes.c_double, P(Params), P(vp),
                                          P(Stats), P(ctypes.c_int), i32]),
    "tp_launch_count": (u64, []),
    "tp_footprint_bytes": (i64, [i64, i64, i32, i32, i32]),
    "tp_server_create": (ctypes.c_int, [i64, i32, P(Params), P(vp)]),
    "tp_server_submit": (ctypes.c_int, [vp, P(Request), P(u64)]),
    "tp_server_wait": (ctypes.c_int, [vp, u64, P(Stats), P(RequestInfo)]),
    "tp_server_peak_in_use": (i64, [vp]),
    "tp_server_destroy": (None, [vp]),
    "tp_profile_enable": (None, [ctypes.c_int]),
    "tp_profile_read": (ctypes.c_int, [P(ProfileEntry), ctypes.c_int, vp]),
}

_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code, where):
    if code != 0:
        raise TpError(code, where)
