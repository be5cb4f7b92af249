"""The C-ABI library loads and exports every entry point include/terapart.h
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "terapart.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tp_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_19119_gb300 import build as b

    b.build()
    return ctypes.CDLL(b.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_abi():
    from paper_2410_19119_gb300 import _lib

    assert set(_lib.SIGNATURES) == set(_declared())


def test_defaults_and_status_strings(lib):
    import paper_2410_19119_gb300 as tp

    p = tp.default_params()
    assert (p.cluster_rounds, p.refine_rounds, p.sub_rounds, p.c_lim, p.ip_attempts) == (5, 5, 8, 160, 8)
    lib.tp_status_string.restype = ctypes.c_char_p
    assert lib.tp_status_string(4) == b"corrupt compressed graph"


def test_footprint_bound_is_monotone_and_validates(lib):
    f = lib.tp_footprint_bytes
    f.restype = ctypes.c_int64
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    base = f(1 << 20, 1 << 24, 64, 0, 0)
    assert base > 0
    assert f((1 << 20) + 1, 1 << 24, 64, 0, 0) > base  # more vertices
    assert f(1 << 20, (1 << 24) + 1, 64, 0, 0) > base  # more adjacency entries
    assert f(1 << 20, 1 << 24, 65, 0, 0) > base        # more blocks
    up = f(1 << 20, 1 << 24, 64, 1, 0)
    assert up > base and f(1 << 20, 1 << 24, 64, 1, 1) > up  # upload, then compression
    # at least the uploaded CSR itself: 8 (n + 1) + 4 m2 bytes
    assert up - base >= 8 * ((1 << 20) + 1) + 4 * (1 << 24)
    assert f(-1, 0, 2, 0, 0) == -1 and f(1, -1, 2, 0, 0) == -1 and f(1, 0, 0, 0, 0) == -1


def test_batch_and_server_reject_bad_arguments_without_a_device(lib):
    # argument checks happen before any device work
    lib.tp_partition_batch.restype = ctypes.c_int
    assert lib.tp_partition_batch(-1, None, None, ctypes.c_double(0.03), None, None, None, None,
                                  4) == 1
    assert lib.tp_partition_batch(0, None, None, ctypes.c_double(0.03), None, None, None, None,
                                  0) == 1  # concurrency < 1
    assert lib.tp_partition_batch(0, None, None, ctypes.c_double(0.03), None, None, None, None,
                                  4) == 0  # empty batch
    lib.tp_server_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.tp_server_create(ctypes.c_int64(0), 4, None, ctypes.byref(out)) == 1  # no budget
    assert lib.tp_server_create(ctypes.c_int64(1 << 30), 0, None, ctypes.byref(out)) == 1
