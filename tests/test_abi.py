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
