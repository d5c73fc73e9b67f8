"""CPU checks of the C ABI: the library loads and exports every symbol that
include/krr.h declares (no compute call: there is no GPU here)."""
import os
import re

import pytest

from paper_2409_01712_gb300 import _build, krr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    try:
        _build.build()
    except RuntimeError as e:  # no nvcc: nothing to check here
        pytest.skip(f"cannot build libkrr.so: {e}")
    return krr.load_library()


def _declared():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(krr_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_binding_symbols():
    assert _declared() == set(krr.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_options(lib):
    o = krr.default_options()
    assert o.tile == 1024 and o.mode == 0 and o.ir_max == 30
    assert o.eps == pytest.approx(6e-4) and o.ir_tol == pytest.approx(1e-7)
    assert o.prec_rule == 0 and o.kernel == 0 and o.lookahead == 1 and o.reserved == 0


def test_struct_layouts_match_header():
    import ctypes

    # int64 + 2 int32 + 2 double + 2 int32 + int64 + 4 int32 = 64 bytes, no padding
    assert ctypes.sizeof(krr.Options) == 64
    assert ctypes.sizeof(krr.FactorInfo) == 8 * 8
    assert ctypes.sizeof(krr.SolveInfo) == 8 + 8 + 32 * 8
