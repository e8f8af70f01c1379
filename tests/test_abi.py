"""The C-ABI library builds, loads and exports every symbol include/kchol.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "kchol.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|kc_status|int32_t|int64_t|double|void)\s+(kc_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def so():
    from paper_1706_02205_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("kc_order_points", "kc_pattern_count", "kc_pattern_fill", "kc_schedule", "kc_factor", "kc_solve",
              "kc_refine", "kc_pca_truncate", "kc_pca_error", "kc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(so):
    lib = ctypes.CDLL(so)
    for n in _declared():
        assert hasattr(lib, n), n
    lib.kc_abi_version.restype = ctypes.c_int32
    # the library, the header and the Python binding agree on the interface version
    from paper_1706_02205_gb300 import kchol
    hdr = open(os.path.join(ROOT, "include", "kchol.h")).read()
    assert int(re.search(r"#define KC_ABI_VERSION (\d+)", hdr).group(1)) == lib.kc_abi_version() == kchol.ABI_VERSION


def test_binding_lists_match_header(so):
    from paper_1706_02205_gb300 import kchol

    assert set(kchol.EXPORTED) <= set(_declared())


def test_argument_errors_without_gpu(so):
    """Invalid arguments are rejected before any device work."""
    lib = ctypes.CDLL(so)
    lib.kc_last_error.restype = ctypes.c_char_p
    st = lib.kc_order_points(None, ctypes.c_int64(10), ctypes.c_int32(2), None, None, None, None)
    assert st == 1 and b"NULL" in lib.kc_last_error()
    st = lib.kc_schedule(ctypes.c_int64(0), None, None, None, ctypes.c_int32(0), None, None, None, None, None, None,
                         None)
    assert st == 1
