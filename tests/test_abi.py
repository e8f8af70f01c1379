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

    assert set(kchol.EXPORTED) == set(_declared())


def test_argument_errors_without_gpu(so):
    """Invalid arguments are rejected before any device work."""
    lib = ctypes.CDLL(so)
    lib.kc_last_error.restype = ctypes.c_char_p
    st = lib.kc_order_points(None, ctypes.c_int64(10), ctypes.c_int32(2), None, None, None, None)
    assert st == 1 and b"NULL" in lib.kc_last_error()
    st = lib.kc_schedule(ctypes.c_int64(0), None, None, None, ctypes.c_int32(0), None, None, None, None, None, None,
                         None)
    assert st == 1


def test_new_entries_reject_bad_arguments_without_gpu(so):
    from paper_1706_02205_gb300 import kchol
    lib = kchol.lib()
    bad = [kchol.Kernel(nu=0.0), kchol.Kernel(nu=60.0), kchol.Kernel(ell=0.0),
           kchol.Kernel(family=kchol.CAUCHY, alpha=2.5), kchol.Kernel(family=kchol.CAUCHY, beta=0.0),
           kchol.Kernel(family=7)]
    for k in bad:
        kk = k.c()
        assert lib.kc_kernel_eval(ctypes.byref(kk), 0, None, 0, None, None) == kchol.KC_EINVAL, k
    ok = kchol.Kernel(nu=0.8).c()
    assert lib.kc_kernel_eval(ctypes.byref(ok), 5, None, 0, None, None) == kchol.KC_EINVAL  # bad prec
    for name in ("kc_l_matvec", "kc_lt_matvec", "kc_llt_matvec"):
        assert getattr(lib, name)(None, 0, None, None, None, None, 1, None, None) == kchol.KC_EINVAL
    v = ctypes.c_double(0.0)
    assert lib.kc_logdet(None, None, ctypes.byref(v), None, None) == kchol.KC_EINVAL
    assert lib.kc_pattern_reverse(0, None, None, None, None, None) == kchol.KC_EINVAL
    assert lib.kc_pattern_reverse(4, None, None, None, None, None) == kchol.KC_EINVAL
    assert lib.kc_gather_entries(4, None, None, None, None, None, None, None, None, None) == kchol.KC_EINVAL
    assert lib.kc_factor_given(None, None, 0, None, None, None, None, None) == kchol.KC_EINVAL
    assert lib.kc_supernodal_count(None, None, 2, 3.0, None, None, None, None, None, None, None, None,
                                   None) == kchol.KC_EINVAL
    assert lib.kc_supernodal_fill(None, None, 2, 3.0, None, None, None, None) == kchol.KC_EINVAL
    assert lib.kc_pattern_validate(None, None) == kchol.KC_EINVAL
    assert lib.kc_supernodal(None, None, 2, 3.0, None, None, None, None, None, None, None, None, 0, None,
                             None) == kchol.KC_EINVAL
    assert lib.kc_refine_sparse(None, 0, None, None, None, None, None, None, None, 1, 1e-10, 10, None, None, None,
                                None, None) == kchol.KC_EINVAL


def test_struct_layouts_match_header(tmp_path):
    """Offsets of the ABI structs as a C compiler lays them out from the header
    equal the binding's ctypes layouts."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    from paper_1706_02205_gb300 import kchol
    structs = {"kc_kernel": kchol.kc_kernel, "kc_opts": kchol.kc_opts, "kc_pattern": kchol.kc_pattern}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kchol.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
