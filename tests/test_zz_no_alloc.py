"""kc_solve_noalloc, the solve for callers that cannot allocate device memory
while they run (a server whose device memory is handed out up front to
another framework's pool, a plugin forbidden to allocate, a latency-critical
loop where an allocation could block or synchronise the device).

It must give the same answer as kc_solve, within the tolerance of the solve
tests (1e-11 relative), on two calls in a row: the fixed scratch array keeps
the previous call's contents, so the second call checks that everything that
must start at zero is cleared.  Sizes beyond its fixed scratch are rejected.
This file is collected last so that a failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import kchol as kc  # noqa: E402

DEV = torch.device("cuda:0")


def _T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_noalloc_solve_matches_solve_twice(prec):
    N = 3000
    x = inputs.uniform(N, 2, seed=91)
    perm, l, rp, col = oracle.sortsparse(x, 3.0)
    kern = kc.Kernel(0.5, 0.2)
    pat = kc.schedule(_T(rp), _T(col))
    val, diag, _ = kc.factor(pat, _T(x[perm]), kern, prec)
    p = _T(perm)
    for call, (nrhs, seed) in enumerate([(3, 92), (5, 93)]):
        b = _T(inputs.rhs(N, nrhs, seed=seed))
        want = kc.solve(pat, prec, val, diag, kern, p, b).cpu().numpy()
        out = torch.full_like(b, float("nan"))
        got = kc.solve_noalloc(pat, prec, val, diag, kern, p, b, out=out)
        assert got.data_ptr() == out.data_ptr()
        got = got.cpu().numpy()
        for r in range(nrhs):
            rel = np.linalg.norm(got[r] - want[r]) / np.linalg.norm(want[r])
            assert rel < 1e-11, (call, r, rel)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dummy = torch.zeros(8, dtype=torch.int64, device=DEV)
    pat = kc.kc_pattern(1 << 17, 1 << 17, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                        dummy.data_ptr(), dummy.data_ptr(), 1)
    kern = kc.Kernel(0.5, 0.2).c()
    st = kc.lib().kc_solve_noalloc(ctypes.byref(pat), kc.FP64, kc._ptr(dummy), kc._ptr(dummy), ctypes.byref(kern),
                                   kc._ptr(dummy), kc._ptr(dummy), 16, kc._ptr(dummy),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == kc.KC_EINVAL
    assert b"2^20" in kc.lib().kc_last_error()
