"""GPU parity for the supernodal multicolour ordering and pattern (the
Construction of the stability section): the order, levels, supernodes,
colours and pattern bit-exact against the oracle; the factor on them within
the bars of the maximin factor."""
import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import kchol as kc  # noqa: E402
from tests import factor_parity as fp  # noqa: E402

DEV = torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


CASES = [
    ("uniform2d_rho2", lambda: inputs.uniform(700, 2, seed=101), 2.0),
    ("uniform2d_rho3", lambda: inputs.uniform(3000, 2, seed=102), 3.0),
    ("uniform3d", lambda: inputs.uniform(1500, 3, seed=103), 2.5),
    ("jitter", lambda: inputs.jittered_grid(48, seed=104), 3.0),
    ("swiss20", lambda: inputs.swiss_roll(1200, seed=105), 2.0),
    ("int_ties", lambda: np.stack(np.meshgrid(np.arange(31.0), np.arange(23.0), indexing="ij"), -1).reshape(-1, 2)
     [inputs.rng(106).permutation(31 * 23)], 2.0),
    ("duplicates", lambda: np.repeat(inputs.uniform(250, 2, seed=107), 2, axis=0), 2.0),
    ("tiny1", lambda: inputs.uniform(1, 2, seed=108), 2.0),
    ("tiny3", lambda: inputs.uniform(3, 2, seed=109), 2.0),
]


def _device(x, rho):
    perm0, l, xo = kc.order_points(T(x))
    pat0 = kc.build_pattern(xo, l, rho)
    sn = kc.supernodal(xo, l, rho, pat0)
    return perm0, sn


@pytest.mark.parametrize("name,make,rho", CASES, ids=[c[0] for c in CASES])
def test_supernodal_bit_exact(name, make, rho):
    x = make()
    ref = oracle.supernodal(x, rho)
    perm0, sn = _device(x, rho)
    assert np.array_equal(H(perm0), ref["perm"])
    newm = H(sn["newm"])
    assert np.array_equal(H(perm0)[newm], ref["order"])
    assert np.array_equal(H(sn["level"]), ref["level"])
    assert np.array_equal(H(sn["node"]), ref["node"])
    assert np.array_equal(H(sn["color"]), ref["color"])
    assert np.array_equal(H(sn["x_new"]), x[ref["order"]])
    assert np.array_equal(H(sn["pat"].rowptr), ref["rowptr"])
    assert np.array_equal(H(sn["pat"].col), ref["col"])


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
@pytest.mark.parametrize("nu,ell,nugget", [(0.5, 0.2, 0.0), (1.5, 0.1, 1e-6)])
def test_supernodal_factor_matches_oracle(prec, nu, ell, nugget):
    x = inputs.uniform(3000, 2, seed=110)
    rho = 3.0
    ref = oracle.supernodal(x, rho)
    ko = oracle.Kernel(nu, ell, 1.0, nugget)
    kg = kc.Kernel(nu, ell, 1.0, nugget)
    xs = x[ref["order"]]
    val_ref, zc_ref, piv = oracle.ichol(xs, ref["rowptr"], ref["col"], ko, pivots=True)
    r = kc.supernodal_pipeline(T(x), rho, kg, prec)
    assert np.array_equal(H(r["perm"]), ref["order"])
    alt = oracle.ichol(xs, ref["rowptr"], ref["col"], ko, reverse_sums=(prec == kc.FP64),
                       store_f32=(prec == kc.FP32_FORM))
    fp.check_factor(prec, H(r["val"]), H(r["diag"]), ref["rowptr"], ref["col"], np.sqrt(1.0 + nugget),
                    (val_ref, zc_ref), alt=alt, piv=piv, strict=(nu == 0.5))


def test_supernodal_larger_structure():
    """8000 points: still bit-exact (many levels, many rounds of the greedy
    passes)."""
    x = inputs.uniform(8000, 2, seed=111)
    ref = oracle.supernodal(x, 3.0)
    perm0, sn = _device(x, 3.0)
    assert np.array_equal(H(perm0)[H(sn["newm"])], ref["order"])
    assert np.array_equal(H(sn["color"]), ref["color"])
    assert np.array_equal(H(sn["pat"].col), ref["col"])


def test_supernodal_two_phase_when_the_buffer_is_short():
    """kc_supernodal with too small a column buffer reports nnz and leaves the
    buffer alone; kc_supernodal_fill then completes the same pattern, and the
    count-only call gives the same rowptr."""
    import ctypes as C
    x = inputs.uniform(2000, 2, seed=112)
    perm0, l, xo = kc.order_points(T(x))
    pat0 = kc.build_pattern(xo, l, 3.0)
    ref = kc.supernodal(xo, l, 3.0, pat0)
    N, d = xo.shape
    lib = kc.lib()
    newm = torch.empty(N, dtype=torch.int32, device=DEV)
    x_new = torch.empty_like(xo)
    rp = torch.empty(N + 1, dtype=torch.int64, device=DEV)
    col = torch.full((4,), -7, dtype=torch.int32, device=DEV)
    nnz = C.c_int64(0)
    kc._check(lib.kc_supernodal(kc._ptr(xo), kc._ptr(l), d, 3.0, pat0.c(), kc._ptr(newm), None, None, None,
                                kc._ptr(x_new), kc._ptr(rp), kc._ptr(col), 4, C.byref(nnz), kc._stream(None)))
    assert nnz.value == ref["pat"].nnz and torch.all(col == -7)
    full = torch.empty(nnz.value, dtype=torch.int32, device=DEV)
    kc._check(lib.kc_supernodal_fill(kc._ptr(xo), kc._ptr(l), d, 3.0, pat0.c(), kc._ptr(rp), kc._ptr(full),
                                     kc._stream(None)))
    assert torch.equal(rp, ref["pat"].rowptr) and torch.equal(full, ref["pat"].col)
    rp2 = torch.empty_like(rp)
    nn2 = C.c_int64(0)
    kc._check(lib.kc_supernodal_count(kc._ptr(xo), kc._ptr(l), d, 3.0, pat0.c(), kc._ptr(newm), None, None, None,
                                      kc._ptr(x_new), kc._ptr(rp2), C.byref(nn2), kc._stream(None)))
    assert nn2.value == nnz.value and torch.equal(rp2, rp)
