"""GPU parity of the factor by column groups (kc_factor_blocked): the
supernodal block factorisation of the stability appendix.

On the supernodal multicolour pattern every supernode is a group of columns
whose rows and columns are whole supernode ranges; the block algorithm equals
Algorithm 2 there (the appendix), so the result is held to the oracle's
ICHOL(0) on the same pattern with the bars of tests/factor_parity.py, and to
the defining identity.  On the maximin pattern every group is one column and
the same bars hold.  The result repeats bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs
from tests import factor_parity as fp
from tests import refmath

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import kchol as kc  # noqa: E402

DEV = torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


def _identity(xs, rp, col, val, ko):
    N = xs.shape[0]
    L = refmath.dense_lower(rp, col, val.astype(np.float64), N)
    Th = refmath.dense_cov(xs, ko)
    return fp.identity_residual_dense(L, Th, rp, col, ko.sigma2 + ko.nugget)


def _supernodal_case(N, d, seed, rho=3.0):
    x = inputs.uniform(N, d, seed=seed)
    ref = oracle.supernodal(x, rho)
    xs = x[ref["order"]]
    return xs, ref


SN_CASES = [  # d, nu, ell, nugget, family, alpha, beta, well-conditioned
    (2, 0.5, 0.2, 0.0, 0, 1.0, 1.0, True),
    (2, 1.5, 0.1, 1e-6, 0, 1.0, 1.0, False),
    (3, 0.5, 0.2, 0.0, 0, 1.0, 1.0, True),
    (2, 0.8, 0.2, 1e-6, 0, 1.0, 1.0, False),
    (2, 1.5, 0.2, 1e-4, 1, 1.0, 0.2, True),
]
_IDS = [f"d{c[0]}_nu{c[1]}_l{c[2]}_fam{c[4]}" for c in SN_CASES]


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
@pytest.mark.parametrize("case", SN_CASES, ids=_IDS)
def test_blocked_factor_on_the_supernodal_pattern(case, prec):
    d, nu, ell, nug, fam, al, be, strict = case
    xs, ref = _supernodal_case(3000 if d == 2 else 2500, d, seed=150 + d)
    rp, col = ref["rowptr"], ref["col"]
    ko = oracle.Kernel(nu, ell, 1.0, nug, fam, al, be)
    kg = kc.Kernel(nu, ell, 1.0, nug, fam, al, be)
    val_ref, zc, piv = oracle.ichol(xs, rp, col, ko, pivots=True)
    alt = oracle.ichol(xs, rp, col, ko, reverse_sums=(prec == kc.FP64), store_f32=(prec == kc.FP32_FORM))
    pat = kc.schedule(T(rp), T(col), T(xs))
    val, diag, zp = kc.factor_blocked(pat, T(xs), kg, prec)
    assert val.dtype == (torch.float64 if prec == kc.FP64 else torch.float32)
    general = fam == 0 and nu not in (0.5, 1.5, 2.5)
    fp.check_factor(prec, H(val), H(diag), rp, col, np.sqrt(1.0 + nug), (val_ref, zc), alt=alt, piv=piv,
                    strict=strict, entries=strict or not (prec == kc.FP64 and general))
    assert _identity(xs, rp, col, H(val), ko) < fp.IDENTITY_BAR[prec] * (2.0 if general and prec == kc.FP64 else 1)
    # the diagonal the solves divide by: the FP64 pivots, zero where dropped
    dg = H(diag)
    assert np.array_equal(dg == 0.0, H(val)[rp[1:] - 1] == 0.0)
    if prec == kc.FP64:
        assert zp == int(zc.sum())
    # the same bits again
    v2, d2, z2 = kc.factor_blocked(pat, T(xs), kg, prec)
    assert torch.equal(v2, val) and torch.equal(d2, diag) and z2 == zp


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_blocked_factor_on_the_maximin_pattern(prec):
    """Every group is one column: Algorithm 2 column by column."""
    x = inputs.uniform(3000, 2, seed=155)
    perm, l, rp, col = oracle.sortsparse(x, 3.0)
    xo = x[perm]
    ko, kg = oracle.Kernel(0.5, 0.2), kc.Kernel(0.5, 0.2)
    val_ref, zc = oracle.ichol(xo, rp, col, ko)
    pat = kc.schedule(T(rp), T(col), T(xo))
    val, diag, zp = kc.factor_blocked(pat, T(xo), kg, prec)
    fp.check_factor(prec, H(val), H(diag), rp, col, 1.0, (val_ref, zc), strict=True)
    assert _identity(xo, rp, col, H(val), ko) < fp.IDENTITY_BAR[prec]


def test_blocked_agrees_with_the_column_kernel_and_solves():
    """On the supernodal pattern the block and the column-task kernels give
    the same factor within the FP64 bar; the solve with the block factor
    solves L L^T x = b."""
    from scipy.sparse import csr_matrix
    xs, ref = _supernodal_case(3000, 2, seed=156)
    rp, col = ref["rowptr"], ref["col"]
    kg = kc.Kernel(0.5, 0.2)
    pat = kc.schedule(T(rp), T(col), T(xs))
    vb, db, _ = kc.factor_blocked(pat, T(xs), kg, kc.FP64)
    vc, dc, _ = kc.factor(pat, T(xs), kg, kc.FP64)
    assert float((vb - vc).abs().max()) < 1e-12
    perm = torch.arange(3000, dtype=torch.int32, device=DEV)
    b = inputs.rhs(3000, 2, seed=157)
    xsol = H(kc.solve(pat, kc.FP64, vb, db, kg, perm, T(b)))
    v = H(vb).copy()
    v[rp[1:] - 1] = H(db)
    L = csr_matrix((v, col, rp), shape=(3000, 3000))
    for r in range(2):
        res = L @ (L.T @ xsol[r]) - b[r]
        assert np.linalg.norm(res) <= 1e-11 * np.linalg.norm(b[r])


def test_blocked_rejects_bad_options():
    xs, ref = _supernodal_case(500, 2, seed=158)
    pat = kc.schedule(T(ref["rowptr"]), T(ref["col"]), T(xs))
    with pytest.raises(kc.KcError):
        kc.factor_blocked(pat, T(xs), kc.Kernel(0.5, 0.2), kc.FP32_FORM, kc.make_opts(lanes_per_row=3))
    with pytest.raises(kc.KcError):
        kc.factor_blocked(pat, T(xs), kc.Kernel(0.5, 0.2), 7)


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
@pytest.mark.parametrize("d", [2, 3])
def test_blocked_same_bits_for_every_task_size(d, prec):
    """Rows per task only split the rows below a group among tasks, and the
    group detection only decides which columns form groups: the default
    choice, explicit sizes (odd, one row, longer than any column) and a
    second call give the same bits.  The coarsest columns here hold every
    later row, so the group detection's long comparisons run in many chunks."""
    xs, ref = _supernodal_case(3000 if d == 2 else 2500, d, seed=160 + d)
    kg = kc.Kernel(0.5, 0.2)
    pat = kc.schedule(T(ref["rowptr"]), T(ref["col"]), T(xs))
    v0, d0, z0 = kc.factor_blocked(pat, T(xs), kg, prec)
    for rpt in (1, 7, 64, 300, 512, 4096, 0):
        v, dg, z = kc.factor_blocked(pat, T(xs), kg, prec, kc.make_opts(rows_per_task=rpt))
        assert torch.equal(v, v0) and torch.equal(dg, d0) and z == z0, rpt
