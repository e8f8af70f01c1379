"""GPU parity for Section 6: factors of a given sparse matrix (a
rough-coefficient grid operator standing in for the precision matrix
A = Theta^{-1}) in the reverse maximin order on the min-rule pattern.

Bars: the reversed pattern, the gathered entries and the count of entries
outside the pattern bit-exact; factors within the row-norm bars of the
kernel factors (norm sqrt(A_jj)); solves within 20x the oracle's own shift
under the rounding the GPU factor carries, and by their residual with the
GPU's own factor.
"""
import math

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


def _op(n, seed=inputs.seed_for(6)):
    x, rp, col, val = inputs.grid_operator(n, seed=seed)
    return x, rp, col, val


@pytest.mark.parametrize("rho", [0.5, 2.0, 3.0])
def test_reverse_pattern_and_gather_bit_exact(rho):
    x, rp, col, val = _op(40)
    r_ref = oracle.reverse_factor(x, rp, col, val, rho)
    perm, l, xo = kc.order_points(T(x))
    assert np.array_equal(H(perm), r_ref["perm"])
    pat = kc.build_pattern(xo, l, rho, kc.RULE_MIN)
    rpat = kc.pattern_reverse(pat, xo)
    assert np.array_equal(H(rpat.rowptr), r_ref["rowptr"]) and np.array_equal(H(rpat.col), r_ref["col"])
    orig = perm.flip(0).contiguous()
    aval, outside = kc.gather_entries(rpat, orig, T(rp), T(col), T(val))
    assert np.array_equal(H(aval), r_ref["aval"])
    assert outside == r_ref["outside"]
    if rho < 1:
        assert outside > 0


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
@pytest.mark.parametrize("rho", [2.0, 4.0])
def test_reverse_factor_matches_oracle(prec, rho):
    x, rp, col, val = _op(48)
    ref = oracle.reverse_factor(x, rp, col, val, rho)
    r = kc.reverse_factor(T(x), T(rp), T(col), T(val), rho, prec)
    assert np.array_equal(H(r["orig"]), ref["orig"])
    assert np.array_equal(H(r["pat"].col), ref["col"])
    assert r["outside"] == ref["outside"] == 0 and r["zero_pivots"] == int(ref["zero_col"].sum()) == 0
    rrp, rcol = ref["rowptr"], ref["col"]
    dpos = ref["aval"][rrp[1:] - 1]
    # every pivot of the shifted grid operator is far from zero: the fixed
    # bars hold on every entry and on the FP64 pivots
    fp.check_factor(prec, H(r["val"]), H(r["diag"]), rrp, rcol, np.sqrt(dpos), (ref["val"], ref["zero_col"]),
                    strict=True)
    np.testing.assert_allclose(H(r["diag"]), ref["val"][rrp[1:] - 1], rtol=fp.BAR[prec])
    # the defining identity (L L^T)_ji = A_ji on the pattern
    N = x.shape[0]
    L = refmath.dense_lower(rrp, rcol, H(r["val"]).astype(np.float64), N)
    L[np.arange(N), np.arange(N)] = H(r["diag"])
    rows = np.repeat(np.arange(N), np.diff(rrp))
    LLt = (L @ L.T)[rows, rcol]
    tol = 1e-12 if prec == kc.FP64 else 1e-6
    assert np.max(np.abs(LLt - ref["aval"]) / np.sqrt(dpos[rows] * dpos[rcol])) < tol


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_reverse_solve(prec):
    """A x = b with the reverse-order factor: against the oracle's solve on
    its own factor, the residual with the GPU factor, and the error against
    A^{-1} b falling with rho (Section 6: a direct solver)."""
    from scipy.sparse import csr_matrix
    x, rp, col, val = _op(40)
    N = x.shape[0]
    A = csr_matrix((val, col, rp), shape=(N, N))
    anorm = float(np.max(np.abs(A).sum(axis=1)))  # >= ||A||_2 (symmetric)
    b = inputs.rhs(N, 2, seed=inputs.seed_for(6, 1))
    exact = [np.linalg.solve(A.toarray(), b[k]) for k in range(2)]
    errs = []
    for rho in (2.0, 3.0, 5.0):
        ref = oracle.reverse_factor(x, rp, col, val, rho)
        r = kc.reverse_factor(T(x), T(rp), T(col), T(val), rho, prec)
        dmax = float(np.max(ref["aval"][ref["rowptr"][1:] - 1]))
        xs = H(kc.solve(r["pat"], prec, r["val"], r["diag"], kc.Kernel(sigma2=dmax), r["orig"], T(b)))
        rrp, rcol, o = ref["rowptr"], ref["col"], ref["orig"]
        alt = (oracle.ichol_given(rrp, rcol, ref["aval"], reverse_sums=True)[0] if prec == kc.FP64
               else oracle.ichol_given(rrp, rcol, ref["aval"], store_f32=True)[0])

        def osolve(vals, rhs):
            dg = oracle.diag_of(rrp, vals)
            z = oracle.solve_upper(rrp, rcol, vals, dg, oracle.solve_lower(rrp, rcol, vals, dg, rhs[o]))
            out = np.empty(N)
            out[o] = z
            return out

        v = H(r["val"]).astype(np.float64).copy()
        v[rrp[1:] - 1] = H(r["diag"])
        Lg = csr_matrix((v, rcol, rrp), shape=(N, N))
        for k in range(2):
            z = osolve(ref["val"], b[k])
            shift = np.linalg.norm(osolve(alt, b[k]) - z) / np.linalg.norm(z)
            assert np.linalg.norm(xs[k] - z) / np.linalg.norm(z) <= max(1e-12, 20 * shift), (rho, k, shift)
            # backward-error scale: u ||A|| ||x|| with the solve's unit roundoff
            # (FP64: 2^-53; FP32 form: its float-pair vectors, about 2^-45)
            res = Lg @ (Lg.T @ xs[k][o]) - b[k][o]
            u = 2.0**-53 if prec == kc.FP64 else 2.0**-45
            assert np.linalg.norm(res) <= 64 * u * anorm * np.linalg.norm(xs[k])
        errs.append(max(np.linalg.norm(xs[k] - exact[k]) / np.linalg.norm(exact[k]) for k in range(2)))
    assert errs[0] > errs[1] > errs[2]


def test_nugget_decomposition_on_gpu():
    """(Theta + sigma^2 I) x = b with Theta = A^{-1}: x = (sigma^2 A + I)^{-1} A b,
    the factor of P (sigma^2 A + I) P from the device at rho = infinity."""
    from scipy.sparse import csr_matrix
    x, rp, col, val = _op(20)
    N = x.shape[0]
    sigma2 = 0.3
    val_n = sigma2 * val
    dpos = np.array([rp[j] + np.nonzero(col[rp[j]:rp[j + 1]] == j)[0][0] for j in range(N)])
    val_n[dpos] += 1.0
    r = kc.reverse_factor(T(x), T(rp), T(col), T(val_n), 1e300, kc.FP64)
    assert r["zero_pivots"] == 0
    A = csr_matrix((val, col, rp), shape=(N, N))
    b = inputs.rhs(N, 1, seed=5)
    Ab = np.stack([A @ b[0]])
    xs = H(kc.solve(r["pat"], kc.FP64, r["val"], r["diag"], kc.Kernel(sigma2=1.0), r["orig"], T(Ab)))[0]
    want = np.linalg.solve(np.linalg.inv(A.toarray()) + sigma2 * np.eye(N), b[0])
    assert np.linalg.norm(xs - want) <= 1e-10 * np.linalg.norm(want)


def test_factor_given_errors():
    x, rp, col, val = _op(8)
    r = kc.reverse_factor(T(x), T(rp), T(col), T(val), 2.0, kc.FP64)
    with pytest.raises(kc.KcError):
        kc.factor_given(r["pat"], r["aval"], prec=7)


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_refine_sparse_reaches_the_solution(prec):
    """CG on the given A preconditioned by its reverse-order factor reaches
    A^{-1} b (SciPy's sparse direct solve) to the accuracy its residual
    allows, and reports that residual."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.linalg import spsolve
    x, rp, col, val = _op(60)
    N = x.shape[0]
    A = csr_matrix((val, col, rp), shape=(N, N))
    kappa = np.linalg.cond(A.toarray())
    b = inputs.rhs(N, 3, seed=inputs.seed_for(6, 3))
    r = kc.reverse_factor(T(x), T(rp), T(col), T(val), 2.0, prec)
    xs, it, rr, st = kc.refine_sparse(r["pat"], prec, r["val"], r["diag"], r["orig"], T(rp), T(col), T(val), T(b),
                                      rtol=1e-10, maxit=300)
    assert st == kc.KC_OK, (it, rr)
    xs = H(xs)
    for k in range(3):
        true = np.linalg.norm(A @ xs[k] - b[k]) / np.linalg.norm(b[k])
        assert true <= 2e-10 and abs(rr[k] - true) <= 1e-12 + 1e-3 * true
        ex = spsolve(A.tocsc(), b[k])
        assert np.linalg.norm(xs[k] - ex) / np.linalg.norm(ex) <= 2e-10 * kappa
    # a better factor (larger rho) needs no more iterations
    r3 = kc.reverse_factor(T(x), T(rp), T(col), T(val), 4.0, prec)
    _, it3, _, st3 = kc.refine_sparse(r3["pat"], prec, r3["val"], r3["diag"], r3["orig"], T(rp), T(col), T(val),
                                      T(b), rtol=1e-10, maxit=300)
    assert st3 == kc.KC_OK and it3 <= it
