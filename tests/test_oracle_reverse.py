"""Pins of the oracle's Section 6 path: ICHOL(0) of a given sparse matrix
(the precision matrix A = Theta^{-1}, or sigma^2 A + I for a nugget) in the
reverse maximin order on the min-rule pattern.

* rho = infinity: the factor is LAPACK's dense Cholesky factor of P A P.
* ICHOL(0) restated as a dense Cholesky with the Schur-complement updates
  masked to the pattern (tests/refmath.py)
  on P A P masked to the reversed pattern equals the oracle's left-looking
  factor.
* The reversed pattern is the maximin pattern flipped in both indices (dense
  masks); the gathered entries are A's at the permuted positions, and the
  count of A's entries outside the pattern is exact.
* Section 6's claim on a rough-coefficient grid operator: the error of the
  reverse-order factor falls fast with rho and ends far below the error of
  the same pattern factored in the forward (maximin) order.
* The nugget decomposition (Section 4.3, "Nuggets"): with Theta = A^{-1},
  (Theta + sigma^2 I)^{-1} b = (sigma^2 A + I)^{-1} A b, the factor of
  P (sigma^2 A + I) P solving the dense system at rho = infinity.
"""
import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs
from tests import refmath


def _dense(rp, col, val, N):
    A = np.zeros((N, N))
    for j in range(N):
        A[j, col[rp[j]:rp[j + 1]]] = val[rp[j]:rp[j + 1]]
    return A


def _op(n=16, seed=inputs.seed_for(6)):
    x, rp, col, val = inputs.grid_operator(n, seed=seed)
    return x, rp, col, val, _dense(rp, col, val, n * n)


def test_rho_infinity_is_dense_cholesky_of_reversed_matrix():
    x, rp, col, val, A = _op(14)
    N = A.shape[0]
    r = oracle.reverse_factor(x, rp, col, val, 1e300)
    assert r["outside"] == 0 and not r["zero_col"].any()
    L = refmath.dense_lower(r["rowptr"], r["col"], r["val"], N)
    C = np.linalg.cholesky(A[np.ix_(r["orig"], r["orig"])])
    assert np.max(np.abs(L - C)) <= 1e-12 * np.max(np.abs(C))
    # the order really is reversed: position 0 holds the last maximin point
    assert r["orig"][0] == r["perm"][-1] and r["orig"][-1] == r["perm"][0] == 0


@pytest.mark.parametrize("rho", [1.5, 2.0, 3.0])
def test_matches_masked_schur_cholesky_on_reversed_matrix(rho):
    x, rp, col, val, A = _op(12)
    N = A.shape[0]
    r = oracle.reverse_factor(x, rp, col, val, rho)
    S = refmath.pattern_mask(r["rowptr"], r["col"], N)
    L_ref = refmath.ichol_masked_schur(A[np.ix_(r["orig"], r["orig"])], S)
    L = refmath.dense_lower(r["rowptr"], r["col"], r["val"], N)
    assert np.max(np.abs(L - L_ref)) <= 1e-12 * np.max(np.abs(L_ref))


def test_reverse_pattern_and_gather():
    x, rp, col, val, A = _op(10)
    N = A.shape[0]
    perm, l = oracle.maximin_brute(x)
    frp, fcol = oracle.pattern(x[perm], l, 2.0, oracle.RULE_MIN)
    colptr, rowidx, _ = oracle.csr_to_csc(frp, fcol)
    rrp, rcol = oracle.pattern_reverse(colptr, rowidx)
    Mf = refmath.pattern_mask(frp, fcol, N)
    Mr = refmath.pattern_mask(rrp, rcol, N)
    assert np.array_equal(Mr, Mf[::-1, ::-1])
    assert all(rcol[rrp[q + 1] - 1] == q for q in range(N))  # diagonal last
    assert all(np.all(np.diff(rcol[rrp[q]:rrp[q + 1]]) > 0) for q in range(N))
    orig = np.ascontiguousarray(perm[::-1])
    aval, outside = oracle.gather_entries(rrp, rcol, orig, rp, col, val)
    rows = np.repeat(np.arange(N), np.diff(rrp))
    assert np.array_equal(aval, A[orig[rows], orig[rcol]])
    PAP = A[np.ix_(orig, orig)]
    assert outside == int(np.count_nonzero((PAP != 0) & ~Mr & ~np.eye(N, dtype=bool)))
    # a pattern too small for the operator: entries outside are counted
    frp1, fcol1 = oracle.pattern(x[perm], l, 0.5, oracle.RULE_MIN)
    c1, r1, _ = oracle.csr_to_csc(frp1, fcol1)
    rrp1, rcol1 = oracle.pattern_reverse(c1, r1)
    _, out1 = oracle.gather_entries(rrp1, rcol1, orig, rp, col, val)
    M1 = refmath.pattern_mask(rrp1, rcol1, N)
    assert out1 == int(np.count_nonzero((PAP != 0) & ~M1 & ~np.eye(N, dtype=bool))) > 0


def test_reverse_order_beats_forward_order():
    """Section 6: the Cholesky factors of the precision matrix decay in the
    reverse elimination order."""
    x, rp, col, val, A = _op(24)
    N = A.shape[0]
    nA = np.linalg.norm(A)
    errs = []
    for rho in (1.5, 2.0, 3.0, 4.0, 6.0):
        r = oracle.reverse_factor(x, rp, col, val, rho)
        L = refmath.dense_lower(r["rowptr"], r["col"], r["val"], N)
        errs.append(np.linalg.norm(A[np.ix_(r["orig"], r["orig"])] - L @ L.T) / nA)
    assert all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-2 * errs[0]
    # forward order, the same (min-rule) pattern
    perm, l = r["perm"], r["l"]
    frp, fcol = oracle.pattern(x[perm], l, 6.0, oracle.RULE_MIN)
    av, _ = oracle.gather_entries(frp, fcol, perm.astype(np.int32), rp, col, val)
    vf, _ = oracle.ichol_given(frp, fcol, av)
    Lf = refmath.dense_lower(frp, fcol, vf, N)
    err_fwd = np.linalg.norm(A[np.ix_(perm, perm)] - Lf @ Lf.T) / nA
    assert errs[-1] < 0.1 * err_fwd


def test_nugget_decomposition_solves_theta_plus_sigma2():
    x, rp, col, val, A = _op(12)
    N = A.shape[0]
    sigma2 = 0.3
    # sigma^2 A + I as CSR (same structure as A)
    val_n = sigma2 * val
    dpos = np.array([rp[j] + np.nonzero(col[rp[j]:rp[j + 1]] == j)[0][0] for j in range(N)])
    val_n[dpos] += 1.0
    r = oracle.reverse_factor(x, rp, col, val_n, 1e300)
    b = inputs.rhs(N, 1, seed=3)[0]
    # (Theta + sigma^2 I) x = b with Theta = A^{-1}  <=>  (sigma^2 A + I) x = A b
    rhs = A @ b
    o = r["orig"]
    dg = oracle.diag_of(r["rowptr"], r["val"])
    y = oracle.solve_lower(r["rowptr"], r["col"], r["val"], dg, rhs[o])
    z = oracle.solve_upper(r["rowptr"], r["col"], r["val"], dg, y)
    xs = np.empty(N)
    xs[o] = z
    want = np.linalg.solve(np.linalg.inv(A) + sigma2 * np.eye(N), b)
    assert np.linalg.norm(xs - want) <= 1e-10 * np.linalg.norm(want)
