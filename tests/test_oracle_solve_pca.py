"""Pins of the oracle's solves, refinement, PCA truncation and work counters.

* Triangular solves against SciPy's dense ``solve_triangular``.
* Theta^S v against the dense masked matrix built from SciPy's Bessel form.
* PCG (Section 4.3) against NumPy's dense solve, for A = Theta^S and A = Theta.
* PCA (Section 2.5) at rho = infinity: Eckart-Young (the error is at least
  lambda_{k+1}), the Schur complement Theta - L_k L_k^T is PSD, and the power
  iteration estimate is within 1% of the dense 2-norm.
* Work counters against brute-force set intersections in Python.
"""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle
from paper_1706_02205_gb300 import inputs
from tests import refmath


def _factor(N=800, d=2, nu=0.5, ell=0.2, rho=3.0, nugget=0.0, seed=71):
    x = inputs.uniform(N, d, seed=seed)
    kern = oracle.Kernel(nu, ell, 1.0, nugget)
    r = oracle.pipeline(x, rho, kern)
    return x, kern, r


def test_triangular_solves_vs_scipy():
    x, kern, r = _factor()
    rp, col, val = r["rowptr"], r["col"], r["val"]
    N = len(rp) - 1
    dg = oracle.solve_diag(r["x_ord"], rp, val, kern)
    L = refmath.dense_lower(rp, col, val, N)
    L[np.diag_indices(N)] = dg
    b = inputs.rhs(N, 1, seed=3)[0]
    y = oracle.solve_lower(rp, col, val, dg, b)
    np.testing.assert_allclose(y, solve_triangular(L, b, lower=True), rtol=1e-12, atol=1e-12)
    z = oracle.solve_upper(rp, col, val, dg, y)
    np.testing.assert_allclose(z, solve_triangular(L.T, y, lower=False), rtol=1e-11, atol=1e-11)


def test_theta_s_matvec_vs_dense_mask():
    x, kern, r = _factor(N=500, nu=1.5)
    rp, col, xo = r["rowptr"], r["col"], r["x_ord"]
    N = len(rp) - 1
    S = refmath.pattern_mask(rp, col, N)
    T = refmath.dense_theta(xo, 1.5, 0.2)
    v = inputs.rhs(N, 1, seed=4)[0]
    np.testing.assert_allclose(oracle.theta_s_matvec(xo, rp, col, kern, v), np.where(S, T, 0) @ v,
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.theta_dense_matvec(xo, kern, v), T @ v, rtol=1e-12, atol=1e-12)


def test_masked_theta_is_indefinite():
    """Theta^S (Theta masked to S) is not positive definite, so it cannot be the
    CG operator of the refinement: the refinement targets the dense Theta."""
    x, kern, r = _factor(N=1000, nu=0.5, ell=0.2, rho=3.0)
    rp, col, xo = r["rowptr"], r["col"], r["x_ord"]
    T = refmath.dense_theta(xo, 0.5, 0.2)
    A = np.where(refmath.pattern_mask(rp, col, len(rp) - 1), T, 0)
    assert np.linalg.eigvalsh(A)[0] < -1.0
    dg = oracle.solve_diag(xo, rp, r["val"], kern)
    b = inputs.rhs(len(rp) - 1, 1, seed=5)[0]
    _, _, _, st = oracle.pcg(xo, rp, col, r["val"], dg, kern, b, op=1, rtol=1e-10, maxit=50)
    assert st == 2                      # nonpositive curvature detected


@pytest.mark.parametrize("nu,ell,rho", [(0.5, 0.2, 3.0), (1.5, 0.2, 3.0)])
def test_pcg_vs_dense_solve(nu, ell, rho):
    op = 2
    x, kern, r = _factor(N=1000, nu=nu, ell=ell, rho=rho)
    rp, col, val, xo = r["rowptr"], r["col"], r["val"], r["x_ord"]
    N = len(rp) - 1
    dg = oracle.solve_diag(xo, rp, val, kern)
    A = refmath.dense_theta(xo, nu, ell)
    b = inputs.rhs(N, 1, seed=5)[0]
    sol, it, relres, st = oracle.pcg(xo, rp, col, val, dg, kern, b, op=op, rtol=1e-10, maxit=300)
    # the recursive residual reaches 1e-10; the true residual may sit a little
    # above it at the FP64 floor of an ill-conditioned Theta
    assert st == 0 and relres <= 1e-9, (st, relres, it)
    ref = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(sol - ref) / np.linalg.norm(ref) <= 1e-10 * kappa


@pytest.mark.parametrize("k", [8, 40])
def test_pca_rank_k_bounds(k):
    N = 400
    x = inputs.uniform(N, 2, seed=81)
    kern = oracle.Kernel(1.5, 0.3, 1.0, 1e-6)
    perm, l = oracle.maximin_brute(x)
    rp, col = oracle.pattern(x[perm], l, 1e300)
    val, zc = oracle.ichol(x[perm], rp, col, kern)
    assert not zc.any()
    Lk = oracle.pca_truncate(rp, col, val, perm, k)          # (k, N), original order
    # the scatter puts column a of L (ordered rows) at the original rows
    L = refmath.dense_lower(rp, col, val, N)
    np.testing.assert_array_equal(Lk[:, perm], L[:, :k].T)
    T = refmath.dense_theta(x, 1.5, 0.3, 1.0, 1e-6)
    B = T - Lk.T @ Lk
    lam = np.linalg.eigvalsh(T)[::-1]
    eb = np.linalg.eigvalsh(B)
    assert eb.min() > -1e-10                                   # Schur complement is PSD
    two = eb.max()
    assert two >= lam[k] * (1 - 1e-9)                          # Eckart-Young
    v0 = inputs.unit_vector(N, seed=6)
    est = oracle.pca_error_power(x, kern, Lk, v0, iters=50)
    assert abs(est / two - 1) < 0.01, (est, two)


def test_work_counters_brute():
    x, kern, r = _factor(N=300, rho=2.5)
    rp, col = r["rowptr"], r["col"]
    N = len(rp) - 1
    R = [set(col[rp[j]:rp[j + 1] - 1].tolist()) for j in range(N)]
    F = M = P = Rs = 0
    for j in range(N):
        Rs += len(R[j])
        for i in R[j]:
            F += len(R[j] & R[i])
            pre = len([k for k in R[j] if k < i])
            P += pre
            M += pre + len(R[i])
    F += Rs
    c = oracle.work_counters(rp, col)
    assert c == dict(F=F, M=M, P=P, Rsum=Rs)
