"""Pins of the oracle's other covariance functions and of tasks (1), (3), (4).

* K_nu from the integral representation against SciPy's ``kv`` and against
  the elementary closed forms of half-integer order.
* Matern with general nu against the Bessel definition (SciPy), continuity
  at the closed-form orders, value sigma2 at r = 0.
* Cauchy class (Section 4.4): the special cases alpha = 2, beta = 2
  (1 / (1 + (r/l)^2)) and alpha = 1, beta = 1 (1 / (1 + r/l)).
* rho = infinity with these kernels: ICHOL(0) is the dense Cholesky factor
  of Theta built with SciPy (NumPy/LAPACK).
* L z and L^T v against dense NumPy products; 2 sum log L_ii against
  NumPy's slogdet of Theta (rho = infinity) and of L L^T (sparse pattern);
  dropped columns counted.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs
from tests import refmath

scipy_special = pytest.importorskip("scipy.special")


@pytest.mark.parametrize("nu", [0.01, 0.1, 0.3, 0.5, 0.75, 1.0, 1.01, 1.5, 1.98, 2.2, 3.7, 7.5, 9.3, 20.5])
def test_bessel_k_vs_scipy(nu):
    x = np.geomspace(1e-6, 300.0, 120)
    got = np.array([oracle.bessel_k(nu, v) for v in x])
    want = scipy_special.kv(nu, x)
    m = want < 1e300  # SciPy's range
    np.testing.assert_allclose(got[m], want[m], rtol=2e-13)


@pytest.mark.parametrize("nu", [0.3, 1.01, 3.7, 20.5])
def test_bessel_k_scaled_vs_scipy(nu):
    """e^x K_nu(x) against SciPy's kve, out to x where K_nu underflows."""
    x = np.geomspace(1e-4, 5000.0, 200)
    got = np.array([oracle.bessel_k_scaled(nu, v) for v in x])
    want = scipy_special.kve(nu, x)
    m = want < 1e300
    np.testing.assert_allclose(got[m], want[m], rtol=2e-13)


def test_matern_far_tail_vs_bessel():
    """Where K_nu(t) is below the normal double range the Matern value is
    still right (e^{-t} taken with the other factors)."""
    from scipy.special import gammaln
    for nu in (3.3, 20.5):
        t = np.linspace(500.0, 720.0, 40)
        r = t * 0.1 / np.sqrt(2 * nu)
        want = np.exp((1 - nu) * np.log(2) - gammaln(nu) + nu * np.log(t) - t) * scipy_special.kve(nu, t)
        got = np.array([oracle.matern(v, nu, 0.1) for v in r])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def test_bessel_k_half_integer_closed_forms():
    x = np.geomspace(1e-4, 200.0, 80)
    base = np.sqrt(np.pi / (2 * x)) * np.exp(-x)
    np.testing.assert_allclose([oracle.bessel_k(0.5, v) for v in x], base, rtol=1e-14)
    np.testing.assert_allclose([oracle.bessel_k(1.5, v) for v in x], base * (1 + 1 / x), rtol=1e-14)
    np.testing.assert_allclose([oracle.bessel_k(2.5, v) for v in x], base * (1 + 3 / x + 3 / x**2), rtol=1e-14)


@pytest.mark.parametrize("nu", [0.2, 0.8, 1.2, 2.0, 3.3])
def test_matern_general_nu_vs_bessel(nu):
    r = np.concatenate([[0.0], np.geomspace(1e-6, 4.0, 150)])
    for ell in (0.05, 0.3):
        want = refmath.matern_general(r, nu, ell, 1.3)
        got = np.array([oracle.matern(v, nu, ell, 1.3) for v in r])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)
    assert oracle.matern(0.0, nu, 0.3, 1.3) == 1.3


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_general_branch_continuous_at_closed_forms(nu):
    """The integral branch just beside a closed-form order agrees with it."""
    r = np.geomspace(1e-4, 2.0, 40)
    for dn in (-1e-9, 1e-9):
        got = np.array([oracle.matern(v, nu + dn, 0.2) for v in r])
        want = np.array([oracle.matern(v, nu, 0.2) for v in r])
        np.testing.assert_allclose(got, want, rtol=1e-7)


def test_cauchy_special_cases():
    r = np.concatenate([[0.0], np.geomspace(1e-5, 50.0, 100)])
    for ell in (0.2, 0.4):
        np.testing.assert_allclose([oracle.cauchy(v, ell, 2.0, 2.0) for v in r], 1.0 / (1.0 + (r / ell) ** 2),
                                   rtol=1e-15)
        np.testing.assert_allclose([oracle.cauchy(v, ell, 1.0, 1.0, 2.5) for v in r], 2.5 / (1.0 + r / ell),
                                   rtol=1e-15)
    # the paper's parameters: slow (algebraic) decay, value sigma2 at 0
    k = oracle.Kernel(family=oracle.CAUCHY, ell=0.4, alpha=0.5, beta=0.025)
    assert oracle.cov(0.0, k) == 1.0
    assert oracle.cov(1e6, k) > 0.5 * (1e6 / 0.4) ** -0.025


KERNELS = [
    ("cauchy_0.4_0.5_0.025", oracle.Kernel(family=oracle.CAUCHY, ell=0.4, alpha=0.5, beta=0.025, nugget=1e-3)),
    ("cauchy_0.2_1_0.2", oracle.Kernel(family=oracle.CAUCHY, ell=0.2, alpha=1.0, beta=0.2, nugget=1e-4)),
    ("matern_0.8", oracle.Kernel(0.8, 0.2, 1.0, 1e-4)),
    ("matern_1.2", oracle.Kernel(1.2, 0.3, 1.0, 1e-3)),
]


@pytest.mark.parametrize("name,kern", KERNELS, ids=[k[0] for k in KERNELS])
def test_rho_infinity_dense_cholesky_other_kernels(name, kern):
    N = 300
    x = inputs.uniform(N, 2, seed=71)
    perm, l, rp, col = oracle.sortsparse(x, 1e300)
    xo = x[perm]
    val, zc = oracle.ichol(xo, rp, col, kern)
    assert not zc.any()
    L = refmath.dense_lower(rp, col, val, N)
    C = np.linalg.cholesky(refmath.dense_cov(xo, kern))
    nrm = np.linalg.norm(C, axis=1)
    assert np.max(np.abs(L - C) / nrm[:, None]) < 1e-9


def _factor(N=600, rho=3.0, nu=1.5, ell=0.2, seed=72, nugget=0.0):
    x = inputs.uniform(N, 2, seed=seed)
    perm, l, rp, col = oracle.sortsparse(x, rho)
    xo = x[perm]
    kern = oracle.Kernel(nu, ell, 1.0, nugget)
    val, zc = oracle.ichol(xo, rp, col, kern)
    return xo, rp, col, val, zc, kern


def test_l_and_lt_matvec_vs_dense():
    xo, rp, col, val, zc, kern = _factor()
    N = xo.shape[0]
    L = refmath.dense_lower(rp, col, val, N)
    r = inputs.rng(73)
    z = r.standard_normal(N)
    np.testing.assert_allclose(oracle.l_matvec(rp, col, val, z), L @ z, rtol=0, atol=1e-13 * np.abs(L).sum(1).max())
    np.testing.assert_allclose(oracle.lt_matvec(rp, col, val, z), L.T @ z, rtol=0,
                               atol=1e-13 * np.abs(L).sum(0).max())
    # task (1): L (L^T v) reproduces Theta v at rho = infinity
    x = inputs.uniform(300, 2, seed=74)
    perm, l, rp2, col2 = oracle.sortsparse(x, 1e300)
    kern2 = oracle.Kernel(1.5, 0.2, 1.0, 1e-3)
    val2, _ = oracle.ichol(x[perm], rp2, col2, kern2)
    v = r.standard_normal(300)
    got = oracle.l_matvec(rp2, col2, val2, oracle.lt_matvec(rp2, col2, val2, v))
    want = refmath.dense_theta(x[perm], 1.5, 0.2, 1.0, 1e-3) @ v
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_logdet_full_pattern_is_slogdet_of_theta():
    x = inputs.uniform(300, 2, seed=75)
    perm, l, rp, col = oracle.sortsparse(x, 1e300)
    xo = x[perm]
    kern = oracle.Kernel(0.5, 0.2, 1.0, 1e-4)
    val, zc = oracle.ichol(xo, rp, col, kern)
    ld, z = oracle.logdet(rp, val)
    sign, want = np.linalg.slogdet(refmath.dense_theta(xo, 0.5, 0.2, 1.0, 1e-4))
    assert z == 0 and sign == 1.0
    assert abs(ld - want) <= 1e-10 * abs(want)


def test_logdet_sparse_pattern_is_slogdet_of_llt_and_counts_drops():
    xo, rp, col, val, zc, kern = _factor(N=600, rho=3.0, nu=0.5, ell=0.2)
    assert not zc.any()
    L = refmath.dense_lower(rp, col, val, xo.shape[0])
    ld, z = oracle.logdet(rp, val)
    sign, want = np.linalg.slogdet(L @ L.T)
    assert z == 0 and sign == 1.0 and abs(ld - want) <= 1e-9 * abs(want)
    # Matern-3/2 at rho = 2 drops pivots: they are counted, the rest summed
    xo, rp, col, val, zc, kern = _factor(N=2000, rho=2.0, nu=1.5, ell=0.2, seed=inputs.seed_for(1))
    ld, z = oracle.logdet(rp, val)
    assert z == int(zc.sum()) > 0
    dg = val[rp[1:] - 1]
    assert abs(ld - 2 * math.fsum(np.log(dg[dg > 0]))) <= 1e-12 * abs(ld)


def test_ichol_float_storage_mode():
    """store_f32: every off-diagonal entry is a float, each satisfies its
    defining equation L_ji L_ii = float(Theta_ji) - sum_k L_jk L_ik to the
    float rounding of L_ji, and the factor stays within float-level distance
    of the FP64 one."""
    xo, rp, col, val, zc, kern = _factor(N=800, rho=3.0, nu=0.5, ell=0.2, seed=76)
    v32, zc32 = oracle.ichol(xo, rp, col, kern, store_f32=True)
    off = np.ones(len(col), bool)
    off[rp[1:] - 1] = False
    assert np.array_equal(v32[off], v32[off].astype(np.float32).astype(np.float64))
    L = refmath.dense_lower(rp, col, v32, xo.shape[0])
    Th = refmath.dense_theta(xo, 0.5, 0.2)
    rows = np.repeat(np.arange(xo.shape[0]), np.diff(rp))
    for e in np.nonzero(off)[0][::37]:
        j, i = rows[e], col[e]
        s = float(np.float32(Th[j, i])) - L[j, :i] @ L[i, :i]
        assert abs(v32[e] * L[i, i] - s) <= (2.0**-24 * abs(v32[e]) + 1e-15) * L[i, i] + 1e-14, e
    assert np.max(np.abs(v32 - val)) < 1e-4 and not zc32.any()


@pytest.mark.parametrize("name,kern", KERNELS + [("matern_2.5", oracle.Kernel(2.5, 0.3, 1.7, 1e-2))],
                         ids=[k[0] for k in KERNELS] + ["matern_2.5"])
def test_theta_entries_vs_dense(name, kern):
    """Single entries Theta_ab (nugget on the diagonal only) equal the dense
    matrix built from SciPy's Bessel function / NumPy."""
    x = inputs.uniform(60, 3, seed=77)
    T = refmath.dense_cov(x, kern)
    got = np.array([[oracle.theta(x, a, b, kern) for b in range(60)] for a in range(60)])
    np.testing.assert_allclose(got, T, rtol=1e-12, atol=0)
