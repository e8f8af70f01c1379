"""GPU parity for the covariance families beyond the closed-form Matern
kernels, and for tasks (1), (3), (4) of Section 1 with the factor.

Bars.  Entries (kc_kernel_eval): FP64 within 1e-12 relative of the oracle
(Temme/Steed against the integral representation); FP32 form within 3e-6
relative plus 2^-24 times the sensitivity of G to the rounded distance.  Factors: as for the
closed-form kernels (row-norm bars of 1e-12 in FP64, the FP32-form bar, the
identity L L^T = Theta on S).  Tasks: the GPU result on the GPU factor
against the oracle's result on the oracle's own factor within the bound the
factor bar implies (triangle inequality), and against an FP64 NumPy product
of the GPU's own factor within rounding (the kernel's arithmetic alone).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs
from tests import refmath

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


def pair(family=0, nu=1.5, ell=0.2, nugget=0.0, alpha=1.0, beta=1.0):
    return (kc.Kernel(nu, ell, 1.0, nugget, family, alpha, beta),
            oracle.Kernel(nu, ell, 1.0, nugget, family, alpha, beta))


FAMILIES = [
    ("matern_0.5", dict(nu=0.5, ell=0.2)),
    ("matern_0.8", dict(nu=0.8, ell=0.2, nugget=1e-6)),
    ("matern_1.2", dict(nu=1.2, ell=0.1)),
    ("matern_3.7", dict(nu=3.7, ell=0.3, nugget=1e-4)),
    ("cauchy_0.4_0.5_0.025", dict(family=1, ell=0.4, alpha=0.5, beta=0.025, nugget=1e-3)),
    ("cauchy_0.2_1_0.2", dict(family=1, ell=0.2, alpha=1.0, beta=0.2, nugget=1e-4)),
    ("cauchy_0.1_2_1", dict(family=1, ell=0.1, alpha=2.0, beta=1.0)),
]


# ------------------------------------------------------------- entries alone

@pytest.mark.parametrize("name,kw", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_kernel_eval_matches_oracle(name, kw):
    kg, ko = pair(**kw)
    r = np.concatenate([[0.0], np.geomspace(1e-7, 30.0, 3001)])
    want = np.array([oracle.cov(v, ko) for v in r])
    got = H(kc.kernel_eval(kg, kc.FP64, T(r)))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)
    got32 = H(kc.kernel_eval(kg, kc.FP32_FORM, T(r)))
    # the FP32 form rounds r to float (relative 2^-24): G moves by at most
    # |d ln G / d ln r| 2^-24 relative, which is <= t for the Matern class
    # (-d ln(t^nu K_nu)/dt = K_{nu-1}/K_nu <= 1 for nu >= 1/2) and <= beta for
    # the Cauchy class; a few float roundings come on top
    sens = kw.get("beta", 1.0) * np.ones_like(r) if kw.get("family") == 1 else \
        math.sqrt(2 * kw["nu"]) * r / kw["ell"]
    big = want > 1e-30  # below that the float result may underflow
    err = np.abs(got32 - want)[big] / want[big]
    assert np.all(err <= 3e-6 + 1.2e-7 * sens[big]), err.max()
    assert got[0] == 1.0 and got32[0] == 1.0


@pytest.mark.parametrize("nu", [0.01, 0.3, 1.01, 1.98, 2.0, 4.4, 7.9, 9.3, 20.5])
def test_kernel_eval_every_branch(nu):
    """Orders that take each evaluation path: the power series (t <= 2) or
    Temme's series (nu within 0.02 of an integer); the Chebyshev pieces
    (t > 2, nu <= 8) or Steed's continued fraction (nu > 8); zero beyond
    t = 1024."""
    kg, ko = pair(nu=nu, ell=0.1)
    t = np.concatenate([[0.0], np.geomspace(1e-6, 2.0, 400), np.linspace(2.0, 40.0, 800)[1:],
                        np.geomspace(40.0, 1100.0, 300)])
    r = t * 0.1 / math.sqrt(2 * nu)
    want = np.array([oracle.cov(v, ko) for v in r])
    got = H(kc.kernel_eval(kg, kc.FP64, T(r)))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)


def test_kernel_eval_empty_and_bad_args():
    kg, _ = pair(nu=0.8)
    assert kc.kernel_eval(kg, kc.FP64, torch.empty(0, dtype=torch.float64, device=DEV)).numel() == 0
    with pytest.raises(kc.KcError):
        kc.kernel_eval(kc.Kernel(nu=-1.0), kc.FP64, T(np.ones(4)))


# ------------------------------------------------------------------ factors

def _ref_pattern(N, rho, seed, d=2):
    x = inputs.uniform(N, d, seed=seed)
    perm, l, rp, col = oracle.sortsparse(x, rho)
    return x, perm, x[perm], rp, col


# Families held to the bars over every entry (no pivot near zero): Matern-0.8
# and 1.2, both Cauchy kernels with beta < 1.  Matern-3.7 (l = 0.3) and the
# Cauchy kernel with alpha = 2 (nearly Gaussian) drop most pivots and are
# checked on their determined columns plus the identity (tests/factor_parity.py).
WELL_CONDITIONED = {"matern_0.8", "matern_1.2", "cauchy_0.4_0.5_0.025", "cauchy_0.2_1_0.2"}
_FAM_ORACLE = {}


def _family_oracle(name, kw):
    if name not in _FAM_ORACLE:
        x, perm, xo, rp, col = _ref_pattern(2500, 3.0, seed=82)
        kg, ko = pair(**kw)
        val_ref, zc_ref, piv = oracle.ichol(xo, rp, col, ko, pivots=True)
        _FAM_ORACLE[name] = dict(xo=xo, rp=rp, col=col, kg=kg, ko=ko, ref=(val_ref, zc_ref), piv=piv,
                                 alt={0: oracle.ichol(xo, rp, col, ko, reverse_sums=True),
                                      1: oracle.ichol(xo, rp, col, ko, store_f32=True)})
    return _FAM_ORACLE[name]


def _identity(o, val):
    """(L L^T)_ji = Theta_ji on S over the kept columns, relative to Theta_jj;
    Theta from the covariance function's definition (SciPy's K_nu)."""
    N = o["xo"].shape[0]
    L = refmath.dense_lower(o["rp"], o["col"], H(val).astype(np.float64), N)
    Th = refmath.dense_cov(o["xo"], o["ko"])
    return fp.identity_residual_dense(L, Th, o["rp"], o["col"], 1.0 + o["ko"].nugget)


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
@pytest.mark.parametrize("name,kw", FAMILIES[1:], ids=[f[0] for f in FAMILIES[1:]])
def test_factor_other_kernels(name, kw, prec):
    o = _family_oracle(name, kw)
    pat = kc.schedule(T(o["rp"]), T(o["col"]))
    val, diag, zp = kc.factor(pat, T(o["xo"]), o["kg"], prec)
    if prec == kc.FP64:
        assert zp == int(o["ref"][1].sum())
    strict = name in WELL_CONDITIONED
    # FP64, a Matern of general nu: the device evaluates Theta from tables
    # held to 1e-12 relative (kc_kernel_eval's bar), which an ill-conditioned
    # factor amplifies beyond the entry bar; such a case is held to the pivot
    # decisions and the identity
    general_nu = kw.get("family", 0) == 0 and kw["nu"] not in (0.5, 1.5, 2.5)
    fp.check_factor(prec, H(val), H(diag), o["rp"], o["col"], math.sqrt(1.0 + o["ko"].nugget), o["ref"],
                    alt=o["alt"][prec], piv=o["piv"], strict=strict,
                    entries=strict or not (prec == kc.FP64 and general_nu))
    # FP64: the device's Theta of a general nu agrees with the definition to
    # 1e-12 relative (kc_kernel_eval's bar), which adds to the identity's 1e-12
    tol = fp.IDENTITY_BAR[prec] * (2.0 if prec == kc.FP64 and kw.get("family", 0) == 0 else 1.0)
    assert _identity(o, val) < tol


def test_factor_other_kernels_deterministic_and_3d():
    x, perm, xo, rp, col = _ref_pattern(2000, 3.0, seed=83, d=3)
    kg, ko = pair(nu=0.8, ell=0.3, nugget=1e-6)
    pat = kc.schedule(T(rp), T(col))
    a = kc.factor(pat, T(xo), kg, kc.FP32_FORM)
    b = kc.factor(pat, T(xo), kg, kc.FP32_FORM)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    val_ref, zc_ref = oracle.ichol(xo, rp, col, ko)
    val, diag, zp = kc.factor(pat, T(xo), kg, kc.FP64)
    assert zp == int(zc_ref.sum())
    alt = oracle.ichol(xo, rp, col, ko, reverse_sums=True)
    fp.check_factor(kc.FP64, H(val), H(diag), rp, col, math.sqrt(1.0 + 1e-6), (val_ref, zc_ref), alt=alt)


def test_batch_mixed_families_equal_sets_alone():
    """A batch whose sets use different covariance families runs the general
    kernel instantiation; each set's values equal the set factored alone."""
    from paper_1706_02205_gb300 import batch as kb
    sets = inputs.batch_sets(n_sets=4, n_min=400, n_max=1500, n_d3=1, seed=inputs.seed_for(4, 12))
    xs = [T(s["x"]) for s in sets]
    kerns = [kc.Kernel(1.5, 0.2), kc.Kernel(0.8, 0.15), kc.Kernel(family=kc.CAUCHY, ell=0.2, alpha=1.0, beta=0.2),
             kc.Kernel(2.5, 0.3)]
    for prec in (kc.FP64, kc.FP32_FORM):
        B = kb.BatchFactor(xs, kerns, 3.0, prec, n_streams=2)
        B.factor()
        for s, (x, k) in enumerate(zip(xs, kerns)):
            r = kc.pipeline(x, 3.0, k, prec)
            a, e = B.offsets[s], B.offsets[s + 1]
            # a closed-form set alone runs the closed-form instantiation, in the
            # batch the general one: same entry code, same merge order, same bits
            assert torch.equal(B.set_values(s), r["val"]), (prec, s)
            assert torch.equal(B.diag[a:e], r["diag"]), (prec, s)


@pytest.mark.parametrize("name,kw", [FAMILIES[2], FAMILIES[5]], ids=[FAMILIES[2][0], FAMILIES[5][0]])
def test_refine_other_kernels(name, kw):
    """CG on the dense Theta (entries from the same covariance code) reaches
    the dense FP64 solution."""
    N = 1500
    x = inputs.uniform(N, 2, seed=84)
    kg, ko = pair(**kw)
    perm, l, xo = kc.order_points(T(x))
    pat = kc.build_pattern(xo, l, 4.0)
    val, diag, zp = kc.factor(pat, xo, kg, kc.FP32_FORM)
    b = inputs.rhs(N, 1, seed=85)
    xs, it, rr, st = kc.refine(pat, xo, kg, kc.FP32_FORM, val, diag, perm, T(b), rtol=1e-10, maxit=400)
    assert st == kc.KC_OK, (st, it, rr)
    Th = refmath.dense_cov(x, ko)
    ref = np.linalg.solve(Th, b[0])
    kappa = np.linalg.cond(Th)
    assert np.linalg.norm(H(xs)[0] - ref) / np.linalg.norm(ref) < 1e-10 * kappa


# -------------------------------------------------------------------- tasks

def _task_case(N=2999, rho=3.0, seed=86, nu=0.5, ell=0.2, nugget=0.0):
    """A well-conditioned factor (every pivot kept, far from zero): the GPU
    factor is within the fixed bars of tests/factor_parity.py of the oracle's
    in every entry, which bounds the tasks' results."""
    x, perm, xo, rp, col = _ref_pattern(N, rho, seed)
    kg, ko = pair(nu=nu, ell=ell, nugget=nugget)
    val_ref, zc_ref = oracle.ichol(xo, rp, col, ko)
    pat = kc.schedule(T(rp), T(col))
    return x, perm, xo, rp, col, kg, ko, val_ref, zc_ref, pat


def _gpu_dense_L(rp, col, val, diag, N):
    """The GPU factor as the task kernels read it: off-diagonal values from
    val, the diagonal from the FP64 diag."""
    v = H(val).astype(np.float64).copy()
    v[rp[1:] - 1] = H(diag)
    return refmath.dense_lower(rp, col, v, N)


def _row_bound(rp, col, w, bar):
    """max_j sum_{k in row j} bar |w_k|: the change of (L w)_j when every entry
    of row j moves by at most bar (Theta_jj = 1 here)."""
    s = np.zeros(rp.shape[0] - 1)
    aw = np.abs(w)
    for j in range(rp.shape[0] - 1):
        s[j] = aw[col[rp[j]:rp[j + 1]]].sum()
    return bar * s.max()


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_l_and_lt_matvec(prec, nrhs):
    x, perm, xo, rp, col, kg, ko, val_ref, zc_ref, pat = _task_case()
    assert not zc_ref.any()
    N = xo.shape[0]
    val, diag, zp = kc.factor(pat, T(xo), kg, prec)
    bar = fp.BAR[prec]
    fp.check_factor(prec, H(val), H(diag), rp, col, math.sqrt(1.0 + ko.nugget), (val_ref, zc_ref), strict=True)
    Lg = _gpu_dense_L(rp, col, val, diag, N)
    z = inputs.rhs(N, nrhs, seed=87)
    y = H(kc.l_matvec(pat, prec, val, diag, T(perm), T(z)))
    w = H(kc.lt_matvec(pat, prec, val, diag, T(perm), T(z)))
    for r in range(nrhs):
        zo = z[r][perm]
        # oracle on its own factor, in ordered positions; scattered back
        y_ref = oracle.l_matvec(rp, col, val_ref, zo)
        w_ref = oracle.lt_matvec(rp, col, val_ref, zo)
        assert np.max(np.abs(y[r][perm] - y_ref)) <= _row_bound(rp, col, zo, bar) + 1e-13
        colsum = np.max(np.bincount(col, weights=np.abs(zo[np.repeat(np.arange(N), np.diff(rp))]), minlength=N))
        assert np.max(np.abs(w[r][perm] - w_ref)) <= bar * colsum + 1e-13
        # the kernels' own arithmetic on the GPU factor
        np.testing.assert_allclose(y[r][perm], Lg @ zo, rtol=0, atol=1e-13 * np.abs(Lg).sum(1).max())
        np.testing.assert_allclose(w[r][perm], Lg.T @ zo, rtol=0, atol=1e-13 * np.abs(Lg).sum(0).max())
    # the same bits on a second run
    assert np.array_equal(H(kc.l_matvec(pat, prec, val, diag, T(perm), T(z))), y)
    assert np.array_equal(H(kc.lt_matvec(pat, prec, val, diag, T(perm), T(z))), w)


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_llt_matvec_approximates_theta(prec):
    """Task (1): L L^T v against the oracle's on its own factor, and against
    the dense Theta v at rho = infinity (L L^T = Theta there)."""
    x, perm, xo, rp, col, kg, ko, val_ref, zc_ref, pat = _task_case(N=2000, nu=1.5, ell=0.2, rho=5.0, nugget=1e-4)
    N = xo.shape[0]
    val, diag, zp = kc.factor(pat, T(xo), kg, prec)
    bar = fp.BAR[prec]
    fp.check_factor(prec, H(val), H(diag), rp, col, math.sqrt(1.0 + ko.nugget), (val_ref, zc_ref), strict=True)
    v = inputs.rhs(N, 2, seed=88)
    y = H(kc.llt_matvec(pat, prec, val, diag, T(perm), T(v)))
    Lg = _gpu_dense_L(rp, col, val, diag, N)
    rows = np.repeat(np.arange(N), np.diff(rp))
    rowabs = np.max(np.bincount(rows, weights=np.abs(val_ref), minlength=N))
    for r in range(2):
        vo = v[r][perm]
        w_ref = oracle.lt_matvec(rp, col, val_ref, vo)
        y_ref = oracle.l_matvec(rp, col, val_ref, w_ref)
        want = Lg @ (Lg.T @ vo)
        np.testing.assert_allclose(y[r][perm], want, rtol=0, atol=1e-12 * np.abs(want).max())
        # (L + dL)(L + dL)^T v - L L^T v, |dL| <= bar entrywise: dL w plus L dw,
        # with |dw| <= bar times the column sums of |v| (second order dropped)
        dw = bar * np.max(np.bincount(col, weights=np.abs(vo[rows]), minlength=N))
        bound = _row_bound(rp, col, w_ref, bar) + rowabs * dw
        assert np.max(np.abs(y[r][perm] - y_ref)) <= 1.01 * bound + 1e-12
    # rho = infinity, small N: the factor is the dense Cholesky factor
    x = inputs.uniform(400, 2, seed=89)
    perm, l, xo = kc.order_points(T(x))
    kg2 = kc.Kernel(1.5, 0.2, 1.0, 1e-3)
    pat2 = kc.build_pattern(xo, l, 1e300)
    val2, diag2, _ = kc.factor(pat2, xo, kg2, kc.FP64)
    v2 = inputs.rhs(400, 1, seed=90)
    y2 = H(kc.llt_matvec(pat2, kc.FP64, val2, diag2, perm, T(v2)))[0]
    want2 = refmath.dense_theta(x, 1.5, 0.2, 1.0, 1e-3) @ v2[0]
    assert np.linalg.norm(y2 - want2) <= 1e-10 * np.linalg.norm(want2)


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_logdet(prec):
    x, perm, xo, rp, col, kg, ko, val_ref, zc_ref, pat = _task_case()
    val, diag, zp = kc.factor(pat, T(xo), kg, prec)
    ld, z = kc.logdet(pat, diag)
    ld_ref, z_ref = oracle.logdet(rp, val_ref)
    assert z == z_ref == 0
    bar = fp.BAR[prec]
    fp.check_factor(prec, H(val), H(diag), rp, col, math.sqrt(1.0 + ko.nugget), (val_ref, zc_ref), strict=True)
    dref = val_ref[rp[1:] - 1]
    assert abs(ld - ld_ref) <= 2 * np.sum(bar / dref)  # first order in |d L_ii| <= bar
    dg = H(diag)
    assert abs(ld - 2 * math.fsum(np.log(dg))) <= 1e-12 * abs(ld)
    assert kc.logdet(pat, diag) == (ld, z)  # same bits again


def test_logdet_counts_dropped_pivots():
    # Matern-3/2 at rho = 2 on 2000 uniform points drops pivots
    x, perm, xo, rp, col, kg, ko, val_ref, zc_ref, pat = _task_case(N=2000, rho=2.0, nu=1.5,
                                                                    seed=inputs.seed_for(1))
    val, diag, zp = kc.factor(pat, T(xo), kg, kc.FP64)
    ld, z = kc.logdet(pat, diag)
    assert z == zp == int(zc_ref.sum()) > 0
    dg = H(diag)
    assert abs(ld - 2 * math.fsum(np.log(dg[dg > 0]))) <= 1e-12 * abs(ld)


def test_tasks_tiny_and_errors():
    for N in (1, 2, 33):
        x = inputs.uniform(N, 2, seed=91 + N)
        kg = kc.Kernel(0.5, 0.3)
        perm, l, xo = kc.order_points(T(x))
        pat = kc.build_pattern(xo, l, 3.0)
        val, diag, _ = kc.factor(pat, xo, kg, kc.FP64)
        z = inputs.rhs(N, 2, seed=92)
        Lg = _gpu_dense_L(H(pat.rowptr), H(pat.col), val, diag, N)
        p = H(perm)
        y = H(kc.l_matvec(pat, kc.FP64, val, diag, perm, T(z)))
        for r in range(2):
            np.testing.assert_allclose(y[r][p], Lg @ z[r][p], rtol=1e-14, atol=1e-15)
        ld, zz = kc.logdet(pat, diag)
        assert zz == 0 and abs(ld - 2 * math.fsum(np.log(H(diag)))) <= 1e-13 * max(1.0, abs(ld))
    with pytest.raises(kc.KcError):
        kc.l_matvec(pat, kc.FP64, val, diag, perm, T(inputs.rhs(N, 17, seed=93)))
