"""GPU parity of the sampled error estimator E of Section 4.4 (kc_frob_error).

* The kernel's arithmetic: on the GPU's own factor, num2 and den2 against
  the same sums in NumPy (sparse products in FP64, Theta from the Bessel
  definition), 1e-10 relative; with every pair (i, j) of a small problem
  sampled once, E equals the dense Frobenius ratio ||L L^T - Theta||_F /
  ||Theta||_F.
* Against the oracle: E of the GPU factor against the oracle's estimator on
  the oracle's own factor, within the bound the factor bars imply: every
  (L L^T)_ij moves by at most bar (||L_i||_1 + ||L_j||_1) when every entry
  moves by at most bar (row norms 1 here), and E by at most the 2-norm of
  those moves over sqrt(den2).
* The same bits on a second run; the keep mask; pair indices out of range.
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


def _case(N=3000, nu=0.5, ell=0.2, rho=3.0, seed=141):
    x = inputs.uniform(N, 2, seed=seed)
    kg, ko = kc.Kernel(nu, ell), oracle.Kernel(nu, ell)
    perm, l, xo = kc.order_points(T(x))
    pat = kc.build_pattern(xo, l, rho)
    return x, kg, ko, perm, xo, pat


def _gpu_L(pat, val, diag):
    from scipy.sparse import csr_matrix
    N = pat.N
    v = H(val).astype(np.float64).copy()
    rp = H(pat.rowptr)
    v[rp[1:] - 1] = H(diag)
    return csr_matrix((v, H(pat.col), rp), shape=(N, N))


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_estimator_arithmetic_on_the_gpu_factor(prec):
    x, kg, ko, perm, xo, pat = _case()
    val, diag, zp = kc.factor(pat, xo, kg, prec)
    N = pat.N
    pi, pj = inputs.sample_pairs(N, 20000, seed=142)
    num2, den2, kept = kc.frob_error(pat, prec, val, diag, xo, kg, perm, T(pi), T(pj))
    assert kept == 20000
    L = _gpu_L(pat, val, diag)
    pos = np.empty(N, np.int64)
    pos[H(perm)] = np.arange(N)
    a, b = pos[pi], pos[pj]
    llt = np.asarray(L[a].multiply(L[b]).sum(axis=1)).ravel()
    xh = H(xo)
    r = np.sqrt(((xh[a] - xh[b]) ** 2).sum(1))
    th = refmath.matern_general(r, 0.5, 0.2)
    th[a == b] = 1.0
    assert abs(num2 / np.sum((llt - th) ** 2) - 1) < 1e-9
    assert abs(den2 / np.sum(th ** 2) - 1) < 1e-12
    # the same bits again
    assert kc.frob_error(pat, prec, val, diag, xo, kg, perm, T(pi), T(pj)) == (num2, den2, kept)


def test_every_pair_once_gives_the_dense_frobenius_ratio():
    x, kg, ko, perm, xo, pat = _case(N=600, nu=1.5, ell=0.2, rho=2.0, seed=143)
    val, diag, zp = kc.factor(pat, xo, kg, kc.FP64)
    N = pat.N
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    num2, den2, kept = kc.frob_error(pat, kc.FP64, val, diag, xo, kg, perm, T(ii.ravel()), T(jj.ravel()))
    L = _gpu_L(pat, val, diag).toarray()
    Th = refmath.dense_theta(H(xo), 1.5, 0.2)
    want = np.linalg.norm(L @ L.T - Th) / np.linalg.norm(Th)
    assert abs(np.sqrt(num2 / den2) / want - 1) < 1e-10
    assert kept == N * N


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_estimator_against_the_oracle(prec):
    x, kg, ko, perm, xo, pat = _case()
    val, diag, zp = kc.factor(pat, xo, kg, prec)
    N = pat.N
    pi, pj = inputs.sample_pairs(N, 50000, seed=144)
    num2, den2, kept = kc.frob_error(pat, prec, val, diag, xo, kg, perm, T(pi), T(pj))
    p_ref, l_ref, rp, col = oracle.sortsparse(x, 3.0)
    assert np.array_equal(H(perm), p_ref)
    xr = x[p_ref]
    v_ref, zc = oracle.ichol(xr, rp, col, ko)
    assert not zc.any()
    n2, d2, c2 = oracle.frob_error(xr, rp, col, v_ref, p_ref, ko, pi, pj)
    assert c2 == kept
    assert abs(den2 / d2 - 1) < 1e-12
    # the bound implied by |dL| <= bar entrywise (row norms are 1 here)
    bar = fp.BAR[prec]
    pos = np.empty(N, np.int64)
    pos[p_ref] = np.arange(N)
    rows = fp.rows_of(rp)
    l1 = np.bincount(rows, weights=np.abs(v_ref), minlength=N)
    dmax = bar * (l1[pos[pi]] + l1[pos[pj]])
    e_gpu, e_ref = np.sqrt(num2 / den2), np.sqrt(n2 / d2)
    assert abs(e_gpu - e_ref) <= 1.01 * np.sqrt(np.sum(dmax ** 2) / d2) + 1e-15
    # and the paper's size of E at rho = 3 for this kernel (Table 1: about 1e-3)
    assert 2e-4 < e_gpu < 5e-3


def test_keep_mask_and_bad_indices():
    x, kg, ko, perm, xo, pat = _case(N=1500, seed=145)
    val, diag, zp = kc.factor(pat, xo, kg, kc.FP32_FORM)
    N = pat.N
    pi, pj = inputs.sample_pairs(N, 5000, seed=146)
    full = kc.frob_error(pat, kc.FP32_FORM, val, diag, xo, kg, perm, T(pi), T(pj))
    ones = kc.frob_error(pat, kc.FP32_FORM, val, diag, xo, kg, perm, T(pi), T(pj),
                         keep=T(np.ones(5000, np.int8)))
    assert ones == full
    keep = (np.arange(5000) % 3 == 0).astype(np.int8)
    n_k, d_k, c_k = kc.frob_error(pat, kc.FP32_FORM, val, diag, xo, kg, perm, T(pi), T(pj), keep=T(keep))
    n_s, d_s, c_s = kc.frob_error(pat, kc.FP32_FORM, val, diag, xo, kg, perm, T(pi[::3]), T(pj[::3]))
    assert c_k == c_s == int(keep.sum())
    assert abs(n_k / n_s - 1) < 1e-12 and abs(d_k / d_s - 1) < 1e-12
    bad = pi.copy()
    bad[17] = N
    with pytest.raises(kc.KcError) as ei:
        kc.frob_error(pat, kc.FP32_FORM, val, diag, xo, kg, perm, T(bad), T(pj))
    assert ei.value.status == kc.KC_EINVAL
    bad[17] = -1
    with pytest.raises(kc.KcError):
        kc.frob_error(pat, kc.FP32_FORM, val, diag, xo, kg, perm, T(pj), T(bad))
    # the context is still usable
    assert kc.frob_error(pat, kc.FP32_FORM, val, diag, xo, kg, perm, T(pi), T(pj)) == full
