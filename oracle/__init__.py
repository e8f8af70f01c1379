"""Plain FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the arithmetic lives in ``kchol_oracle.c`` (single-threaded C, compiled with
``-O2 -ffp-contract=off``), and this module only marshals NumPy arrays.

Each wrapper names the passage of the paper it follows (Schaefer, Sullivan,
Owhadi, arXiv:1706.02205):

* ``maximin_brute``      -- maximin ordering and length scales, by definition
                            (Section 2.3), O(N^2).
* ``sortsparse``         -- ordering and pattern by the paper's heap algorithm
                            (Algorithm 3, Section 4.1).
* ``pattern``            -- S_rho by definition (Section 2.3), O(N^2).
* ``matern`` / ``cauchy`` / ``theta`` -- covariance functions of Section 4.4:
                            Matern (Eq. (Matern)), closed forms for nu in
                            {1/2, 3/2, 5/2}, other nu > 0 through ``bessel_k``
                            (the integral representation of K_nu, Abramowitz &
                            Stegun 9.6.24); the Cauchy class of Gneiting.
* ``ichol``              -- ICHOL(0), Algorithm 2, left-looking form; the
                            zero-column rule for nonpositive pivots (Section 4.4).
* ``solve_lower`` / ``solve_upper`` / ``pcg`` -- task (2) of Section 1, and CG
                            preconditioned with the factor (Section 4.3).
* ``frob_error``         -- the sampled error estimator E (Section 4.4).
* ``pca_truncate`` / ``pca_error_power`` -- rank-k PCA from the first k
                            columns (Section 2.5).
* ``l_matvec`` / ``lt_matvec`` / ``logdet`` -- tasks (1), (3), (4) of Section 1
                            with the factor: L z, L^T v, 2 sum log L_ii.
* ``ichol_given`` / ``pattern_reverse`` / ``gather_entries`` / ``reverse_factor``
                         -- Section 6: ICHOL(0) of a given sparse matrix (the
                            precision matrix, or sigma^2 A + I) in the reverse
                            maximin order on the min-rule pattern.
* ``supernodal``         -- the supernodal multicolour ordering and pattern
                            (Construction of the stability section), brute force.
* ``work_counters``      -- exact multiply-add / merge-step / operand counts of
                            the left-looking factor (roofline denominators).

Every function above is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kchol_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkchol_oracle.so")

RULE_MAX = 0
RULE_MIN = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None

i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")


class _SortSparseResult(C.Structure):
    _fields_ = [("N", C.c_int64), ("perm", C.POINTER(C.c_int32)), ("l", C.POINTER(C.c_double)),
                ("nnz", C.c_int64), ("rowptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32))]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d, i, I = C.c_double, C.c_int64, C.c_int32
        L.ko_d2.restype = d
        L.ko_d2.argtypes = [f64p, f64p, I]
        L.ko_maximin_brute.argtypes = [f64p, i, I, i32p, f64p]
        L.ko_sortsparse.restype = C.POINTER(_SortSparseResult)
        L.ko_sortsparse.argtypes = [f64p, i, I, d, I]
        L.ko_sortsparse_free.argtypes = [C.POINTER(_SortSparseResult)]
        L.ko_pattern_count.argtypes = [f64p, f64p, i, I, d, I, i64p]
        L.ko_pattern_fill.argtypes = [f64p, f64p, i, I, d, I, i64p, i32p]
        K = C.POINTER(KoKernel)
        L.ko_bessel_k.restype = d
        L.ko_bessel_k.argtypes = [d, d]
        L.ko_bessel_k_scaled.restype = d
        L.ko_bessel_k_scaled.argtypes = [d, d]
        L.ko_matern.restype = d
        L.ko_matern.argtypes = [d, d, d, d]
        L.ko_cauchy.restype = d
        L.ko_cauchy.argtypes = [d, d, d, d, d]
        L.ko_cov.restype = d
        L.ko_cov.argtypes = [d, K]
        L.ko_theta.restype = d
        L.ko_theta.argtypes = [f64p, I, i, i, K]
        L.ko_csr_to_csc.argtypes = [i, i64p, i32p, i64p, i32p, i64p]
        L.ko_ichol.restype = i
        L.ko_ichol.argtypes = [f64p, i, I, K, i64p, i32p, f64p, u8p, I, C.c_void_p, I]
        L.ko_ichol_given.restype = i
        L.ko_ichol_given.argtypes = [i, i64p, i32p, f64p, f64p, u8p, I, I]
        L.ko_pattern_reverse.argtypes = [i, i64p, i32p, i64p, i32p]
        L.ko_supernodal.restype = i
        L.ko_supernodal.argtypes = [f64p, i, I, i32p, f64p, d, i32p, i32p, i32p, i32p, i64p,
                                    C.POINTER(C.POINTER(C.c_int32))]
        L.ko_free.argtypes = [C.c_void_p]
        L.ko_gather_entries.restype = i
        L.ko_gather_entries.argtypes = [i, i64p, i32p, i32p, i64p, i32p, f64p, f64p]
        L.ko_solve_lower.argtypes = [i, i64p, i32p, f64p, f64p, f64p, f64p]
        L.ko_solve_upper.argtypes = [i, i64p, i32p, f64p, f64p, f64p, f64p]
        L.ko_l_matvec.argtypes = [i, i64p, i32p, f64p, f64p, f64p]
        L.ko_lt_matvec.argtypes = [i, i64p, i32p, f64p, f64p, f64p]
        L.ko_logdet.restype = d
        L.ko_logdet.argtypes = [i, i64p, f64p, C.POINTER(C.c_int64)]
        L.ko_theta_s_matvec.argtypes = [f64p, i, I, K, i64p, i32p, f64p, f64p]
        L.ko_theta_dense_matvec.argtypes = [f64p, i, I, K, f64p, f64p]
        L.ko_pcg.restype = I
        L.ko_pcg.argtypes = [f64p, i, I, K, i64p, i32p, f64p, f64p, I, f64p, d, I, f64p,
                             C.POINTER(C.c_double), C.POINTER(C.c_int32)]
        L.ko_llt_entry.restype = d
        L.ko_llt_entry.argtypes = [i64p, i32p, f64p, i, i]
        L.ko_frob_error.argtypes = [f64p, i, I, K, i64p, i32p, f64p, i64p, i, i64p, i64p,
                                    C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64)]
        L.ko_pca_truncate.argtypes = [i, i64p, i32p, f64p, i32p, I, f64p]
        L.ko_pca_error_power.restype = d
        L.ko_pca_error_power.argtypes = [f64p, i, I, K, I, f64p, f64p, I]
        L.ko_work_counters.argtypes = [i, i64p, i32p] + [C.POINTER(C.c_int64)] * 4
        _lib = L
    return _lib


def _pts(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    return x, x.shape[0], x.shape[1]


MATERN = 0
CAUCHY = 1


class KoKernel(C.Structure):
    _fields_ = [("family", C.c_int32), ("nu", C.c_double), ("ell", C.c_double), ("sigma2", C.c_double),
                ("nugget", C.c_double), ("alpha", C.c_double), ("beta", C.c_double)]


class Kernel:
    """Covariance parameters (Section 4.4): the Matern class (smoothness
    nu > 0, length scale ell, variance sigma2) or, with family=CAUCHY, the
    Cauchy class (ell, alpha in (0, 2], beta > 0, sigma2); a nugget is added
    on the diagonal."""

    def __init__(self, nu=1.5, ell=0.2, sigma2=1.0, nugget=0.0, family=MATERN, alpha=1.0, beta=1.0):
        if family == MATERN and not nu > 0:
            raise ValueError("nu must be positive")
        if family == CAUCHY and not (0 < alpha <= 2 and beta > 0):
            raise ValueError("the Cauchy class needs 0 < alpha <= 2 and beta > 0")
        self.family = int(family)
        self.nu, self.ell, self.sigma2, self.nugget = float(nu), float(ell), float(sigma2), float(nugget)
        self.alpha, self.beta = float(alpha), float(beta)

    def c(self):
        return KoKernel(self.family, self.nu, self.ell, self.sigma2, self.nugget, self.alpha, self.beta)

    def args(self):
        return (C.byref(self.c()),)


# --------------------------------------------------------------------------
# ordering and pattern
# --------------------------------------------------------------------------

def maximin_brute(x):
    """(perm, l): perm[k] = original index of the k-th point, l[k] its length scale."""
    x, N, d = _pts(x)
    perm = np.zeros(N, np.int32)
    l = np.zeros(N, np.float64)
    if N:
        lib().ko_maximin_brute(x, N, d, perm, l)
    return perm, l


def sortsparse(x, rho, rule=RULE_MAX):
    """(perm, l, rowptr, col) from the paper's heap algorithm (needs rho >= 1)."""
    if rho < 1.0:
        raise ValueError("the heap algorithm needs rho >= 1")
    x, N, d = _pts(x)
    R = lib().ko_sortsparse(x, N, d, float(rho), int(rule))
    try:
        r = R.contents
        perm = np.ctypeslib.as_array(r.perm, shape=(N,)).copy() if N else np.zeros(0, np.int32)
        l = np.ctypeslib.as_array(r.l, shape=(N,)).copy() if N else np.zeros(0)
        rowptr = np.ctypeslib.as_array(r.rowptr, shape=(N + 1,)).copy()
        col = np.ctypeslib.as_array(r.col, shape=(r.nnz,)).copy() if r.nnz else np.zeros(0, np.int32)
    finally:
        lib().ko_sortsparse_free(R)
    return perm, l, rowptr, col


def pattern(x_ord, l, rho, rule=RULE_MAX):
    """CSR (rowptr int64[N+1], col int32[nnz]) of L's pattern, by definition."""
    x_ord, N, d = _pts(x_ord)
    l = np.ascontiguousarray(l, dtype=np.float64)
    rowptr = np.zeros(N + 1, np.int64)
    lib().ko_pattern_count(x_ord, l, N, d, float(rho), int(rule), rowptr)
    col = np.zeros(int(rowptr[-1]), np.int32)
    lib().ko_pattern_fill(x_ord, l, N, d, float(rho), int(rule), rowptr, col)
    return rowptr, col


def csr_to_csc(rowptr, col):
    N = rowptr.shape[0] - 1
    nnz = int(rowptr[-1])
    colptr = np.zeros(N + 1, np.int64)
    rowidx = np.zeros(nnz, np.int32)
    slot = np.zeros(nnz, np.int64)
    lib().ko_csr_to_csc(N, rowptr, col, colptr, rowidx, slot)
    return colptr, rowidx, slot


# --------------------------------------------------------------------------
# kernel entries
# --------------------------------------------------------------------------

def bessel_k(nu, x):
    """K_nu(x), x > 0, from the integral representation (A&S 9.6.24)."""
    return lib().ko_bessel_k(float(nu), float(x))


def bessel_k_scaled(nu, x):
    """e^x K_nu(x), x > 0, the same integral with e^x taken inside."""
    return lib().ko_bessel_k_scaled(float(nu), float(x))


def matern(r, nu, ell, sigma2=1.0):
    return lib().ko_matern(float(r), float(nu), float(ell), float(sigma2))


def cauchy(r, ell, alpha, beta, sigma2=1.0):
    return lib().ko_cauchy(float(r), float(ell), float(alpha), float(beta), float(sigma2))


def cov(r, kern: Kernel):
    """The covariance function of kern at distance r (no nugget)."""
    k = kern.c()
    return lib().ko_cov(float(r), C.byref(k))


def theta(x_ord, a, b, kern: Kernel):
    x_ord, N, d = _pts(x_ord)
    return lib().ko_theta(x_ord, d, int(a), int(b), *kern.args())


# --------------------------------------------------------------------------
# factor, solves, refinement
# --------------------------------------------------------------------------

def ichol(x_ord, rowptr, col, kern: Kernel, reverse_sums=False, pivots=False, store_f32=False):
    """ICHOL(0) values on the CSR pattern; returns (val float64[nnz], zero_col bool[N])
    and, with pivots=True, also the pivot p of every column before its test.
    reverse_sums=True sums in descending k (same arithmetic, other rounding
    order) to measure the problem's sensitivity to FP64 rounding order;
    store_f32=True rounds each off-diagonal Theta_ji and L_ji to float when
    it is computed (the roundings of a factor with float entries), to size
    FP32-form tolerances."""
    x_ord, N, d = _pts(x_ord)
    val = np.zeros(int(rowptr[-1]), np.float64)
    zc = np.zeros(N, np.int8)
    piv = np.zeros(N, np.float64)
    lib().ko_ichol(x_ord, N, d, *kern.args(), np.ascontiguousarray(rowptr, np.int64),
                   np.ascontiguousarray(col, np.int32), val, zc, int(bool(reverse_sums)),
                   piv.ctypes.data_as(C.c_void_p), int(bool(store_f32)))
    if pivots:
        return val, zc.astype(bool), piv
    return val, zc.astype(bool)


def ichol_given(rowptr, col, aval, reverse_sums=False, store_f32=False):
    """ICHOL(0) of a given symmetric matrix on the pattern: aval[e] is its entry
    at the CSR position e (Section 6).  Returns (val, zero_col)."""
    N = rowptr.shape[0] - 1
    val = np.zeros(int(rowptr[-1]), np.float64)
    zc = np.zeros(N, np.int8)
    lib().ko_ichol_given(N, np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(col, np.int32),
                         np.ascontiguousarray(aval, np.float64), val, zc, int(bool(reverse_sums)),
                         int(bool(store_f32)))
    return val, zc.astype(bool)


def supernodal(x, rho):
    """The supernodal multicolour ordering and pattern (the paper's
    Construction, stability section) from the maximin ordering of x: order
    (new position -> original index), level, node (maximin index of the
    supernode) and colour of every new position, and the CSR pattern (lower
    triangle in the new order).  O(N^2): small cases only."""
    x, N, d = _pts(x)
    perm, l = maximin_brute(x)
    order = np.zeros(N, np.int32)
    level = np.zeros(N, np.int32)
    node = np.zeros(N, np.int32)
    color = np.zeros(N, np.int32)
    rowptr = np.zeros(N + 1, np.int64)
    cp = C.POINTER(C.c_int32)()
    nnz = lib().ko_supernodal(x, N, d, perm, l, float(rho), order, level, node, color, rowptr, C.byref(cp))
    if nnz < 0:
        raise MemoryError(f"oracle.supernodal: no memory for the dense {N} x {N} supernode set")
    try:
        col = np.ctypeslib.as_array(cp, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
    finally:
        lib().ko_free(cp)
    return dict(perm=perm, l=l, order=order, level=level, node=node, color=color, rowptr=rowptr, col=col)


def pattern_reverse(colptr, rowidx):
    """CSR (rowptr, col) of a symmetric pattern in the reversed order, from the
    CSC of its lower triangle in the original (maximin) order (Section 6)."""
    N = colptr.shape[0] - 1
    rowptr = np.zeros(N + 1, np.int64)
    col = np.zeros(int(colptr[-1]), np.int32)
    lib().ko_pattern_reverse(N, np.ascontiguousarray(colptr, np.int64), np.ascontiguousarray(rowidx, np.int32),
                             rowptr, col)
    return rowptr, col


def gather_entries(rowptr, col, orig, a_rowptr, a_col, a_val):
    """(aval, outside): the given matrix (CSR in original numbering) at every
    pattern position (orig: position -> original index), and the number of
    its off-diagonal entries outside the pattern."""
    N = rowptr.shape[0] - 1
    aval = np.zeros(int(rowptr[-1]), np.float64)
    out = lib().ko_gather_entries(N, np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(col, np.int32),
                                  np.ascontiguousarray(orig, np.int32), np.ascontiguousarray(a_rowptr, np.int64),
                                  np.ascontiguousarray(a_col, np.int32), np.ascontiguousarray(a_val, np.float64),
                                  aval)
    return aval, int(out)


def reverse_factor(x, a_rowptr, a_col, a_val, rho, store_f32=False):
    """Section 6: maximin ordering of x, the min-rule pattern, reversed, the
    given matrix gathered onto it and factored.  Returns a dict with the
    reversed order (orig[q] = original index of position q), the pattern,
    the entries, the factor and its dropped columns."""
    x, N, d = _pts(x)
    perm, l = maximin_brute(x)
    rp, col = pattern(x[perm], l, rho, RULE_MIN)
    colptr, rowidx, _ = csr_to_csc(rp, col)
    rrp, rcol = pattern_reverse(colptr, rowidx)
    orig = np.ascontiguousarray(perm[::-1])
    aval, outside = gather_entries(rrp, rcol, orig, a_rowptr, a_col, a_val)
    val, zc = ichol_given(rrp, rcol, aval, store_f32=store_f32)
    return dict(perm=perm, l=l, orig=orig, rowptr=rrp, col=rcol, aval=aval, outside=outside, val=val,
                zero_col=zc)


def diag_of(rowptr, val):
    return np.ascontiguousarray(val[rowptr[1:] - 1])


def solve_diag(x_ord, rowptr, val, kern: Kernel):
    """Diagonal used by the solves: L_ii, or sqrt(Theta_ii) for a zeroed column."""
    dg = diag_of(rowptr, val).copy()
    z = ~(dg > 0.0)
    dg[z] = np.sqrt(kern.sigma2 + kern.nugget)
    return dg


def solve_lower(rowptr, col, val, diag, b):
    N = rowptr.shape[0] - 1
    y = np.zeros(N)
    lib().ko_solve_lower(N, rowptr, col, val, np.ascontiguousarray(diag, np.float64),
                         np.ascontiguousarray(b, np.float64), y)
    return y


def solve_upper(rowptr, col, val, diag, y):
    N = rowptr.shape[0] - 1
    x = np.zeros(N)
    lib().ko_solve_upper(N, rowptr, col, val, np.ascontiguousarray(diag, np.float64),
                         np.ascontiguousarray(y, np.float64), x)
    return x


def l_matvec(rowptr, col, val, z):
    """y = L z in ordered positions (task (4): a sample of N(0, L L^T) when z ~ N(0, I))."""
    N = rowptr.shape[0] - 1
    y = np.zeros(N)
    lib().ko_l_matvec(N, rowptr, col, np.ascontiguousarray(val, np.float64), np.ascontiguousarray(z, np.float64), y)
    return y


def lt_matvec(rowptr, col, val, v):
    """w = L^T v in ordered positions."""
    N = rowptr.shape[0] - 1
    w = np.zeros(N)
    lib().ko_lt_matvec(N, rowptr, col, np.ascontiguousarray(val, np.float64), np.ascontiguousarray(v, np.float64), w)
    return w


def logdet(rowptr, val):
    """(2 sum log L_ii over kept columns, number of dropped columns): task (3)."""
    N = rowptr.shape[0] - 1
    z = C.c_int64(0)
    v = lib().ko_logdet(N, rowptr, np.ascontiguousarray(val, np.float64), C.byref(z))
    return v, int(z.value)


def theta_s_matvec(x_ord, rowptr, col, kern: Kernel, v):
    x_ord, N, d = _pts(x_ord)
    y = np.zeros(N)
    lib().ko_theta_s_matvec(x_ord, N, d, *kern.args(), rowptr, col, np.ascontiguousarray(v, np.float64), y)
    return y


def theta_dense_matvec(x, kern: Kernel, v):
    x, N, d = _pts(x)
    y = np.zeros(N)
    lib().ko_theta_dense_matvec(x, N, d, *kern.args(), np.ascontiguousarray(v, np.float64), y)
    return y


def pcg(x_ord, rowptr, col, val, diag, kern: Kernel, b, op=1, rtol=1e-10, maxit=200):
    """PCG on Theta^S (op=1) or dense Theta (op=2) with preconditioner L L^T.

    Returns (x, iterations, relres, status) with status 0 converged,
    1 not converged, 2 nonpositive curvature.
    """
    x_ord, N, d = _pts(x_ord)
    x = np.zeros(N)
    rr = C.c_double(0.0)
    st = C.c_int32(0)
    it = lib().ko_pcg(x_ord, N, d, *kern.args(), rowptr, col, val, np.ascontiguousarray(diag, np.float64),
                      int(op), np.ascontiguousarray(b, np.float64), float(rtol), int(maxit), x,
                      C.byref(rr), C.byref(st))
    return x, int(it), float(rr.value), int(st.value)


def llt_entry(rowptr, col, val, a, b):
    return lib().ko_llt_entry(rowptr, col, val, int(a), int(b))


def frob_error(x_ord, rowptr, col, val, perm, kern: Kernel, pi, pj, keep=None):
    """Returns (num2, den2, kept) of the sampled estimator; E = sqrt(num2/den2)."""
    x_ord, N, d = _pts(x_ord)
    pos = np.empty(N, np.int64)
    pos[np.asarray(perm)] = np.arange(N, dtype=np.int64)
    a, b, c = C.c_double(), C.c_double(), C.c_int64()
    kp = None
    if keep is not None:
        keep = np.ascontiguousarray(keep, dtype=np.int8)
        kp = keep.ctypes.data_as(C.c_void_p)
    lib().ko_frob_error(x_ord, N, d, *kern.args(), rowptr, col, val, pos, int(len(pi)),
                        np.ascontiguousarray(pi, np.int64), np.ascontiguousarray(pj, np.int64), kp,
                        C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def pca_truncate(rowptr, col, val, perm, k):
    N = rowptr.shape[0] - 1
    Lk = np.zeros(N * k)
    lib().ko_pca_truncate(N, rowptr, col, val, np.ascontiguousarray(perm, np.int32), int(k), Lk)
    return Lk.reshape(k, N)          # row a = column a of L_k, original row order


def pca_error_power(x, kern: Kernel, Lk, v0, iters=50):
    x, N, d = _pts(x)
    k = Lk.shape[0]
    return lib().ko_pca_error_power(x, N, d, *kern.args(), int(k), np.ascontiguousarray(Lk, np.float64).ravel(),
                                    np.ascontiguousarray(v0, np.float64), int(iters))


def work_counters(rowptr, col):
    """dict(F, M, P, Rsum) of the left-looking factor on this pattern."""
    N = rowptr.shape[0] - 1
    out = [C.c_int64() for _ in range(4)]
    lib().ko_work_counters(N, rowptr, col, *[C.byref(o) for o in out])
    return dict(F=out[0].value, M=out[1].value, P=out[2].value, Rsum=out[3].value)


def bytes_op(rowptr, counters, N, d, s):
    """Operand bytes of the left-looking factor with value size s (4 or 8):
    the pivot row staged once per column, the row-j prefix and x_j per entry,
    the pattern read and L written once, the points read once."""
    nnz = int(rowptr[-1])
    offdiag = nnz - N
    return (counters["Rsum"] * (4 + s) + counters["P"] * (4 + s) + offdiag * 8 * d
            + nnz * (4 + s) + N * d * 8)


# --------------------------------------------------------------------------
# the whole pipeline on one point set
# --------------------------------------------------------------------------

def pipeline(x, rho, kern: Kernel, rule=RULE_MAX, method="sortsparse"):
    """Ordering, pattern and FP64 factor of one point set."""
    x, N, d = _pts(x)
    if method == "sortsparse":
        perm, l, rowptr, col = sortsparse(x, rho, rule)
    else:
        perm, l = maximin_brute(x)
        rowptr, col = pattern(x[perm], l, rho, rule)
    x_ord = np.ascontiguousarray(x[perm])
    val, zc = ichol(x_ord, rowptr, col, kern)
    return dict(perm=perm, l=l, x_ord=x_ord, rowptr=rowptr, col=col, val=val, zero_col=zc)
