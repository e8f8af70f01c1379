"""Independent textbook/library computations used to pin the oracle.

Nothing here calls the oracle: the Matern kernel is evaluated from its
general Bessel-function definition (Eq. (Matern), Section 4.4) with SciPy's
``kv``, distances with SciPy's ``cdist``, and factors with NumPy/SciPy's dense
LAPACK routines.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial.distance import cdist
from scipy.special import gamma, kv


def matern_general(r, nu, ell, sigma2=1.0):
    """sigma2 * 2^{1-nu}/Gamma(nu) * (sqrt(2 nu) r / ell)^nu K_nu(sqrt(2 nu) r / ell), value sigma2 at r=0."""
    r = np.asarray(r, dtype=np.float64)
    t = math.sqrt(2.0 * nu) * r / ell
    out = np.full(r.shape, sigma2, dtype=np.float64)
    nz = t > 0
    tt = t[nz]
    out[nz] = sigma2 * (2.0 ** (1.0 - nu) / gamma(nu)) * tt ** nu * kv(nu, tt)
    return out


def dense_theta(x, nu, ell, sigma2=1.0, nugget=0.0):
    D = cdist(x, x)
    T = matern_general(D, nu, ell, sigma2)
    T[np.diag_indices_from(T)] = sigma2 + nugget
    return T


def dense_cov(x, kern):
    """Dense Theta of any covariance family (attributes family, nu, ell,
    sigma2, nugget, alpha, beta): the Cauchy class
    sigma2 (1 + (r/ell)^alpha)^{-beta/alpha} (family 1) in NumPy, else the
    Matern Bessel definition; nugget on the diagonal."""
    if getattr(kern, "family", 0) == 1:
        D = cdist(x, x)
        T = kern.sigma2 * (1.0 + (D / kern.ell) ** kern.alpha) ** (-kern.beta / kern.alpha)
        T[np.diag_indices_from(T)] = kern.sigma2 + kern.nugget
        return T
    return dense_theta(x, kern.nu, kern.ell, kern.sigma2, kern.nugget)


def cov_values(r, kern):
    """The covariance function (no nugget) at distances r, by its definition."""
    r = np.asarray(r, dtype=np.float64)
    if getattr(kern, "family", 0) == 1:
        return kern.sigma2 * (1.0 + (r / kern.ell) ** kern.alpha) ** (-kern.beta / kern.alpha)
    return matern_general(r, kern.nu, kern.ell, kern.sigma2)


def dense_lower(rowptr, col, val, N):
    L = np.zeros((N, N))
    for j in range(N):
        for e in range(rowptr[j], rowptr[j + 1]):
            L[j, col[e]] = val[e]
    return L


def pattern_mask(rowptr, col, N):
    M = np.zeros((N, N), dtype=bool)
    for j in range(N):
        M[j, col[rowptr[j]:rowptr[j + 1]]] = True
    return M | M.T


def ichol_masked_schur(A, S):
    """ICHOL(0) as a dense Cholesky factorisation whose Schur-complement
    updates are kept only on the pattern S (the definition behind Algorithm 2,
    Section 2.2), vectorised over whole trailing blocks.

    A is first restricted to S.  Eliminating pivot i forms the column
    l = A[i:, i] / sqrt(A_ii), which is zero off S because A stays supported on
    S, and subtracts the rank-one update l l^T from the trailing matrix, masked
    by S.  A nonpositive pivot leaves column i zero and updates nothing (the
    zero-column rule of Section 4.4).
    """
    S = np.asarray(S, dtype=bool)
    A = np.where(S, A, 0.0).astype(np.float64)
    N = A.shape[0]
    L = np.zeros_like(A)
    for i in range(N):
        p = A[i, i]
        if not p > 0.0:
            continue
        l = A[i:, i] / math.sqrt(p)
        L[i:, i] = l
        t = l[1:]
        A[i + 1:, i + 1:] -= np.outer(t, t) * S[i + 1:, i + 1:]
    return L
