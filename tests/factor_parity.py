"""Parity bars of the ICHOL(0) factor against the FP64 oracle.

Errors are measured against the row norm ||L_j,:||, which equals
sqrt(Theta_jj) for a factor that reproduces Theta on S (the backward-stable
scale of Cholesky).  The bars are fixed, not derived from the problem:

* FP64:      |L~_ji - L_ji| <= 1e-12 ||L_j,:||
* FP32 form: |L~_ji - L_ji| <= 1e-4  ||L_j,:||

A *well-conditioned* case (no pivot dropped, every pivot far from zero) is
held to these bars over every entry (``strict=True``).

In an ill-conditioned case (smooth kernels, many pivots dropped by the rule of
Section 4.4) some columns follow tiny pivots, p = Theta_ii - sum_k L_ik^2 with
p of order 1e-8 Theta_ii, and their entries are not determined by the method
at the working precision: the oracle itself moves them by up to O(1) when its
arithmetic is perturbed the way the GPU's is (FP64: its sums in the other
order; FP32 form: every Theta_ji and L_ji rounded to float as produced).  Such
a case is checked in three parts:

1. pivot decisions: the same as the oracle's, except where the oracle's
   pivot is within 1e-5 Theta_ii of zero (FP32 form) or where the pivot is
   not determined: the perturbed rerun decides it otherwise, or moves an
   entry of row i (the L_ik that form p_i) by more than a hundredth of the
   bar;
2. entries: every column that the oracle's perturbed rerun moves by at most a
   hundredth of the bar, whose decision agrees in all three factors, and
   that does not depend (through the dependency DAG: column i needs every
   column k in R_i) on a column whose decision the GPU took otherwise, is
   held to the bar itself; these must be at least ``min_entries`` (half) of
   all entries.  A decision taken otherwise changes its column by O(1), a
   perturbation the rerun's roundings never make, so its descendants are
   left to the identity.  The margin of 100 covers the GPU's roundings being of
   another kind and a few times larger than the rerun's: Theta_ji evaluated
   in float arithmetic (a few ulp) rather than rounded once, compensated
   sums in another order.  On the GB300 the largest ratio seen between the
   GPU's error and the rerun's shift in a column was 17.5;
3. every kept column: the defining identity (L L^T)_ji = Theta_ji on S
   (1e-12 FP64, 1e-6 FP32 form, relative to Theta_jj), which does not depend
   on conditioning (checked by the caller, which has the dense Theta).
"""
from __future__ import annotations

import numpy as np

BAR = {0: 1e-12, 1: 1e-4}          # FP64, FP32 form
IDENTITY_BAR = {0: 1e-12, 1: 1e-6}
PIVOT_FLIP = 1e-5                  # FP32 form: decisions may differ within this of zero
DETERMINED = 100.0                 # determined: the rerun moves the column by <= bar / DETERMINED


def rows_of(rp):
    return np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))


def check_factor(prec, val, diag, rp, col, rownorm, ref, alt=None, piv=None, strict=False,
                 min_entries=0.5, entries=True):
    """Assert the bars above; returns a dict of what was compared.

    prec      0 (FP64) or 1 (FP32 form)
    val, diag the GPU factor (NumPy), val in the CSR layout of (rp, col)
    rownorm   sqrt(Theta_jj) per row (NumPy array) or a scalar
    ref       (val_ref, zero_col_ref) of the FP64 oracle
    alt       (val_alt, zero_col_alt) of the oracle's perturbed rerun
              (needed unless strict)
    piv       the oracle's pivots p_i (needed for the FP32 form if a decision
              differs)
    entries   False: decisions only (a factor whose Theta the GPU evaluates
              less accurately than the bar, in an ill-conditioned case)
    """
    val_ref, zc_ref = ref
    bar = BAR[prec]
    N = rp.shape[0] - 1
    rows = rows_of(rp)
    rn = np.broadcast_to(np.asarray(rownorm, dtype=np.float64), (N,))
    err = np.abs(np.asarray(val, dtype=np.float64) - val_ref) / rn[rows]
    z = np.asarray(diag) == 0.0
    differ = z != zc_ref
    if strict:
        assert not differ.any(), np.nonzero(differ)[0][:10]
        worst = float(err.max(initial=0.0))
        assert worst <= bar, worst
        return {"compared": 1.0, "max_err": worst, "flips": 0}
    val_alt, zc_alt = alt
    moved = np.abs(val_alt - val_ref) / rn[rows]
    sens = np.zeros(N)                      # per column
    np.maximum.at(sens, col, moved)
    offd = col != rows
    row_sens = np.zeros(N)                  # per row, entries left of the diagonal
    np.maximum.at(row_sens, rows[offd], moved[offd])
    if differ.any():
        near_zero = (np.abs(piv[differ]) <= PIVOT_FLIP * rn[differ] ** 2) if prec == 1 else False
        undetermined = (zc_alt[differ] != zc_ref[differ]) | (row_sens[differ] > bar / DETERMINED)
        ok = near_zero | undetermined
        assert np.all(ok), np.nonzero(differ)[0][~ok][:10]
    if not entries:
        return {"compared": 0.0, "max_err": None, "flips": int(differ.sum())}
    det = (sens <= bar / DETERMINED) & ~differ & (zc_alt == zc_ref) & ~descendants(rp, col, differ)
    m = det[col]
    frac = float(m.mean()) if m.size else 1.0
    assert frac >= min_entries, frac
    worst = float(err[m].max(initial=0.0))
    assert worst <= bar, (worst, int(np.argmax(np.where(m, err, 0))))
    return {"compared": frac, "max_err": worst, "flips": int(differ.sum())}


def descendants(rp, col, seed):
    """Columns reachable from the `seed` columns in the dependency DAG of the
    factor (column i depends on every k in R_i), the seeds included."""
    N = rp.shape[0] - 1
    out = np.asarray(seed, dtype=bool).copy()
    if not out.any():
        return out
    for i in range(int(np.argmax(out)) + 1, N):
        if not out[i]:
            r = col[rp[i]:rp[i + 1] - 1]
            if r.size and out[r].any():
                out[i] = True
    return out


def identity_residual_dense(L, Th, rp, col, scale):
    """max over (j,i) in S with L_ii > 0 of |(L L^T)_ji - Theta_ji| / scale_j."""
    N = L.shape[0]
    keep = np.diag(L) != 0
    rows = rows_of(rp)
    m = keep[col]
    LLt = L @ L.T
    s = np.broadcast_to(np.asarray(scale, dtype=np.float64), (N,))
    return float(np.max(np.abs(LLt[rows[m], col[m]] - Th[rows[m], col[m]]) / s[rows[m]], initial=0.0))
