"""Pins of the oracle's supernodal multicolour ordering and pattern (the
Construction of the stability section) and of ICHOL(0) on them.

* The construction's own requirements: supernodes of a level are farther
  apart than rho (in the hierarchical pseudometric) and every point lies
  within rho of its supernode, which is the nearest; colours differ across
  every same-level pair of the supernode pattern and are greedy-minimal; the
  ordering goes by level, then colour, and keeps supernodes contiguous.
* The pattern holds every pair with d(i, j) <= rho and is the union of
  blocks of supernode pairs.
* The appendix's equivalence: Algorithm 2 in this ordering and pattern equals
  the supernodal block factorisation (a block Cholesky with the updates masked
  to the supernode pairs of the pattern, NumPy), and at
  rho = infinity the dense Cholesky factor.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs
from tests import refmath


def _pseudo(x, lev, l1, a, b):
    k = min(lev[a], lev[b])
    return math.sqrt(oracle.lib().ko_d2(np.ascontiguousarray(x[a]), np.ascontiguousarray(x[b]), x.shape[1])) / (
        l1 * 2.0 ** -k)


@pytest.mark.parametrize("N,d,rho", [(700, 2, 2.0), (700, 2, 3.0), (500, 3, 2.5)])
def test_construction_properties(N, d, rho):
    x = inputs.uniform(N, d, seed=91)
    r = oracle.supernodal(x, rho)
    perm, l = r["perm"], r["l"]
    l1 = l[1]
    # levels of the maximin positions, from their definition
    lev_m = np.ones(N, int)
    for m in range(1, N):
        k = 1
        while not l[m] >= math.ldexp(l1, -k):
            k += 1
        lev_m[m] = k
    # per new position: maximin index m, its level and supernode
    inv = np.empty(N, int)
    inv[perm] = np.arange(N)
    m_of = inv[r["order"]]
    assert np.array_equal(r["level"], lev_m[m_of])
    xo = x[perm]
    node = np.empty(N, int)
    node[m_of] = r["node"]
    sups = np.unique(node)
    assert np.all(node[sups] == sups)  # a supernode belongs to itself
    R = rho * l1
    for s in sups:
        for t in sups:
            if s < t and lev_m[s] == lev_m[t]:
                assert math.sqrt(oracle.lib().ko_d2(xo[s], xo[t], d)) > math.ldexp(R, -int(lev_m[s]))
    for m in range(N):
        s = node[m]
        assert lev_m[s] == lev_m[m]
        dm = oracle.lib().ko_d2(xo[m], xo[s], d)
        assert math.sqrt(dm) <= math.ldexp(R, -int(lev_m[m]))
        same = sups[lev_m[sups] == lev_m[m]]
        d2s = np.array([oracle.lib().ko_d2(xo[m], xo[t], d) for t in same])
        assert dm == d2s.min() and s == same[d2s == dm].min()
    # ordering: levels nondecreasing, then colours, supernodes contiguous
    lv, co, nd = r["level"], r["color"], r["node"]
    key = lv.astype(np.int64) * 10**6 + co
    assert np.all(np.diff(key) >= 0)
    starts = {}
    for q in range(N):
        starts.setdefault(nd[q], q)
    for q in range(N):
        assert q - starts[nd[q]] == np.count_nonzero(nd[starts[nd[q]]:q + 1] == nd[q]) - 1
    # supernode pattern from S: (A, B) adjacent iff the block is in S
    S = refmath.pattern_mask(r["rowptr"], r["col"], N)
    adj = {}
    for q in range(N):
        for p in r["col"][r["rowptr"][q]:r["rowptr"][q + 1]]:
            adj.setdefault(nd[q], set()).add(nd[p])
            adj.setdefault(nd[p], set()).add(nd[q])
    # blocks: S is the union of full supernode blocks (lower triangle)
    for q in range(N):
        for p in range(q + 1):
            assert S[q, p] == (nd[p] in adj.get(nd[q], set()))
    # every pair with d <= rho is in S
    xs = x[r["order"]]
    for q in range(N):
        for p in range(q):
            kmin = min(lv[q], lv[p])
            if math.sqrt(oracle.lib().ko_d2(xs[q], xs[p], d)) <= math.ldexp(R, -int(kmin)):
                assert S[q, p]
    # colours: valid on same-level adjacent supernodes, greedy-minimal
    col_of = {nd[q]: co[q] for q in range(N)}
    lev_of = {nd[q]: lv[q] for q in range(N)}
    for a, nb in adj.items():
        earlier = [b for b in nb if b != a and lev_of[b] == lev_of[a]]
        assert all(col_of[b] != col_of[a] for b in earlier)
        used = {col_of[b] for b in earlier if b < a}
        assert all(c in used for c in range(col_of[a]))


def _block_ichol(A, node):
    """The supernodal block factorisation of the stability appendix, restated
    as a block Cholesky whose Schur-complement updates are kept only on the
    supernode pairs of the pattern: for each supernode I in order, its
    diagonal block is factored densely (L_II L_II^T = A_II), the rows below
    are L_KI = A_KI L_II^{-T}, and the trailing matrix loses L_KI L_JI^T on the
    block pairs (K, J) the pattern contains.  A is restricted to the pattern
    first (dense, on the supernodal order)."""
    N = A.shape[0]
    starts = np.flatnonzero(np.r_[True, node[1:] != node[:-1]])
    bounds = list(zip(starts, np.r_[starts[1:], N]))
    blk = np.repeat(np.arange(len(bounds)), [e - b for b, e in bounds])
    nb = len(bounds)
    adj = np.zeros((nb, nb), bool)
    for u, (b0, e0) in enumerate(bounds):
        for v, (b1, e1) in enumerate(bounds):
            adj[u, v] = np.any(A[b0:e0, b1:e1] != 0)
    mask = adj[np.ix_(blk, blk)]
    A = A.copy()
    L = np.zeros_like(A)
    for b, e in bounds:
        C = np.linalg.cholesky(A[b:e, b:e])
        L[b:e, b:e] = C
        W = np.linalg.solve(C, A[e:, b:e].T).T
        L[e:, b:e] = W
        A[e:, e:] -= (W @ W.T) * mask[e:, e:]
    return L


@pytest.mark.parametrize("rho", [2.0, 3.0])
def test_algorithm2_equals_supernodal_block_algorithm(rho):
    x = inputs.uniform(400, 2, seed=92)
    r = oracle.supernodal(x, rho)
    kern = oracle.Kernel(0.5, 0.2, 1.0, 1e-3)
    xs = x[r["order"]]
    val, zc = oracle.ichol(xs, r["rowptr"], r["col"], kern)
    assert not zc.any()
    L = refmath.dense_lower(r["rowptr"], r["col"], val, 400)
    S = refmath.pattern_mask(r["rowptr"], r["col"], 400)
    A = np.where(S, refmath.dense_theta(xs, 0.5, 0.2, 1.0, 1e-3), 0.0)
    Lb = _block_ichol(A, r["node"])
    assert np.max(np.abs(L - Lb)) <= 1e-10 * np.max(np.abs(Lb))


def test_rho_infinity_dense_cholesky():
    x = inputs.uniform(300, 2, seed=93)
    r = oracle.supernodal(x, 1e300)
    kern = oracle.Kernel(1.5, 0.2, 1.0, 1e-3)
    xs = x[r["order"]]
    val, zc = oracle.ichol(xs, r["rowptr"], r["col"], kern)
    L = refmath.dense_lower(r["rowptr"], r["col"], val, 300)
    C = np.linalg.cholesky(refmath.dense_theta(xs, 1.5, 0.2, 1.0, 1e-3))
    assert np.max(np.abs(L - C)) <= 1e-9 * np.max(np.abs(C))
