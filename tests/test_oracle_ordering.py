"""Pins of the oracle's ordering and pattern (CPU only).

* Hand-worked examples (tests/golden/maximin_1d.json, Section 2.3).
* The definition by brute force (O(N^2)) equals the paper's heap algorithm
  (Algorithm 3; Theorem "compSortSparse" states that they coincide).
* Covering/packing invariants of a maximin ordering checked with SciPy's
  distances, and the count nnz(L)/N^2 against the paper's Tables 1 and 2.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_1706_02205_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "maximin_1d.json")


def test_hand_worked_examples():
    cases = json.load(open(GOLD))["cases"]
    for c in cases:
        x = np.array(c["x"])[:, None]
        perm, l = oracle.maximin_brute(x)
        assert perm.tolist() == c["perm"], c["name"]
        assert l.tolist() == c["l"], c["name"]
        rp, col = oracle.pattern(x[perm], l, c["rho"])
        assert rp.tolist() == c["rowptr"] and col.tolist() == c["col"], c["name"]
        p2, l2, rp2, col2 = oracle.sortsparse(x, max(c["rho"], 1.0))
        assert p2.tolist() == c["perm"] and rp2.tolist() == c["rowptr"] and col2.tolist() == c["col"]


@pytest.mark.parametrize("N,d,seed", [(1, 2, 0), (2, 2, 1), (3, 3, 2), (700, 2, 3), (1500, 3, 4), (2500, 2, 5)])
def test_brute_equals_heap_uniform(N, d, seed):
    x = inputs.uniform(N, d, seed=seed)
    p1, l1 = oracle.maximin_brute(x)
    for rho in (2.0, 3.0):
        p2, l2, rp2, col2 = oracle.sortsparse(x, rho)
        assert np.array_equal(p1, p2)
        assert np.array_equal(l1, l2)
        rp, col = oracle.pattern(x[p1], l1, rho)
        assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
        rpm, colm = oracle.pattern(x[p1], l1, rho, oracle.RULE_MIN)
        p3, l3, rp3, col3 = oracle.sortsparse(x, rho, oracle.RULE_MIN)
        assert np.array_equal(rpm, rp3) and np.array_equal(colm, col3)


def test_brute_equals_heap_ties_integer_grid():
    g = np.stack(np.meshgrid(np.arange(23.0), np.arange(19.0), indexing="ij"), -1).reshape(-1, 2)
    g = g[inputs.rng(11).permutation(len(g))]
    p1, l1 = oracle.maximin_brute(g)
    p2, l2, rp2, col2 = oracle.sortsparse(g, 2.0)
    assert np.array_equal(p1, p2) and np.array_equal(l1, l2)
    rp, col = oracle.pattern(g[p1], l1, 2.0)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


def test_brute_equals_heap_other_shapes():
    for x in (inputs.jittered_grid(40, seed=3), inputs.swiss_roll(1200, seed=4)):
        p1, l1 = oracle.maximin_brute(x)
        p2, l2, rp2, col2 = oracle.sortsparse(x, 3.0)
        assert np.array_equal(p1, p2) and np.array_equal(l1, l2)
        rp, col = oracle.pattern(x[p1], l1, 3.0)
        assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


def test_maximin_invariants_scipy():
    x = inputs.uniform(600, 2, seed=21)
    perm, l = oracle.maximin_brute(x)
    assert perm[0] == 0 and np.isinf(l[0])
    assert sorted(perm.tolist()) == list(range(600))
    assert np.all(np.diff(l[1:]) <= 0)                      # non-increasing
    D = cdist(x[perm], x[perm])
    for k in range(1, 600):
        # l[k] is the distance of the k-th point to the earlier ones
        assert np.isclose(D[k, :k].min(), l[k], rtol=1e-14, atol=0)
        # covering: every later point is within l[k] of the first k points
        if k + 1 < 600:
            assert D[k:, :k].min(axis=1).max() <= l[k] * (1 + 1e-14)
    # packing: the first k points are pairwise at least l[k-1] apart
    for k in (5, 50, 300):
        sub = D[:k, :k] + np.diag(np.full(k, np.inf))
        assert sub.min() >= l[k - 1] * (1 - 1e-14)


def test_pattern_definition_scipy():
    x = inputs.uniform(400, 3, seed=8)
    perm, l = oracle.maximin_brute(x)
    rho = 2.5
    rp, col = oracle.pattern(x[perm], l, rho)
    D = cdist(x[perm], x[perm])
    N = 400
    for j in range(N):
        expect = [i for i in range(j) if D[i, j] <= rho * l[i]] + [j]
        assert col[rp[j]:rp[j + 1]].tolist() == expect
    # the diagonal is last in every row and rows are ascending
    assert np.all(col[rp[1:] - 1] == np.arange(N))


@pytest.mark.parametrize("d,expect", [(2, 5.26e-3), (3, 1.30e-2)])
def test_nnz_matches_paper_table(d, expect):
    """nnz(L)/N^2 at N=20000, rho=3, uniform points (Table 1 and Table 2, first
    rows).  Other random points: the count agrees to a few percent."""
    N = 20000
    x = inputs.uniform(N, d, seed=inputs.seed_for(1, 100 + d))
    perm, l, rp, col = oracle.sortsparse(x, 3.0)
    ratio = rp[-1] / N**2
    assert abs(ratio / expect - 1.0) < 0.03, ratio
