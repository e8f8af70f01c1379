"""Full-size checks: the 1024 x 1024 jittered grid (N = 2^20), Matern-1/2 with
l = 0.1, rho = 3, FP32 form, with the same default options as the timed bench
step.

* ordering and pattern against the oracle: the whole permutation, every
  length scale and every row of S bit-exact against the oracle's Algorithm 3
  (its heap algorithm, Section 4.1), which runs at this size in about 80 s;
* factor against the oracle: every entry of the FP32-form and of the FP64
  factor against the oracle's ICHOL(0) (about 2 minutes at this size) within
  the fixed bars (1e-4 and 1e-12 of the row norm): Matern-1/2 keeps every
  pivot far from zero, so the whole factor is compared;

The rest is checked on samples the oracle can compute one by one, and through
properties that hold at any size:

* ordering: a permutation starting at original index 0 with non-increasing
  l; l[k] of sampled positions equals the exact distance to the nearest
  earlier point (bit for bit, same rounded operations); at sampled steps no
  later point lies farther from the earlier ones than l[k] (the greedy rule);
* pattern: sampled rows equal their definition (Section 2.3, max rule),
  checked by brute force over every earlier point;
* factor: the defining identity of ICHOL(0), (L L^T)_ji = Theta_ji on S,
  for 10^5 sampled entries of S (pivots included), within the FP32 form's
  bar of 1e-6 of Theta_jj;
* solve: the residual of L L^T x = b for two right-hand sides, with L's
  diagonal the FP64 pivots the solves divide by;
* the block factorisation by column groups on the supernodal multicolour
  pattern of the same points (default options, as the bench times it): the
  same bits with another task size, and the defining identity on 10^5
  sampled entries of the columns it keeps.
"""
import numpy as np
import pytest

from paper_1706_02205_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import kchol as kc  # noqa: E402

DEV = torch.device("cuda:0")
N_SIDE, RHO, NU, ELL = 1024, 3.0, 0.5, 0.1


@pytest.fixture(scope="module")
def full():
    x = inputs.jittered_grid(N_SIDE, seed=inputs.seed_for(2))
    kern = kc.Kernel(NU, ELL)
    perm, l, xo = kc.order_points(torch.from_numpy(x).to(DEV))
    pat = kc.build_pattern(xo, l, RHO)
    val, diag, zp = kc.factor(pat, xo, kern, kc.FP32_FORM)
    b = inputs.rhs(x.shape[0], 2, seed=inputs.seed_for(2, 61))
    xs = kc.solve(pat, kc.FP32_FORM, val, diag, kern, perm, torch.from_numpy(b).to(DEV))
    torch.cuda.synchronize()
    return dict(x=x, perm=perm.cpu().numpy(), l=l.cpu().numpy(), xo=xo.cpu().numpy(),
                rowptr=pat.rowptr.cpu().numpy(), col=pat.col.cpu().numpy(), val=val.cpu().numpy(),
                diag=diag.cpu().numpy(), zp=zp, b=b, xs=xs.cpu().numpy())


def _d2(a, P):
    """Squared distances from point a to the rows of P, coordinate by
    coordinate with every operation rounded on its own (as the kernels do)."""
    s = np.zeros(P.shape[0])
    for t in range(P.shape[1]):
        w = P[:, t] - a[t]
        s = s + w * w
    return s


def _samples(N, n, seed):
    r = np.random.default_rng(seed)
    return np.unique(np.concatenate([[1, 2, 3, N - 1], np.exp(r.uniform(0, np.log(N - 1), n)).astype(np.int64)]))


def test_full_ordering(full):
    N = full["x"].shape[0]
    perm, l, xo = full["perm"], full["l"], full["xo"]
    assert perm[0] == 0 and np.array_equal(np.sort(perm), np.arange(N))
    assert np.array_equal(xo, full["x"][perm])
    assert np.isinf(l[0]) and np.all(np.diff(l[1:]) <= 0)
    for k in _samples(N, 40, 1):
        assert np.sqrt(_d2(xo[k], xo[:k]).min()) == l[k], k
    from scipy.spatial import cKDTree
    for k in (10, 1000, 100000):
        dmin, _ = cKDTree(xo[:k]).query(xo[k:])
        assert dmin.max() <= l[k] * (1 + 1e-12), k


def test_full_pattern_rows(full):
    N = full["x"].shape[0]
    xo, l, rp, col = full["xo"], full["l"], full["rowptr"], full["col"]
    assert rp[0] == 0 and rp[-1] == len(col) and np.all(np.diff(rp) >= 1)
    R = RHO * l  # each product rounded once, as on the device
    for j in _samples(N, 40, 2):
        d2 = _d2(xo[j], xo[:j])
        want = np.nonzero(np.isinf(R[:j]) | (np.sqrt(d2) <= R[:j]))[0]
        got = col[rp[j]:rp[j + 1]]
        assert got[-1] == j and np.array_equal(got[:-1], want), j


@pytest.fixture(scope="module")
def full_oracle(full):
    """The oracle's ordering and pattern (Algorithm 3) and its FP64 factor of
    the whole 2^20 workload."""
    import time

    import oracle
    t0 = time.perf_counter()
    perm, l, rp, col = oracle.sortsparse(full["x"], RHO)
    t1 = time.perf_counter()
    val, zc = oracle.ichol(full["x"][perm], rp, col, oracle.Kernel(NU, ELL))
    t2 = time.perf_counter()
    print(f"oracle at N={len(perm)}: Algorithm 3 {t1 - t0:.1f} s, ICHOL(0) {t2 - t1:.1f} s")
    return dict(perm=perm, l=l, rowptr=rp, col=col, val=val, zero_col=zc)


def test_full_ordering_and_pattern_equal_algorithm3(full, full_oracle):
    """The whole 2^20 output against the oracle's Algorithm 3 (which the oracle
    tests pin to the brute-force definitions at smaller sizes)."""
    assert np.array_equal(full["perm"], full_oracle["perm"])
    assert np.array_equal(full["l"], full_oracle["l"])
    assert np.array_equal(full["rowptr"], full_oracle["rowptr"])
    assert np.array_equal(full["col"], full_oracle["col"])


@pytest.mark.parametrize("prec", [kc.FP32_FORM, kc.FP64])
def test_full_factor_every_entry_against_oracle(full, full_oracle, prec):
    from tests import factor_parity as fp
    assert not full_oracle["zero_col"].any()
    if prec == kc.FP32_FORM:
        val, diag = full["val"], full["diag"]
    else:
        pat = kc.build_pattern(torch.from_numpy(full["xo"]).to(DEV), torch.from_numpy(full["l"]).to(DEV), RHO)
        v, d, zp = kc.factor(pat, torch.from_numpy(full["xo"]).to(DEV), kc.Kernel(NU, ELL), kc.FP64)
        val, diag = v.cpu().numpy(), d.cpu().numpy()
        del pat, v, d
    info = fp.check_factor(prec, val, diag, full_oracle["rowptr"], full_oracle["col"], 1.0,
                           (full_oracle["val"], full_oracle["zero_col"]), strict=True)
    print(f"prec {prec}: max row-relative error over all {len(val)} entries {info['max_err']:.3e}")


def test_full_factor_identity(full):
    """(L L^T)_ji = Theta_ji on 10^5 entries of S drawn uniformly (the
    diagonal among them), each product a sparse row merge in FP64."""
    from scipy.sparse import csr_matrix
    N = full["x"].shape[0]
    xo, rp, col, val, diag = full["xo"], full["rowptr"], full["col"], full["val"].astype(np.float64), full["diag"]
    assert full["zp"] == 0 and np.all(diag > 0)
    L = csr_matrix((val, col, rp), shape=(N, N))
    r = np.random.default_rng(3)
    e = r.integers(0, len(col), size=100_000)
    e = np.concatenate([e, rp[1:][r.integers(0, N, size=2000)] - 1])  # some diagonal entries for sure
    rows = np.searchsorted(rp, e, side="right") - 1
    cols = col[e]
    llt = np.asarray(L[rows].multiply(L[cols]).sum(axis=1)).ravel()
    dist = np.sqrt(((xo[rows] - xo[cols]) ** 2).sum(axis=1))
    th = np.exp(-dist / ELL)
    worst = float(np.max(np.abs(llt - th)))
    assert worst < 1e-6, worst


def test_full_solve_residual(full):
    from scipy.sparse import csr_matrix
    N = full["x"].shape[0]
    data = full["val"].astype(np.float64)
    data[full["rowptr"][1:] - 1] = full["diag"]  # the solves divide by the FP64 pivots (diag)
    L = csr_matrix((data, full["col"], full["rowptr"]), shape=(N, N))
    perm = full["perm"]
    for r in range(full["b"].shape[0]):
        xp = full["xs"][r][perm]
        bp = full["b"][r][perm]
        res = L @ (L.T @ xp) - bp
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(bp), r


def test_full_supernodal_block_factor(full):
    """kc_factor_blocked on the supernodal multicolour pattern built from this
    maximin order and pattern (the bench's supernodal leg): default options
    (512 rows per task here) and 96 rows per task give the same bits, and
    (L L^T)_ji = Theta_ji holds on 10^5 sampled entries of S whose column i
    is kept (a dropped column is zero, diagonal included), within the FP32
    form's bar of 1e-6."""
    from scipy.sparse import csr_matrix
    xo_d = torch.from_numpy(full["xo"]).to(DEV)
    l_d = torch.from_numpy(full["l"]).to(DEV)
    pat0 = kc.build_pattern(xo_d, l_d, RHO)
    sn = kc.supernodal(xo_d, l_d, RHO, pat0, with_schedule=False)
    del pat0
    spat = kc.schedule(sn["rowptr"], sn["col"], sn["x_new"])
    kern = kc.Kernel(NU, ELL)
    v, d, zp = kc.factor_blocked(spat, sn["x_new"], kern, kc.FP32_FORM)
    v2, d2, zp2 = kc.factor_blocked(spat, sn["x_new"], kern, kc.FP32_FORM, kc.make_opts(rows_per_task=96))
    assert torch.equal(v, v2) and torch.equal(d, d2) and zp == zp2
    del v2, d2
    xn, rp, col = sn["x_new"].cpu().numpy(), spat.rowptr.cpu().numpy(), spat.col.cpu().numpy()
    val, diag = v.cpu().numpy(), d.cpu().numpy()
    del v, d, spat, sn
    N = xn.shape[0]
    assert np.array_equal(diag == 0.0, val[rp[1:] - 1] == 0.0) and int((diag == 0.0).sum()) == zp
    L = csr_matrix((val.astype(np.float64), col, rp), shape=(N, N))
    r = np.random.default_rng(5)
    e = np.concatenate([r.integers(0, len(col), size=100_000), rp[1:][r.integers(0, N, size=2000)] - 1])
    e = e[diag[col[e]] > 0]
    rows = np.searchsorted(rp, e, side="right") - 1
    cols = col[e]
    llt = np.asarray(L[rows].multiply(L[cols]).sum(axis=1)).ravel()
    th = np.exp(-np.sqrt(((xn[rows] - xn[cols]) ** 2).sum(axis=1)) / ELL)
    worst = float(np.max(np.abs(llt - th)))
    assert worst < 1e-6, worst
