"""Full-size checks: the 1024 x 1024 jittered grid (N = 2^20), Matern-1/2 with
l = 0.1, rho = 3, FP32 form, with the same default options as the timed bench
step.  The oracle cannot run the whole path at this size in a test, so the
outputs are checked on samples it can compute one by one, and through
properties that hold at any size:

* ordering: a permutation starting at original index 0 with non-increasing
  l; l[k] of sampled positions equals the exact distance to the nearest
  earlier point (bit for bit, same rounded operations); at sampled steps no
  later point lies farther from the earlier ones than l[k] (the greedy rule);
* pattern: sampled rows equal their definition (Section 2.3, max rule),
  checked by brute force over every earlier point;
* factor: the defining identity of ICHOL(0), (L L^T)_ji = Theta_ji on S,
  for sampled entries and the pivots of sampled columns, within the FP32
  form's bar of 1e-6 of Theta_jj;
* solve: the residual of L L^T x = b for two right-hand sides, with L's
  diagonal the FP64 pivots the solves divide by.
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


def test_full_factor_identity(full):
    N = full["x"].shape[0]
    xo, rp, col, val, diag = full["xo"], full["rowptr"], full["col"], full["val"].astype(np.float64), full["diag"]
    assert full["zp"] == 0 and np.all(diag > 0)

    def row(j):
        a, e = rp[j], rp[j + 1]
        return col[a:e], val[a:e]

    def llt(j, i):
        cj, vj = row(j)
        ci, vi = row(i)
        _, a, b = np.intersect1d(cj, ci, assume_unique=True, return_indices=True)
        return float(np.dot(vj[a], vi[b]))

    worst = 0.0
    for j in _samples(N, 60, 3):
        cj, _ = row(j)
        for i in np.random.default_rng(int(j)).choice(cj, size=min(8, len(cj)), replace=False):
            th = np.exp(-np.sqrt(_d2(xo[j], xo[i:i + 1])[0]) / ELL) if i != j else 1.0
            worst = max(worst, abs(llt(j, i) - th))
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
