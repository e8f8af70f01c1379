"""Full-size checks of the other two timed workloads, in the bench's launch
configuration, on samples the oracle's arithmetic can compute one by one and
on properties that hold at any size.

* 3-D: 2^18 points uniform in [0,1]^3, Matern-5/2, l = 0.3, nugget 1e-6,
  rho = 4, FP32 form, rank-k PCA for k in {64, 512} (power iteration, 20
  steps here, 50 in the bench): sampled length scales exact, sampled pattern rows equal their
  definition, the identity (L L^T)_ji = Theta_ji on sampled entries, L_k
  equal to the first k columns of L, and the PCA error estimates ordered
  (k = 512 below k = 64 below ||Theta||).
* Batched: the 256 sets of N log-uniform in [2000, 50000] (192 2-D, 64 3-D),
  Matern-3/2, l ~ U[0.05, 0.3], rho = 3, FP32 form, in one launch: the
  smallest, a middle and the largest set equal the same sets factored alone
  bit for bit, and the smallest set agrees with the oracle's FP64 factor
  within the FP32-form bar.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import kchol as kc  # noqa: E402
from tests import factor_parity as fp  # noqa: E402

DEV = torch.device("cuda:0")


def _d2(a, P):
    s = np.zeros(P.shape[0])
    for t in range(P.shape[1]):
        w = P[:, t] - a[t]
        s = s + w * w
    return s


def _samples(N, n, seed):
    r = np.random.default_rng(seed)
    return np.unique(np.concatenate([[1, 2, 3, N - 1], np.exp(r.uniform(0, np.log(N - 1), n)).astype(np.int64)]))


def _matern52(r, ell):
    t = math.sqrt(5.0) * r / ell
    return (1.0 + t + t * t / 3.0) * math.exp(-t)


@pytest.fixture(scope="module")
def cube():
    N = 2**18
    x = inputs.uniform(N, 3, seed=inputs.seed_for(3))
    kern = kc.Kernel(2.5, 0.3, 1.0, 1e-6)
    perm, l, xo = kc.order_points(torch.from_numpy(x).to(DEV))
    pat = kc.build_pattern(xo, l, 4.0)
    val, diag, zp = kc.factor(pat, xo, kern, kc.FP32_FORM)
    L64 = kc.pca_truncate(pat, kc.FP32_FORM, val, perm, 64)
    L512 = kc.pca_truncate(pat, kc.FP32_FORM, val, perm, 512)
    v0 = torch.from_numpy(inputs.unit_vector(N, seed=inputs.seed_for(3, 9))).to(DEV)
    xd = torch.from_numpy(x).to(DEV)
    e64 = kc.pca_error(xd, kern, L64, v0, iters=20)
    e512 = kc.pca_error(xd, kern, L512, v0, iters=20)
    e0 = kc.pca_error(xd, kern, L64[:0], v0, iters=20)
    torch.cuda.synchronize()
    return dict(x=x, perm=perm.cpu().numpy(), l=l.cpu().numpy(), xo=xo.cpu().numpy(),
                rowptr=pat.rowptr.cpu().numpy(), col=pat.col.cpu().numpy(), val=val.cpu().numpy(),
                diag=diag.cpu().numpy(), zp=zp, L64=L64.cpu().numpy(), L512=L512.cpu().numpy(), e=(e0, e64, e512))


def test_cube_ordering_and_pattern(cube):
    N = cube["x"].shape[0]
    xo, l, rp, col = cube["xo"], cube["l"], cube["rowptr"], cube["col"]
    assert np.array_equal(np.sort(cube["perm"]), np.arange(N)) and np.isinf(l[0])
    assert np.all(np.diff(l[1:]) <= 0)
    R = 4.0 * l
    for j in _samples(N, 30, 5):
        d2 = _d2(xo[j], xo[:j])
        assert np.sqrt(d2.min()) == l[j], j
        want = np.nonzero(np.isinf(R[:j]) | (np.sqrt(d2) <= R[:j]))[0]
        got = col[rp[j]:rp[j + 1]]
        assert got[-1] == j and np.array_equal(got[:-1], want), j


def test_cube_factor_identity(cube):
    N = cube["x"].shape[0]
    xo, rp, col = cube["xo"], cube["rowptr"], cube["col"]
    val = cube["val"].astype(np.float64)
    val[rp[1:] - 1] = cube["diag"]
    keep = cube["diag"] > 0

    def row(j):
        return col[rp[j]:rp[j + 1]], val[rp[j]:rp[j + 1]]

    worst = 0.0
    for j in _samples(N, 40, 6):
        cj, vj = row(j)
        for i in np.random.default_rng(int(j)).choice(cj, size=min(6, len(cj)), replace=False):
            if not keep[i]:
                continue
            ci, vi = row(i)
            _, a, b = np.intersect1d(cj, ci, assume_unique=True, return_indices=True)
            llt = float(np.dot(vj[a], vi[b]))
            th = 1.0 + 1e-6 if i == j else _matern52(math.sqrt(_d2(xo[j], xo[i:i + 1])[0]), 0.3)
            worst = max(worst, abs(llt - th))
    assert worst < 1e-6 * (1.0 + 1e-6), worst


def test_cube_pca(cube):
    N = cube["x"].shape[0]
    perm, rp, col, val = cube["perm"], cube["rowptr"], cube["col"], cube["val"]
    for Lk, k in ((cube["L64"], 64), (cube["L512"], 512)):
        for j in _samples(N, 40, 7):
            c = col[rp[j]:rp[j + 1]]
            v = val[rp[j]:rp[j + 1]]
            want = np.zeros(k, np.float32)
            m = c < k
            want[c[m]] = v[m]
            assert np.array_equal(Lk[:, perm[j]], want), (k, j)
    e0, e64, e512 = cube["e"]
    assert 0 < e512 < e64 < e0


def test_batch_full_size_sets_alone_and_oracle():
    from paper_1706_02205_gb300 import batch as kb
    sets = inputs.batch_sets(n_sets=256)
    xs = [torch.from_numpy(s["x"]).to(DEV) for s in sets]
    kerns = [kc.Kernel(1.5, s["ell"]) for s in sets]
    B = kb.BatchFactor(xs, kerns, 3.0, kc.FP32_FORM, n_streams=8)
    B.factor()
    sizes = np.array([s["x"].shape[0] for s in sets])
    order = np.argsort(sizes, kind="stable")
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    for s in pick:
        r = kc.pipeline(xs[s], 3.0, kerns[s], kc.FP32_FORM)
        a, e = B.offsets[s], B.offsets[s + 1]
        assert torch.equal(B.set_values(s), r["val"]) and torch.equal(B.diag[a:e], r["diag"]), s
    s = pick[0]
    ko = oracle.Kernel(1.5, sets[s]["ell"])
    ref = oracle.pipeline(sets[s]["x"], 3.0, ko)
    assert np.array_equal(B.sets[s]["perm"].cpu().numpy(), ref["perm"])
    v = B.set_values(s).cpu().numpy().astype(np.float64)
    _, _, piv = oracle.ichol(ref["x_ord"], ref["rowptr"], ref["col"], ko, pivots=True)
    alt = oracle.ichol(ref["x_ord"], ref["rowptr"], ref["col"], ko, store_f32=True)
    fp.check_factor(kc.FP32_FORM, v, B.diag[B.offsets[s]:B.offsets[s + 1]].cpu().numpy(), ref["rowptr"],
                    ref["col"], 1.0, (ref["val"], ref["zero_col"]), alt=alt, piv=piv)
