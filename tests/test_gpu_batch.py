"""Batched launch: several independent point sets of uneven size and
dimension, each with its own length scale, factored in one persistent launch
(plan API, CUDA graph replay) must equal every set factored alone, entry for
entry (each lane's share of a row merge is fixed relative to the row's start,
so a set's sums round the same way at any offset), and the batched solve
must equal the per-set solves.
"""
import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs
from tests import factor_parity as fp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import batch as kb  # noqa: E402
from paper_1706_02205_gb300 import kchol as kc  # noqa: E402

DEV = torch.device("cuda:0")


def _sets():
    sets = inputs.batch_sets(n_sets=7, n_min=300, n_max=2500, n_d3=3, seed=inputs.seed_for(4, 11))
    xs = [torch.from_numpy(s["x"]).to(DEV) for s in sets]
    kerns = [kc.Kernel(1.5, s["ell"]) for s in sets]
    return sets, xs, kerns


@pytest.mark.parametrize("prec", [kc.FP64, kc.FP32_FORM])
def test_batch_equals_sets_alone(prec):
    sets, xs, kerns = _sets()
    opts = kc.make_opts(lanes_per_row=8, unroll=4)
    B = kb.BatchFactor(xs, kerns, 3.0, prec, opts, n_streams=3)
    zp = B.factor()
    total_zp = 0
    for s, (x, k) in enumerate(zip(xs, kerns)):
        r = kc.pipeline(x, 3.0, k, prec, opts=opts)
        total_zp += r["zero_pivots"]
        a, e = B.offsets[s], B.offsets[s + 1]
        assert torch.equal(B.sets[s]["perm"], r["perm"])
        assert torch.equal(B.set_values(s), r["val"]), s
        assert torch.equal(B.diag[a:e], r["diag"]), s
    assert zp == total_zp
    # the same launch recorded in a CUDA graph and replayed gives the same bits
    ref = B.val.clone()
    B.val.zero_()
    B.capture()
    B.replay()
    torch.cuda.synchronize()
    assert torch.equal(B.val, ref)


def test_batch_solve_and_tuner():
    sets, xs, kerns = _sets()
    B = kb.BatchFactor(xs, kerns, 3.0, kc.FP32_FORM, n_streams=4)
    best = B.tune()
    assert best["lanes_per_row"] in (2, 4, 8, 16) and best["unroll"] in (8, 16) and best["ms"] > 0
    B.factor()
    Ntot = sum(B.Ns)
    b = torch.from_numpy(inputs.rhs(Ntot, 1, seed=3)).to(DEV)
    xb = B.solve(b).cpu().numpy()[0]
    # each set solved alone with the batch's own factor values of that set
    for s, k in enumerate(kerns):
        a, e = B.offsets[s], B.offsets[s + 1]
        pat = kc.schedule(B.sets[s]["rowptr"], B.sets[s]["col"])
        xs_ = kc.solve(pat, kc.FP32_FORM, B.set_values(s).clone(), B.diag[a:e].clone(), k, B.sets[s]["perm"],
                       b[:, a:e].contiguous()).cpu().numpy()[0]
        assert np.linalg.norm(xb[a:e] - xs_) / np.linalg.norm(xs_) < 1e-11, s


def test_batch_matches_oracle_per_set():
    sets, xs, kerns = _sets()
    B = kb.BatchFactor(xs, kerns, 3.0, kc.FP64, n_streams=2)
    B.factor()
    for s in (0, 3, 6):
        ref = oracle.pipeline(sets[s]["x"], 3.0, oracle.Kernel(1.5, sets[s]["ell"]))
        assert np.array_equal(B.sets[s]["perm"].cpu().numpy(), ref["perm"])
        assert np.array_equal(B.sets[s]["col"].cpu().numpy(), ref["col"])
        v = B.set_values(s).cpu().numpy()
        dg = B.diag[B.offsets[s]:B.offsets[s + 1]].cpu().numpy()
        alt = oracle.ichol(ref["x_ord"], ref["rowptr"], ref["col"], oracle.Kernel(1.5, sets[s]["ell"]),
                           reverse_sums=True)
        fp.check_factor(kc.FP64, v, dg, ref["rowptr"], ref["col"], 1.0, (ref["val"], ref["zero_col"]), alt=alt)
