"""The factor parity bars (tests/factor_parity.py) on the CPU: they accept a
factor computed with rounding of the GPU's kind (the oracle with every entry
rounded to float and its sums in the other order, a perturbation neither
reference uses), and reject planted mistakes of the size the bars exist to
catch.  Mistakes are planted in copies of the oracle's output."""
import numpy as np
import pytest

import oracle
from paper_1706_02205_gb300 import inputs
from tests import factor_parity as fp


def _case(nu, ell, rho, nugget, N=1500, seed=32):
    x = inputs.uniform(N, 2, seed=seed)
    perm, l, rp, col = oracle.sortsparse(x, rho)
    xo = x[perm]
    ko = oracle.Kernel(nu, ell, 1.0, nugget)
    val, zc, piv = oracle.ichol(xo, rp, col, ko, pivots=True)
    return dict(rp=rp, col=col, ref=(val, zc), piv=piv, rn=np.sqrt(1.0 + nugget),
                alt32=oracle.ichol(xo, rp, col, ko, store_f32=True),
                alt64=oracle.ichol(xo, rp, col, ko, reverse_sums=True),
                other32=oracle.ichol(xo, rp, col, ko, store_f32=True, reverse_sums=True))


@pytest.fixture(scope="module")
def well():
    return _case(1.5, 0.2, 5.0, 1e-4)


@pytest.fixture(scope="module")
def ill():
    return _case(2.5, 0.3, 4.0, 1e-6)


def _diag(rp, val):
    return val[rp[1:] - 1]


def test_accepts_an_independent_fp32_rounding(well, ill):
    for c, strict in ((well, True), (ill, False)):
        v, z = c["other32"]
        info = fp.check_factor(1, v, _diag(c["rp"], v), c["rp"], c["col"], c["rn"], c["ref"], alt=c["alt32"],
                               piv=c["piv"], strict=strict, min_entries=0.35)
        assert info["compared"] >= 0.35 and info["max_err"] <= 1e-4
    # the ill-conditioned case really is: the old scaled bar was meaningless
    assert np.max(np.abs(ill["alt32"][0] - ill["ref"][0])) > 1e-2
    assert ill["ref"][1].sum() > 500


def test_fp64_accepts_the_oracle_itself(well):
    v, z = well["ref"]
    fp.check_factor(0, v, _diag(well["rp"], v), well["rp"], well["col"], well["rn"], well["ref"], strict=True)


def test_rejects_an_entry_off_by_twice_the_bar(well, ill):
    for c, strict in ((well, True), (ill, False)):
        v = c["other32"][0].copy()
        col, rp = c["col"], c["rp"]
        # a determined entry below the diagonal of a kept column
        sens = np.zeros(rp.shape[0] - 1)
        np.maximum.at(sens, col, np.abs(c["alt32"][0] - c["ref"][0]))
        rows = fp.rows_of(rp)
        cand = np.nonzero((sens[col] < 1e-6) & (col != rows) & ~c["ref"][1][col])[0]
        e = cand[len(cand) // 2]
        v[e] += 2e-4 * c["rn"]
        with pytest.raises(AssertionError):
            fp.check_factor(1, v, _diag(rp, v), rp, col, c["rn"], c["ref"], alt=c["alt32"], piv=c["piv"],
                            strict=strict)


def test_rejects_a_flipped_decision_at_a_determined_pivot(ill):
    c = ill
    v = c["ref"][0].copy()
    rp, col = c["rp"], c["col"]
    dg = _diag(rp, v).copy()
    kept = np.nonzero(~c["ref"][1] & (np.abs(c["piv"]) > 1e-2))[0]
    i = int(kept[0])
    dg[i] = 0.0
    with pytest.raises(AssertionError):
        fp.check_factor(1, v, dg, rp, col, c["rn"], c["ref"], alt=c["alt32"], piv=c["piv"])
    with pytest.raises(AssertionError):
        fp.check_factor(0, v, dg, rp, col, c["rn"], c["ref"], alt=c["alt64"], piv=c["piv"])


def test_rejects_fp64_error_above_1e12(well):
    v = well["ref"][0].copy()
    v[len(v) // 3] += 3e-12
    with pytest.raises(AssertionError):
        fp.check_factor(0, v, _diag(well["rp"], v), well["rp"], well["col"], well["rn"], well["ref"],
                        strict=True)


def test_rejects_a_vacuous_comparison(ill):
    """If fewer than the required share of entries are determined, the check
    fails instead of comparing almost nothing."""
    c = ill
    v = c["other32"][0]
    with pytest.raises(AssertionError):
        fp.check_factor(1, v, _diag(c["rp"], v), c["rp"], c["col"], c["rn"], c["ref"], alt=c["alt32"],
                        piv=c["piv"], min_entries=0.99)
