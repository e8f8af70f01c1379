"""kc_pattern_validate: the patterns this library builds pass, and corrupted
copies of them are reported (KC_EINVAL) without being used."""
import numpy as np
import pytest

from paper_1706_02205_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import kchol as kc  # noqa: E402

DEV = torch.device("cuda:0")


def _pattern():
    x = torch.from_numpy(inputs.uniform(2000, 2, seed=121)).to(DEV)
    perm, l, xo = kc.order_points(x)
    return x, perm, l, xo, kc.build_pattern(xo, l, 3.0)


def _copy(pat, **repl):
    a = {k: getattr(pat, k).clone() for k in ("rowptr", "col", "colptr", "rowidx", "slot", "level", "order")}
    for k, fn in repl.items():
        fn(a[k])
    return kc.Pattern(a["rowptr"], a["col"], a["colptr"], a["rowidx"], a["slot"], a["level"], a["order"], pat.depth)


def test_library_patterns_pass():
    x, perm, l, xo, pat = _pattern()
    kc.pattern_validate(pat)
    kc.pattern_validate(kc.build_pattern(xo, l, 2.0, kc.RULE_MIN))
    kc.pattern_validate(kc.pattern_reverse(kc.build_pattern(xo, l, 2.0, kc.RULE_MIN), xo))
    kc.pattern_validate(kc.supernodal(xo, l, 3.0, pat)["pat"])


def _set(i, v):
    def f(t):
        t[i] = v
    return f


@pytest.mark.parametrize("what,repl", [
    ("rowptr", {"rowptr": _set(5, 10**12)}),
    ("col_order", {"col": lambda t: t.__setitem__(slice(100, 102), t[100:102].flip(0))}),
    ("col_range", {"col": _set(300, -4)}),
    ("colptr", {"colptr": _set(-1, 7)}),
    ("rowidx", {"rowidx": _set(50, 10**9)}),
    ("slot", {"slot": lambda t: t.__setitem__(40, t[41])}),
    ("order", {"order": lambda t: t.__setitem__(3, t[4])}),
])
def test_corrupt_copies_are_reported(what, repl):
    x, perm, l, xo, pat = _pattern()
    bad = _copy(pat, **repl)
    with pytest.raises(kc.KcError) as ei:
        kc.pattern_validate(bad)
    assert ei.value.status == kc.KC_EINVAL
    kc.pattern_validate(pat)  # the original is untouched and passes


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
@pytest.mark.parametrize("where", [0, 777, 3999])
def test_non_finite_points_rejected(bad, where):
    """A non-finite coordinate anywhere in the input (first, middle, last
    element) is reported as KC_EINVAL by the ordering and by the pattern
    count, before any other device work; the context stays usable."""
    x_h = inputs.uniform(2000, 2, seed=122)
    xb = x_h.copy().reshape(-1)
    xb[where] = bad
    xb = xb.reshape(2000, 2)
    with pytest.raises(kc.KcError) as ei:
        kc.order_points(torch.from_numpy(xb).to(DEV))
    assert ei.value.status == kc.KC_EINVAL and "finite" in str(ei.value)
    x = torch.from_numpy(x_h).to(DEV)
    perm, l, xo = kc.order_points(x)
    xo_bad = xo.clone().view(-1)
    xo_bad[where] = bad
    with pytest.raises(kc.KcError) as ei:
        kc.pattern_count(xo_bad.view(2000, 2), l, 3.0)
    assert ei.value.status == kc.KC_EINVAL
    # the same call on the clean input still works and agrees with itself
    rp, nnz = kc.pattern_count(xo, l, 3.0)
    assert nnz == kc.build_pattern(xo, l, 3.0).nnz


@pytest.mark.parametrize("bad", ["repeated", "out_of_range"])
def test_solve_with_a_perm_that_is_no_permutation(bad):
    """The permutation steps of the solve touch nothing outside their arrays
    when perm is not a permutation (repeated or out-of-range indices): the
    call completes and the context stays usable; a later solve with the real
    permutation gives its usual result bit for bit."""
    x, perm, l, xo, pat = _pattern()
    kern = kc.Kernel(0.5, 0.2)
    val, diag, _ = kc.factor(pat, xo, kern, kc.FP64)
    b = torch.from_numpy(inputs.rhs(2000, 3, seed=122)).to(DEV)
    ref = kc.solve(pat, kc.FP64, val, diag, kern, perm, b)
    wrong = perm.clone()
    if bad == "repeated":
        wrong[:1000] = wrong[1000:]
    else:
        wrong[::7] = 10**6
    kc.solve(pat, kc.FP64, val, diag, kern, wrong, b)
    torch.cuda.synchronize()
    again = kc.solve(pat, kc.FP64, val, diag, kern, perm, b)
    assert torch.equal(again, ref)
