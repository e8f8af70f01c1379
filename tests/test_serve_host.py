"""Host logic of the serving loop on the CPU: the resident-factor cache evicts
least recently used first and never a pinned factor; the request stream's
repeat solves refer to point sets requested earlier."""
import numpy as np
import pytest

from paper_1706_02205_gb300 import inputs

torch = pytest.importorskip("torch")

from paper_1706_02205_gb300 import serve  # noqa: E402


def _res(key, n):
    z = torch.zeros(n, dtype=torch.float64)
    i = torch.zeros(n, dtype=torch.int32)
    return serve.Resident(key, n, z, i, z.float(), z, None, 1, torch.zeros(n + 1, dtype=torch.int64), i)


def test_cache_lru_order_and_pins():
    c = serve.FactorCache()
    for k in "abcd":
        c.put(_res(k, 100))
    per = c.entries["a"].nbytes()
    assert c.bytes == 4 * per
    c.get("a")                      # a becomes the most recently used
    c.entries["b"].pins = 1         # b is in use
    c.evict_until(2 * per)          # two must go: c, d are the oldest unpinned after b
    assert list(c.entries) == ["b", "a"] and c.evictions == 2 and c.bytes == 2 * per
    c.evict_until(0)
    assert list(c.entries) == ["b"]  # pinned: never evicted
    c.entries["b"].pins = 0
    c.evict_until(0)
    assert not c.entries and c.bytes == 0


def test_cache_replaces_same_key():
    c = serve.FactorCache()
    c.put(_res("a", 10))
    c.put(_res("a", 50))
    assert len(c.entries) == 1 and c.bytes == c.entries["a"].nbytes()


def test_request_stream_repeats_refer_to_earlier_sets():
    reqs = inputs.serving_requests(200, rate_hz=5.0, seed=inputs.seed_for(5, 9), repeat_frac=0.5)
    seen = {}
    t = 0.0
    for r in reqs:
        assert r["t_arrival"] >= t
        t = r["t_arrival"]
        assert 1 <= r["nrhs"] <= 8
        if r["type"] == "factor":
            assert 10_000 <= r["N"] <= 1_000_000 and r["rho"] in (3.0, 4.0)
            assert r["d"] in (2, 3, 20) and (r["d"] == 20) == (r["kind"] == "swiss")
            seen[r["key"]] = r["N"]
        else:
            assert r["key"] in seen and r["N"] == seen[r["key"]]
    n_solve = sum(r["type"] == "solve" for r in reqs)
    assert 60 <= n_solve <= 140
    # the same seed gives the same stream; repeat_frac = 0 gives factors only
    assert inputs.serving_requests(20, 5.0, seed=3) == inputs.serving_requests(20, 5.0, seed=3)
    assert all(r["type"] == "factor" for r in inputs.serving_requests(30, 5.0, seed=3, repeat_frac=0.0))


def test_solve_payload_shapes():
    reqs = inputs.serving_requests(8, rate_hz=5.0, n_min=2000, n_max=4000, seed=11, repeat_frac=0.5)
    pay = serve.make_payloads(reqs)
    for r, (x, b) in zip(reqs, pay):
        assert b.shape == (r["nrhs"], r["N"])
        assert (x is None) == (r["type"] == "solve")
        if x is not None:
            assert x.shape == (r["N"], r["d"]) and np.isfinite(x).all()
