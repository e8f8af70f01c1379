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


def test_summary_splits_latency_into_wait_and_service():
    """p50/p99 over all requests and per type; a request's latency is its
    queue wait (arrival to admission) plus its service (admission to done)."""
    recs = []
    for i in range(10):
        typ = "factor" if i % 2 == 0 else "solve"
        arr, adm, done = 0.1 * i, 0.1 * i + 0.01 * i, 0.1 * i + 0.01 * i + (0.2 if typ == "factor" else 0.05)
        recs.append({"id": i, "type": typ, "key": i, "N": 10, "nnz": 100 if typ == "factor" else 0,
                     "cache": "new" if typ == "factor" else "hit", "group": 1, "t_arrival": arr, "t_admit": adm,
                     "t_done": done, "latency_ms": (done - arr) * 1e3, "x": None, "error": None})
    s = serve.summarize(recs, wall_s=2.0)
    assert s["requests"] == 10 and s["errors"] == 0 and s["throughput_req_s"] == 5.0
    assert s["factor"]["n"] == 5 and s["solve"]["n"] == 5
    for typ, service in (("factor", 200.0), ("solve", 50.0)):
        assert s[typ]["service_p50_ms"] == pytest.approx(service)
        waits = [(r["t_admit"] - r["t_arrival"]) * 1e3 for r in recs if r["type"] == typ]
        assert s[typ]["wait_p50_ms"] == pytest.approx(float(np.percentile(waits, 50)))
        lat = [r["latency_ms"] for r in recs if r["type"] == typ]
        assert s[typ]["p50_ms"] == pytest.approx(float(np.percentile(lat, 50)))
    assert s["solve_cache_hits"] == 5 and s["refactors"] == 0
    assert s["factor_nnz_per_s"] == pytest.approx(5 * 100 / 2.0)
