"""Serving loop: requests admitted concurrently (each on its own stream) give
the same solutions as the same requests served one at a time; a repeat solve
against a resident factor equals the first solve bit for bit; small requests
grouped into one plan launch equal the same requests alone; an evicted factor
is refactored with the same bits; admission respects the memory budget."""
import numpy as np
import pytest

from paper_1706_02205_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_02205_gb300 import kchol as kc  # noqa: E402
from paper_1706_02205_gb300 import serve  # noqa: E402


def _reqs(n=6, repeat_frac=0.0, n_max=20000, seed=3):
    reqs = inputs.serving_requests(n, rate_hz=100.0, n_min=2000, n_max=n_max, seed=inputs.seed_for(5, seed),
                                   repeat_frac=repeat_frac)
    return reqs, serve.make_payloads(reqs)


def test_mix_equals_alone():
    reqs, pay = _reqs()
    alone = serve.Server(max_inflight=1, keep_solutions=True, group_n_max=0).run(reqs, pay, realtime=False)
    srv = serve.Server(max_inflight=3, keep_solutions=True, group_n_max=0)
    mix = srv.run(reqs, pay, realtime=False)
    assert srv.max_inflight_seen > 1
    for a, m in zip(alone, mix):
        assert a["error"] is None and m["error"] is None
        assert a["nnz"] == m["nnz"]
        assert np.array_equal(a["x"], m["x"]), a["id"]  # deterministic kernels: the same bits


def _factor_then_solve(req, x, b, gap=0.0):
    """A factor request with right-hand sides b, then a repeat solve of the
    same b against its resident factor."""
    f = dict(req, type="factor", t_arrival=0.0)
    s = {"id": req["id"] + 1000, "type": "solve", "key": req["key"], "t_arrival": gap, "N": x.shape[0],
         "nrhs": b.shape[0], "seed": 0}
    return [f, s], [(x, b), (None, b)]


def test_repeat_solve_equals_first_bit_for_bit():
    reqs, pay = _reqs(2)
    rs, ps = [], []
    for r, (x, b) in zip(reqs, pay):
        a, p = _factor_then_solve(r, x, b)
        rs += a
        ps += p
    srv = serve.Server(max_inflight=2, keep_solutions=True, group_n_max=0)
    recs = srv.run(rs, ps, realtime=False)
    assert all(r["error"] is None for r in recs)
    for k in range(0, len(recs), 2):
        first, again = recs[k], recs[k + 1]
        assert first["type"] == "factor" and again["type"] == "solve" and again["cache"] == "hit"
        assert np.array_equal(first["x"], again["x"])
    # and the solution solves the system: residual with the resident factor
    res = srv.cache.get(reqs[0]["key"])
    assert res is not None


def test_grouped_small_requests_equal_alone():
    """Small factor requests that arrive together go into one plan launch; each
    request's solution equals the same request served alone (the factor bits
    are the same; the solves differ only in the padded right-hand-side
    layout)."""
    reqs, pay = _reqs(6)
    grouped = serve.Server(max_inflight=1, keep_solutions=True, group_n_max=10**6)
    g = grouped.run(reqs, pay, realtime=False)
    assert max(r["group"] for r in g) > 1
    alone = serve.Server(max_inflight=1, keep_solutions=True, group_n_max=0).run(reqs, pay, realtime=False)
    for a, b in zip(alone, g):
        assert a["error"] is None and b["error"] is None
        rel = np.linalg.norm(a["x"] - b["x"]) / np.linalg.norm(a["x"])
        assert rel < 1e-11, (a["id"], rel)
    # a repeat solve against a grouped (now resident) factor builds its schedule once and agrees
    r0 = reqs[0]
    b = pay[0][1]
    s = {"id": 99, "type": "solve", "key": r0["key"], "t_arrival": 0.0, "N": pay[0][0].shape[0],
         "nrhs": b.shape[0], "seed": 0}
    again = grouped.run([s], [(None, b)], realtime=False)[0]
    assert again["cache"] == "hit"
    assert np.linalg.norm(again["x"] - g[0]["x"]) / np.linalg.norm(g[0]["x"]) < 1e-11


def test_eviction_then_refactor_same_bits():
    """A budget that holds one resident factor: the second factor evicts the
    first, and a later solve on the first refactors it from its points, with
    the same bits as its first solve."""
    reqs, pay = _reqs(2)
    (xa, ba), (xb, bb) = pay
    fa = dict(reqs[0], type="factor", t_arrival=0.0)
    fb = dict(reqs[1], type="factor", t_arrival=0.0)
    sa = {"id": 77, "type": "solve", "key": fa["key"], "t_arrival": 0.0, "N": xa.shape[0], "nrhs": ba.shape[0],
          "seed": 0}
    need = max(serve.estimate_bytes(x.shape[0], x.shape[1], r["rho"], b.shape[0],
                                    2 if r["kind"] == "swiss" else None) for r, (x, b) in zip(reqs, pay))
    srv = serve.Server(max_inflight=1, keep_solutions=True, group_n_max=0, hbm_budget_bytes=need + 1)
    recs = srv.run([fa, fb, sa], [(xa, ba), (xb, bb), (None, ba)], realtime=False)
    assert all(r["error"] is None for r in recs)
    assert srv.cache.evictions >= 1
    assert recs[2]["cache"] == "miss"
    assert np.array_equal(recs[0]["x"], recs[2]["x"])


def test_memory_admission_serialises():
    reqs, pay = _reqs(4, repeat_frac=0.5)
    srv = serve.Server(max_inflight=4, hbm_budget_bytes=1)
    recs = srv.run(reqs, pay, realtime=False)
    assert srv.max_inflight_seen == 1
    assert all(r["error"] is None for r in recs)
    s = serve.summarize(recs, srv.wall_s)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_realtime_stream_with_repeats():
    """A short Poisson stream with repeat solves: every request completes,
    repeat solves hit resident factors, latency is arrival to completion."""
    reqs, pay = _reqs(12, repeat_frac=0.5, seed=4)
    srv = serve.Server(max_inflight=3)
    recs = srv.run(reqs, pay, realtime=True)
    s = serve.summarize(recs, srv.wall_s)
    assert s["errors"] == 0 and s["requests"] == 12
    assert s["solve_cache_hits"] == sum(1 for r in reqs if r["type"] == "solve")
    assert all(r["latency_ms"] > 0 for r in recs)


def test_footprint_estimate_covers_measured_pattern():
    reqs, pay = _reqs(3)
    for r, (x, b) in zip(reqs, pay):
        _, res, info = serve.factor_one(r, x, b, torch.cuda.Stream())
        # the estimate assumes ~48 B per entry of L; it must not undercount nnz
        est = serve.estimate_bytes(x.shape[0], x.shape[1], r["rho"], b.shape[0],
                                   2 if r["kind"] == "swiss" else None)
        assert est >= 48 * info["nnz"]
        assert res.nbytes() < est


def test_factor_headroom_gives_the_same_bits():
    """A persistent factor that leaves CTA slots free (ctas_per_sm < 0, as the
    server launches it next to its solve lanes) computes the same bits; a
    request for more headroom than the SM has runs on one CTA per SM."""
    reqs, pay = _reqs(1)
    x = torch.from_numpy(pay[0][0]).cuda()
    perm, l, xo = kc.order_points(x)
    pat = kc.build_pattern(xo, l, 3.0)
    kern = kc.Kernel(1.5, 0.1)
    for prec in (kc.FP32_FORM, kc.FP64):
        v0, d0, z0 = kc.factor(pat, xo, kern, prec)
        for c in (-1, -64):
            v1, d1, z1 = kc.factor(pat, xo, kern, prec, kc.make_opts(ctas_per_sm=c))
            assert torch.equal(v0, v1) and torch.equal(d0, d1) and z0 == z1
