"""A serving loop for factor-and-solve requests on one GPU.

Two kinds of request arrive on a timeline:

* ``factor``: a point set (with its kernel, rho and right-hand sides) to
  order, pattern, schedule, factor and solve; the factor then stays resident
  on the device under the request's ``key``;
* ``solve``: right-hand sides for the resident factor of ``key`` (the paper's
  task (2) repeated against one factorisation).  If that factor was evicted,
  the request refactors it from the point set registered under the key.

Scheduling (continuous batching, not a queue drained one at a time):

* requests are admitted in arrival order as soon as a worker slot is free
  and their device-memory footprint fits the HBM budget next to the resident
  factors; admitted jobs run concurrently, each on its own CUDA stream (host
  worker threads; the library calls release the GIL), so their kernels
  overlap on the device;
* resident factors are counted in the budget and evicted least recently
  used first when a new job needs the memory (never one a running job uses);
* small factor requests that have arrived by the time one of them is
  admitted are grouped (same rho and sigma2/nugget) into one batched job:
  their patterns are concatenated and factored by one persistent plan
  launch, and solved together;
* solve requests for the same factor that are waiting are coalesced into one
  solve with their right-hand sides side by side (at most 16).

Latency = completion - arrival.
"""
from __future__ import annotations

import math
import threading
import time
from collections import OrderedDict
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np
import torch

from . import inputs
from . import kchol as kc

SERVE_KERNEL = dict(nu=1.5, ell=0.1)


def estimate_bytes(N: int, d: int, rho: float, nrhs: int, intrinsic_d: int | None = None) -> int:
    """A-priori device footprint of one factor job (before its pattern exists).

    nnz(L)/N grows like a * rho^d * ln N (Section 2.3: C rho^d N log N entries);
    a = 1.45 fits the 2-D counts measured here and overestimates 3-D ones.
    Peak bytes per entry: column indices, CSC rows and slots, values, and the
    schedule's sort buffers (about 48 B); plus per-point and right-hand-side
    arrays."""
    return int(estimate_nnz(N, d, rho, intrinsic_d) * 48 + N * (d * 8 * 4 + 96) + nrhs * N * 8 * 4 + (64 << 20))


def estimate_nnz(N: int, d: int, rho: float, intrinsic_d: int | None = None) -> float:
    de = intrinsic_d if intrinsic_d is not None else min(d, 3)
    return N * min(1.45 * rho ** de * math.log(max(N, 2)), N)


def solve_bytes(N: int, nrhs: int) -> int:
    """Footprint of one solve job on a resident factor: the right-hand sides in
    and out, the point-major copies and the solver's work vectors."""
    ns = 1 << max(0, (max(nrhs, 1) - 1).bit_length())
    return int(N * 8 * (2 * nrhs + 5 * ns) + N * 16 + (16 << 20))


@dataclass
class Resident:
    """A factor kept on the device for repeated solves."""
    key: object
    N: int
    x_ord: torch.Tensor
    perm: torch.Tensor
    val: torch.Tensor
    diag: torch.Tensor
    kern: kc.Kernel
    prec: int
    rowptr: torch.Tensor
    col: torch.Tensor
    pat: kc.Pattern | None = None   # schedule of the pattern (built on first solve for grouped sets)
    pins: int = 0
    lock: threading.Lock = field(default_factory=threading.Lock)

    def nbytes(self) -> int:
        t = [self.x_ord, self.perm, self.val, self.diag, self.rowptr, self.col]
        if self.pat is not None:
            t += [self.pat.colptr, self.pat.rowidx, self.pat.slot, self.pat.level, self.pat.order]
        return int(sum(a.numel() * a.element_size() for a in t))

    def pattern(self, stream) -> kc.Pattern:
        with self.lock:
            if self.pat is None:
                self.pat = kc.schedule(self.rowptr, self.col, self.x_ord, stream=stream)
            return self.pat


class FactorCache:
    """Resident factors by key, least recently used first; not thread-safe on
    its own (the server calls it under its condition variable)."""

    def __init__(self):
        self.entries: OrderedDict = OrderedDict()
        self.bytes = 0
        self.evictions = 0

    def get(self, key):
        e = self.entries.get(key)
        if e is not None:
            self.entries.move_to_end(key)
        return e

    def put(self, e: Resident):
        old = self.entries.pop(e.key, None)
        if old is not None:
            self.bytes -= old.nbytes()
        self.entries[e.key] = e
        self.bytes += e.nbytes()

    def evictable(self) -> int:
        return sum(e.nbytes() for e in self.entries.values() if e.pins == 0)

    def evict_until(self, limit: int):
        """Drop unpinned entries, least recently used first, until the cache
        holds at most `limit` bytes (or nothing more can go)."""
        for key in list(self.entries.keys()):
            if self.bytes <= limit:
                break
            e = self.entries[key]
            if e.pins:
                continue
            del self.entries[key]
            self.bytes -= e.nbytes()
            self.evictions += 1

    def refresh(self, e: Resident):
        """Re-count an entry whose size changed (its schedule was built)."""
        if e.key in self.entries:
            self.bytes = sum(v.nbytes() for v in self.entries.values())


def _kernel_of(req) -> kc.Kernel:
    return kc.Kernel(req.get("nu", SERVE_KERNEL["nu"]), req.get("ell", SERVE_KERNEL["ell"]))


def factor_one(req, x_host: np.ndarray, b_host: np.ndarray, stream, prec=kc.FP32_FORM, opts=None):
    """Order, pattern, schedule, factor and solve one point set on `stream`.
    Returns (solution on the host, Resident)."""
    with torch.cuda.stream(stream):
        x = torch.from_numpy(x_host).to("cuda", non_blocking=True)
        b = torch.from_numpy(b_host).to("cuda", non_blocking=True)
        kern = _kernel_of(req)
        perm, l, xo = kc.order_points(x, stream=stream)
        pat = kc.build_pattern(xo, l, req["rho"], stream=stream)
        val, diag, zp = kc.factor(pat, xo, kern, prec, opts, stream=stream)
        xs = kc.solve(pat, prec, val, diag, kern, perm, b, stream=stream)
        out = xs.cpu()
        res = Resident(req["key"], x_host.shape[0], xo, perm, val, diag, kern, prec, pat.rowptr, pat.col, pat=pat)
    stream.synchronize()
    return out.numpy(), res, {"nnz": pat.nnz, "zero_pivots": zp}


def factor_group(reqs, xs_host, bs_host, stream, prec=kc.FP32_FORM, opts=None):
    """Factor several small point sets in one persistent plan launch (their
    patterns concatenated block-diagonally) and solve them together.
    Returns per request (solution, Resident, info)."""
    from . import batch as kb
    with torch.cuda.stream(stream):
        xs = [torch.from_numpy(x).to("cuda", non_blocking=True) for x in xs_host]
        kerns = [_kernel_of(r) for r in reqs]
        B = kb.BatchFactor(xs, kerns, reqs[0]["rho"], prec, opts=opts, n_streams=1, stream=stream)
        zp = B.factor(stream=stream)
        nr = max(b.shape[0] for b in bs_host)
        bcat = np.zeros((nr, sum(B.Ns)))
        for s, b in enumerate(bs_host):
            bcat[:b.shape[0], B.offsets[s]:B.offsets[s + 1]] = b
        xcat = B.solve(torch.from_numpy(bcat).to("cuda", non_blocking=True), stream=stream).cpu().numpy()
        out = []
        for s, r in enumerate(reqs):
            a, e = B.offsets[s], B.offsets[s + 1]
            st = B.sets[s]
            res = Resident(r["key"], e - a, st["x_ord"], st["perm"], B.set_values(s).clone(), B.diag[a:e].clone(),
                           kerns[s], prec, st["rowptr"], st["col"])
            nnz = int(B.nnz_offsets[s + 1] - B.nnz_offsets[s])
            out.append((xcat[:bs_host[s].shape[0], a:e].copy(), res, {"nnz": nnz, "zero_pivots": None}))
    stream.synchronize()
    return out, zp


def solve_resident(res: Resident, b_host: np.ndarray, stream):
    """Solve with a resident factor on `stream`."""
    with torch.cuda.stream(stream):
        b = torch.from_numpy(b_host).to("cuda", non_blocking=True)
        pat = res.pattern(stream)
        xs = kc.solve(pat, res.prec, res.val, res.diag, res.kern, res.perm, b, stream=stream)
        out = xs.cpu()
    stream.synchronize()
    return out.numpy()


class Server:
    def __init__(self, max_inflight: int = 4, hbm_budget_bytes: int | None = None, prec=kc.FP32_FORM,
                 keep_solutions: bool = False, group_n_max: int = 60_000, group_max: int = 32, solve_slots: int = 2,
                 headroom: int = 0):
        self.k = max_inflight
        self.solve_slots = solve_slots
        if hbm_budget_bytes is None:
            free, total = torch.cuda.mem_get_info()
            hbm_budget_bytes = int(0.8 * free)
        self.budget = hbm_budget_bytes
        self.prec = prec
        self.keep = keep_solutions
        self.group_n_max = group_n_max
        self.group_max = group_max
        # the solve lanes' streams take their SM slots first whenever slots free up,
        # and the persistent factor kernels leave `headroom` CTA slots per SM
        # (kc_opts.ctas_per_sm < 0), so that a repeat solve does not wait for a
        # running factorisation to end
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)] + \
                       [torch.cuda.Stream(priority=-1) for _ in range(solve_slots)]
        self.factor_opts = kc.make_opts(ctas_per_sm=-headroom) if solve_slots > 0 and headroom > 0 else None
        self.cache = FactorCache()
        self.points = {}  # key -> (host points, the factor request) for refactoring after eviction

    # -- job construction (under the condition variable) --------------------
    def _need(self, job):
        if job["type"] == "solve" and job["res"] is not None:
            return solve_bytes(job["res"].N, job["nrhs"])
        return sum(estimate_bytes(x.shape[0], x.shape[1], r["rho"], b.shape[0],
                                  2 if r.get("kind") == "swiss" else None)
                   for r, x, b in zip(job["reqs"], job["xs"], job["bs"]))

    def run(self, requests, payloads, realtime=True):
        """requests: dicts with type ('factor' or 'solve'), key, t_arrival (s),
        and for factors rho, nrhs, ...; payloads: (x_host or None, b_host) per
        request.  Returns per-request records."""
        order = sorted(range(len(requests)), key=lambda i: requests[i]["t_arrival"])
        for i in order:
            r = requests[i]
            if r.get("type", "factor") == "factor":
                self.points[r["key"]] = (payloads[i][0], r)
        cv = threading.Condition()
        state = {"inflight": 0, "solves": 0, "bytes": 0, "max_inflight": 0}
        free_streams = list(range(self.k))
        free_solve = list(range(self.k, self.k + self.solve_slots))
        records = [None] * len(requests)
        ex = ThreadPoolExecutor(max_workers=self.k + self.solve_slots)
        t0 = time.perf_counter()
        pending = []   # arrived, not admitted (indices)
        busy_keys = set()  # keys whose factor job is running
        nxt = 0

        def now():
            return time.perf_counter() - t0

        def arrived_until(t):
            nonlocal nxt
            while nxt < len(order) and (not realtime or requests[order[nxt]]["t_arrival"] <= t):
                pending.append(order[nxt])
                nxt += 1

        def make_job(head):
            """The job of the head request plus what joins it (under cv)."""
            r = requests[head]
            typ = r.get("type", "factor")
            if typ == "solve":
                res = self.cache.get(r["key"])
                if res is not None:
                    ids, nr = [head], r["nrhs"]
                    for q in pending:
                        rq = requests[q]
                        if q != head and rq.get("type") == "solve" and rq["key"] == r["key"] \
                                and nr + rq["nrhs"] <= 16:
                            ids.append(q)
                            nr += rq["nrhs"]
                    return {"type": "solve", "ids": ids, "res": res, "nrhs": nr}
                # evicted (or never seen): refactor from the registered points
                x_h, fr = self.points[r["key"]]
                rr = dict(fr, nrhs=r["nrhs"])
                return {"type": "factor", "ids": [head], "reqs": [rr], "xs": [x_h], "bs": [payloads[head][1]],
                        "refactor": True}
            x_h = payloads[head][0]
            ids, reqs_, xs, bs = [head], [r], [x_h], [payloads[head][1]]
            if x_h.shape[0] <= self.group_n_max:
                for q in pending:
                    rq = requests[q]
                    if len(ids) >= self.group_max:
                        break
                    if q != head and rq.get("type", "factor") == "factor" and rq["rho"] == r["rho"] \
                            and payloads[q][0].shape[0] <= self.group_n_max and rq["key"] not in self.cache.entries:
                        ids.append(q)
                        reqs_.append(rq)
                        xs.append(payloads[q][0])
                        bs.append(payloads[q][1])
            return {"type": "factor", "ids": ids, "reqs": reqs_, "xs": xs, "bs": bs, "refactor": False}

        def work(job, sid, need, t_admit):
            st = self.streams[sid]
            err = None
            sols, infos = [None] * len(job["ids"]), [{}] * len(job["ids"])
            try:
                if job["type"] == "solve":
                    bcat = np.concatenate([payloads[i][1] for i in job["ids"]], axis=0)
                    x = solve_resident(job["res"], bcat, st)
                    o = 0
                    for m, i in enumerate(job["ids"]):
                        n = payloads[i][1].shape[0]
                        sols[m] = x[o:o + n]
                        infos[m] = {"nnz": job["res"].val.numel(), "cache": "hit"}
                        o += n
                elif len(job["ids"]) == 1:
                    x, res, info = factor_one(job["reqs"][0], job["xs"][0], job["bs"][0], st, self.prec,
                                              self.factor_opts)
                    sols[0] = x
                    infos[0] = dict(info, cache="miss" if job["refactor"] else "new", group=1)
                    job["new"] = [res]
                else:
                    outs, _ = factor_group(job["reqs"], job["xs"], job["bs"], st, self.prec, self.factor_opts)
                    job["new"] = []
                    for m, (x, res, info) in enumerate(outs):
                        sols[m] = x
                        infos[m] = dict(info, cache="new", group=len(job["ids"]))
                        job["new"].append(res)
            except Exception as e:  # reported per request, the server keeps going
                err = repr(e)
                job["new"] = []
            t_done = now()
            with cv:
                if job["type"] == "solve":
                    job["res"].pins -= 1
                    self.cache.refresh(job["res"])
                for res in job.get("new", []):
                    self.cache.put(res)
                if job["type"] == "factor":
                    for r in job["reqs"]:
                        busy_keys.discard(r["key"])
                if job.get("lane") == "solve":
                    state["solves"] -= 1
                    free_solve.append(sid)
                else:
                    state["inflight"] -= 1
                    free_streams.append(sid)
                state["bytes"] -= need
                for m, i in enumerate(job["ids"]):
                    req = requests[i]
                    arr = req["t_arrival"] if realtime else 0.0
                    records[i] = {"id": req.get("id", i), "type": req.get("type", "factor"), "key": req["key"],
                                  "N": (payloads[i][0].shape[0] if payloads[i][0] is not None
                                        else (job["res"].N if job.get("res") is not None else job["xs"][0].shape[0])),
                                  "nnz": infos[m].get("nnz", 0), "cache": infos[m].get("cache"),
                                  "group": infos[m].get("group", len(job["ids"])), "t_arrival": arr,
                                  "t_admit": t_admit, "t_done": t_done, "latency_ms": (t_done - arr) * 1e3,
                                  "x": sols[m] if self.keep else None, "error": err}
                cv.notify_all()

        def try_admit():
            """The next job that can start now, or None.  Factor requests start in
            arrival order on the factor slots.  A solve on a resident factor may
            pass a factor request that waits for a slot or for memory: it runs on
            a solve lane (or a free factor slot); a solve whose factor is still
            being computed waits for it."""
            factor_seen = False
            for q in list(pending):
                rq = requests[q]
                if rq.get("type", "factor") == "solve":
                    if rq["key"] in busy_keys:
                        continue
                    if self.cache.get(rq["key"]) is not None:
                        if state["solves"] >= self.solve_slots and state["inflight"] >= self.k:
                            continue
                        job = make_job(q)
                        need = self._need(job)
                        if fits(need) or state["inflight"] + state["solves"] == 0:
                            return job, need
                        continue
                if factor_seen:
                    continue  # factor requests (and refactors) in arrival order
                factor_seen = True
                if state["inflight"] >= self.k:
                    continue
                job = make_job(q)
                need = self._need(job)
                if fits(need) or state["inflight"] + state["solves"] == 0:
                    return job, need  # (a job larger than the whole budget runs alone)
            return None

        def fits(need):
            """The memory next to the resident factors; evicts unpinned factors,
            least recently used first, to make room."""
            over = state["bytes"] + self.cache.bytes + need - self.budget
            if over > 0:
                self.cache.evict_until(max(0, self.cache.bytes - over))
                over = state["bytes"] + self.cache.bytes + need - self.budget
            return over <= 0

        while nxt < len(order) or pending:
            if not pending:
                if realtime:
                    wait = requests[order[nxt]]["t_arrival"] - now()
                    if wait > 0:
                        time.sleep(wait)
                arrived_until(now())
                continue
            with cv:
                while True:
                    arrived_until(now())
                    got = try_admit()
                    if got is not None:
                        job, need = got
                        break
                    # wait for a job to finish (or, in real time, for an arrival)
                    cv.wait(timeout=0.005 if realtime and nxt < len(order) else None)
                for i in job["ids"]:
                    pending.remove(i)
                lane_solve = job["type"] == "solve" and state["solves"] < self.solve_slots
                job["lane"] = "solve" if lane_solve else "slot"
                if job["type"] == "solve":
                    job["res"].pins += 1
                else:
                    for r in job["reqs"]:
                        busy_keys.add(r["key"])
                if lane_solve:
                    state["solves"] += 1
                else:
                    state["inflight"] += 1
                state["bytes"] += need
                state["max_inflight"] = max(state["max_inflight"], state["inflight"])
                sid = (free_solve if lane_solve else free_streams).pop(0)
            ex.submit(work, job, sid, need, now())
        ex.shutdown(wait=True)
        self.max_inflight_seen = state["max_inflight"]
        self.wall_s = time.perf_counter() - t0
        return records


def summarize(records, wall_s):
    lat = np.array([r["latency_ms"] for r in records])
    nnz = sum(r["nnz"] for r in records if r["type"] == "factor")
    out = {"requests": len(records), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "throughput_req_s": len(records) / wall_s,
           "factor_nnz_per_s": nnz / wall_s, "errors": sum(1 for r in records if r["error"])}
    for typ in ("factor", "solve"):
        lt = np.array([r["latency_ms"] for r in records if r["type"] == typ])
        if lt.size:
            wt = np.array([(r["t_admit"] - r["t_arrival"]) * 1e3 for r in records if r["type"] == typ])
            sv = np.array([(r["t_done"] - r["t_admit"]) * 1e3 for r in records if r["type"] == typ])
            out[typ] = {"n": int(lt.size), "p50_ms": float(np.percentile(lt, 50)),
                        "p99_ms": float(np.percentile(lt, 99)), "wait_p50_ms": float(np.percentile(wt, 50)),
                        "service_p50_ms": float(np.percentile(sv, 50))}
    out["solve_cache_hits"] = sum(1 for r in records if r["type"] == "solve" and r["cache"] == "hit")
    out["refactors"] = sum(1 for r in records if r["cache"] == "miss")
    out["grouped_factor_requests"] = sum(1 for r in records if r["type"] == "factor" and (r["group"] or 1) > 1)
    return out


def make_payloads(reqs):
    """(points, right-hand sides) per request; solve requests carry no points."""
    out = []
    for r in reqs:
        if r.get("type", "factor") == "factor":
            x = inputs.request_points(r)
            out.append((x, inputs.rhs(x.shape[0], r["nrhs"], seed=r["seed"] + 1)))
        else:
            out.append((None, inputs.rhs(r["N"], r["nrhs"], seed=r["seed"] + 1)))
    return out


def bench(args):
    """The request stream of the serving configuration at one load level.

    Capacity is measured with every request admitted at t = 0; the stream is
    then replayed as a Poisson process at `rate_frac` of it (and at the other
    fractions asked for)."""
    n_req = getattr(args, "n_req", 40)
    n_max = getattr(args, "serve_n_max", 1_000_000)
    fracs = getattr(args, "serve_fracs", (0.8,))
    probe = inputs.serving_requests(n_req, rate_hz=1.0, n_max=n_max, seed=inputs.seed_for(5, 1))
    payloads = make_payloads(probe)
    srv = Server(max_inflight=getattr(args, "slots", 4))
    warm = [dict(r, key=("warm", r["key"])) for r in probe[:3] if r["type"] == "factor"]
    srv.run(warm, [payloads[probe.index(r)] for r in probe[:3] if r["type"] == "factor"], realtime=False)
    srv.cache = FactorCache()
    recs = srv.run(probe, payloads, realtime=False)
    cap = len(recs) / srv.wall_s
    nf = sum(1 for r in probe if r["type"] == "factor")
    out = {"workload": f"{n_req} requests ({nf} factor+solve, {n_req - nf} repeat solves on resident factors), "
                       f"N log-U[1e4,{n_max:g}], half U[0,1]^d (d in 2,3) half swiss roll in R^20, "
                       f"Matern-3/2 l=0.1, rho in {{3,4}}, 1-8 rhs, FP32 form",
           "slots": srv.k, "hbm_budget_gb": srv.budget / 1e9, "capacity_req_s": cap,
           "capacity_run": summarize(recs, srv.wall_s), "rates": {}}
    for frac in fracs:
        reqs = inputs.serving_requests(n_req, rate_hz=frac * cap, n_max=n_max, seed=inputs.seed_for(5, 1))
        srv.cache = FactorCache()
        recs = srv.run(reqs, payloads, realtime=True)
        s = summarize(recs, srv.wall_s)
        s["max_inflight"] = srv.max_inflight_seen
        s["rate_req_s"] = frac * cap
        out["rates"][f"{frac:.2f}"] = s
    return out
