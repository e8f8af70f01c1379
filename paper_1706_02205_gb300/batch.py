"""Many independent point sets factored in one persistent launch.

Each set is ordered and its pattern built on its own CUDA stream (host
threads, so the per-set steps overlap on the GPU); the patterns are then
concatenated block-diagonally, scheduled once, and one factor plan covers
all sets, with every column carrying its set's Matern parameters.  Because the
concatenated pattern is block-diagonal, its ICHOL(0) is exactly the per-set
factors.  The plan's launch allocates nothing and never waits on the host, so
it can be recorded in a CUDA graph and replayed.
"""
from __future__ import annotations

import concurrent.futures as cf

import torch

from . import kchol as kc


def prepare_sets(xs, rho, n_streams=8, rule=kc.RULE_MAX, stream=None):
    """Order and build the pattern of every set (list of (N_s, d_s) float64 CUDA
    tensors) on `n_streams` streams, or one after another on `stream` (which
    is then the only stream synchronised: other work on the device goes on).
    Returns a list of dicts."""
    if stream is not None:
        out = []
        with torch.cuda.stream(stream):
            for x in xs:
                perm, l, xo = kc.order_points(x, stream=stream)
                rowptr, col = kc.pattern_rows(xo, l, rho, rule, stream=stream)
                out.append({"perm": perm, "l": l, "x_ord": xo, "rowptr": rowptr, "col": col})
        stream.synchronize()
        return out
    streams = [torch.cuda.Stream() for _ in range(max(1, n_streams))]

    def one(k):
        st = streams[k % len(streams)]
        with torch.cuda.stream(st):
            perm, l, xo = kc.order_points(xs[k], stream=st)
            rowptr, col = kc.pattern_rows(xo, l, rho, rule, stream=st)
        st.synchronize()
        return {"perm": perm, "l": l, "x_ord": xo, "rowptr": rowptr, "col": col}

    # one worker per stream: sets on the same stream run in order
    with cf.ThreadPoolExecutor(max_workers=len(streams)) as ex:
        out = list(ex.map(one, range(len(xs))))
    torch.cuda.synchronize()
    return out


class BatchFactor:
    """Block-diagonal batch of point sets with one factor plan."""

    def __init__(self, xs, kerns, rho, prec=kc.FP32_FORM, opts=None, n_streams=8, prepared=None, stream=None):
        self.kerns = list(kerns)
        if len({(k.sigma2, k.nugget) for k in self.kerns}) > 1:
            raise ValueError("the sets of a batch share sigma2 and nugget (nu and ell may differ)")
        self.prec = prec
        self.sets = prepared if prepared is not None else prepare_sets(xs, rho, n_streams, stream=stream)
        self.Ns = [s["perm"].numel() for s in self.sets]
        self.offsets = [0]
        for n in self.Ns:
            self.offsets.append(self.offsets[-1] + n)
        rowptr, col, self.col_set = kc.pattern_concat([s["rowptr"] for s in self.sets],
                                                      [s["col"] for s in self.sets])
        self.x_ord = kc.points_concat([s["x_ord"] for s in self.sets])
        self.perm = kc.index_concat([s["perm"] for s in self.sets])
        self.pat = kc.schedule(rowptr, col, self.x_ord)
        self.nnz_offsets = [int(v) for v in rowptr[self.offsets].cpu()]
        self.plan = kc.FactorPlan(self.pat, self.x_ord, self.kerns, self.col_set if len(self.kerns) > 1 else None,
                                  prec, opts)
        dt = torch.float64 if prec == kc.FP64 else torch.float32
        self.val = torch.empty(self.pat.nnz, dtype=dt, device=self.x_ord.device)
        self.diag = torch.empty(self.pat.N, dtype=torch.float64, device=self.x_ord.device)
        self.graph = None

    def tune(self):
        return self.plan.tune(self.val, self.diag)

    def factor(self, stream=None):
        """One launch; returns the number of dropped pivots."""
        self.plan.launch(self.val, self.diag, stream=stream)
        return self.plan.finish(stream=stream)

    def capture(self):
        """Record the plan's launch in a CUDA graph (replay with replay())."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.plan.launch(self.val, self.diag, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def set_values(self, s):
        """Factor values of set s (its CSR rows, positions local to the set)."""
        return self.val[self.nnz_offsets[s]:self.nnz_offsets[s + 1]]

    def solve(self, b, stream=None):
        """Solve every set at once: b is (nrhs, sum N) in the concatenated
        original order.  A dropped pivot is replaced by sqrt(sigma2 + nugget),
        which the sets share (they may differ in nu and ell)."""
        return kc.solve(self.pat, self.prec, self.val, self.diag, self.kerns[0], self.perm, b, stream=stream)
