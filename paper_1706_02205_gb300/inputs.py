"""Seeded synthetic inputs shaped like the paper's workloads (Section 4.4).

This module only draws random numbers: it holds none of the method's
arithmetic (no distances, no kernel, no ordering), so both the CPU oracle's
tests and the CUDA path consume the very same arrays.

Every generator uses NumPy's PCG64 bit generator; the default seed of a
workload is ``SEED_BASE + 1000 * workload_id + replicate``.

Workloads
---------
* ``uniform(N, d)``: x ~ U[0,1]^d i.i.d., the paper's default point cloud
  (Section 4.4, Tables 1-5).
* ``jittered_grid(n_side)``: a regular n_side x n_side grid of cell centres in
  [0,1]^2 with i.i.d. uniform jitter of +-0.25 cell, listed in a seeded random
  order so that the input order carries no structure.
* ``swiss_roll(N, ambient)``: a 2-D swiss-roll surface embedded by a seeded
  orthonormal map into R^ambient, plus Gaussian noise sigma=1e-3 (stands in for
  the paper's high-dimensional point sets of Section 4.4, whose exact
  structures are shown only in a figure).
* ``batch_sets`` / ``serving_requests``: the mixes of many independent sets.
* ``rhs(N, nrhs)``: right-hand sides ~ N(0, I), column-major (N x nrhs).
* ``sample_pairs(N, m)``: index pairs i.i.d. uniform on I x I, the sample the
  paper's error estimator E draws (Section 4.4).
* ``grid_operator(n_side)``: a sparse symmetric positive-definite matrix on the
  nodes of an n_side x n_side grid in [0,1]^2 -- the 5-point graph Laplacian
  with seeded rough edge weights (log-uniform in [1/10, 10]) plus a
  zeroth-order term -- standing in for the discretised elliptic operators
  whose inverse is a kernel matrix (Section 6); nodes listed in a seeded
  random order, matrix given by CSR rows in that order.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1706_02205


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def seed_for(workload: int, replicate: int = 0) -> int:
    return SEED_BASE + 1000 * workload + replicate


def uniform(N: int, d: int, seed: int = seed_for(1)) -> np.ndarray:
    """N points i.i.d. uniform in [0,1]^d, float64, row-major (N, d)."""
    return rng(seed).random((N, d), dtype=np.float64)


def jittered_grid(n_side: int, jitter: float = 0.25, seed: int = seed_for(2)) -> np.ndarray:
    """n_side^2 cell-centred grid points in [0,1]^2, jitter +-``jitter`` cell.

    x = (c + 0.5 + u) / n_side with c in {0..n_side-1}^2 and u ~ U[-jitter,
    jitter]^2, then shuffled by a seeded permutation.
    """
    g = rng(seed)
    c = np.arange(n_side, dtype=np.float64)
    cx, cy = np.meshgrid(c, c, indexing="ij")
    base = np.stack([cx.ravel(), cy.ravel()], axis=1)
    u = g.uniform(-jitter, jitter, size=base.shape)
    x = (base + 0.5 + u) / float(n_side)
    p = g.permutation(x.shape[0])
    return np.ascontiguousarray(x[p])


def swiss_roll(N: int, ambient: int = 20, noise: float = 1e-3, seed: int = seed_for(5)) -> np.ndarray:
    """Swiss roll (intrinsic dimension 2) embedded in R^ambient.

    t ~ U[1.5 pi, 4.5 pi], h ~ U[0, 1]; y = (t cos t, 10 h, t sin t) / (4.5 pi);
    x = Q y + noise * xi with Q an ambient x 3 orthonormal matrix (QR of a seeded
    Gaussian matrix) and xi ~ N(0, I).
    """
    g = rng(seed)
    t = g.uniform(1.5 * math.pi, 4.5 * math.pi, size=N)
    h = g.uniform(0.0, 1.0, size=N)
    y = np.stack([t * np.cos(t), 10.0 * h, t * np.sin(t)], axis=1) / (4.5 * math.pi)
    q, _ = np.linalg.qr(g.standard_normal((ambient, 3)))
    x = y @ q.T + noise * g.standard_normal((N, ambient))
    return np.ascontiguousarray(x)


def rhs(N: int, nrhs: int = 1, seed: int = seed_for(1, 7)) -> np.ndarray:
    """Right-hand sides b ~ N(0, I), column-major: shape (nrhs, N), b[r] is RHS r."""
    return np.ascontiguousarray(rng(seed).standard_normal((nrhs, N)))


def sample_pairs(N: int, m: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """m index pairs i.i.d. uniform on {0..N-1}^2 with replacement (diagonal allowed)."""
    g = rng(seed)
    i = g.integers(0, N, size=m, dtype=np.int64)
    j = g.integers(0, N, size=m, dtype=np.int64)
    return i, j


def unit_vector(N: int, seed: int) -> np.ndarray:
    """A start vector ~ N(0, I) normalised to unit 2-norm (power iteration)."""
    v = rng(seed).standard_normal(N)
    return v / np.linalg.norm(v)


def batch_sets(n_sets: int = 256, n_min: int = 2000, n_max: int = 50000, n_d3: int = 64,
               ell_lo: float = 0.05, ell_hi: float = 0.3, seed: int = seed_for(4)):
    """Independent point sets of uneven size for one batched launch.

    N_s = floor(exp(U[ln n_min, ln n_max])); the last ``n_d3`` sets are 3-D, the
    rest 2-D; points U[0,1]^d; Matern length scale ell_s ~ U[ell_lo, ell_hi].
    Returns a list of dicts {"x": (N_s, d) float64, "ell": float}.
    """
    g = rng(seed)
    out = []
    for s in range(n_sets):
        n = int(math.floor(math.exp(g.uniform(math.log(n_min), math.log(n_max)))))
        d = 3 if s >= n_sets - n_d3 else 2
        ell = float(g.uniform(ell_lo, ell_hi))
        out.append({"x": g.random((n, d), dtype=np.float64), "ell": ell})
    return out


def serving_requests(n_req: int, rate_hz: float, n_min: int = 10_000, n_max: int = 1_000_000,
                     seed: int = seed_for(5, 1), repeat_frac: float = 0.5):
    """A Poisson stream of factor+solve requests of mixed size and dimension,
    with repeated solves against factors requested earlier.

    Inter-arrival times ~ Exp(rate).  Each request is, with probability
    repeat_frac (once some point set exists), a repeat solve ("solve") for a
    point set drawn uniformly from the earlier ones, else a new point set
    ("factor"): N ~ log-U[n_min, n_max]; half U[0,1]^d with d uniform in
    {2, 3}, half a swiss roll in R^20; rho uniform in {3, 4}.  Every request
    has nrhs uniform in {1..8}.  Points are not drawn here: each point set
    carries its own seed (its key) so that it can be regenerated alone.
    """
    g = rng(seed)
    t = 0.0
    reqs = []
    sets = []
    for r in range(n_req):
        t += float(g.exponential(1.0 / rate_hz))
        repeat = bool(sets) and g.random() < repeat_frac
        nrhs = int(g.integers(1, 9))
        if repeat:
            base = sets[int(g.integers(0, len(sets)))]
            reqs.append({"id": r, "type": "solve", "key": base["key"], "t_arrival": t, "N": base["N"],
                         "nrhs": nrhs, "seed": int(g.integers(0, 2**62))})
            continue
        n = int(math.floor(math.exp(g.uniform(math.log(n_min), math.log(n_max)))))
        kind = "swiss" if g.random() < 0.5 else "cube"
        d = 20 if kind == "swiss" else int(g.integers(2, 4))
        rho = float(g.choice([3.0, 4.0]))
        sd = int(g.integers(0, 2**62))
        req = {"id": r, "type": "factor", "key": sd, "t_arrival": t, "N": n, "kind": kind, "d": d, "rho": rho,
               "nrhs": nrhs, "seed": sd}
        reqs.append(req)
        sets.append(req)
    return reqs


def request_points(req) -> np.ndarray:
    if req["kind"] == "swiss":
        return swiss_roll(req["N"], ambient=req["d"], seed=req["seed"])
    return uniform(req["N"], req["d"], seed=req["seed"])


def grid_operator(n_side: int, shift: float = 1.0, contrast: float = 10.0, seed: int = seed_for(6)):
    """(x, rowptr, col, val): nodes x (N, 2), N = n_side^2, and the CSR rows
    (columns ascending, diagonal included) of A = sum over grid edges (u, v)
    of w_uv (e_u - e_v)(e_u - e_v)^T + shift * I, w_uv log-uniform in
    [1/contrast, contrast], scaled by n_side^2 (the mesh size h^-2)."""
    r = rng(seed)
    N = n_side * n_side
    h = 1.0 / n_side
    gi, gj = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    order = r.permutation(N)            # node of each list position
    pos = np.empty(N, np.int64)
    pos[order] = np.arange(N)
    x = np.stack([(gi.ravel() + 0.5) * h, (gj.ravel() + 0.5) * h], 1)[order]
    node = np.arange(N).reshape(n_side, n_side)
    eu = np.concatenate([node[:-1, :].ravel(), node[:, :-1].ravel()])
    ev = np.concatenate([node[1:, :].ravel(), node[:, 1:].ravel()])
    w = np.exp(r.uniform(-math.log(contrast), math.log(contrast), eu.shape[0])) * n_side * n_side
    u, v = pos[eu], pos[ev]
    rows = np.concatenate([u, v, u, v, np.arange(N)])
    cols = np.concatenate([v, u, u, v, np.arange(N)])
    vals = np.concatenate([-w, -w, w, w, np.full(N, shift)])
    key = rows * N + cols
    o = np.argsort(key, kind="stable")
    key, vals = key[o], vals[o]
    uk, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(vals, start)
    rr, cc = uk // N, uk % N
    rowptr = np.zeros(N + 1, np.int64)
    np.add.at(rowptr, rr + 1, 1)
    rowptr = np.cumsum(rowptr)
    return x, rowptr, cc.astype(np.int32), sums
