"""Host-side pieces of bench.py on the CPU: the algorithmic bytes of the factor
(the roofline numerator) against the oracle's exact work counters, and the
DRAM traffic it reports from the ncu capture only while the factor's sources
are the ones the counters were taken on."""
import os
import sys

import numpy as np

import oracle
from paper_1706_02205_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_bytes_op_equals_the_oracle_work_counters():
    x = inputs.uniform(1200, 2, seed=131)
    perm, l, rp, col = oracle.sortsparse(x, 3.0)
    c = oracle.work_counters(rp, col)
    for s in (4, 8):
        assert bench.bytes_op(rp, len(rp) - 1, 2, s) == oracle.bytes_op(rp, c, len(rp) - 1, 2, s)
    # the prefix term is the sum over the entries (j, i) of |R_j cap [0, i)|
    r = np.diff(rp) - 1
    assert c["P"] == int((r * (r - 1) // 2).sum()) and c["Rsum"] == int(r.sum())


def test_traffic_is_reported_for_the_captured_sources_only(tmp_path, monkeypatch):
    bop = 141_822_862_952
    t = bench.factor_traffic(bop)
    assert t is not None and abs(t / bop - bench.TRAFFIC_CAPTURE["dram_per_algorithmic_byte"]) < 1e-12
    # a changed source: no traffic
    cap = dict(bench.TRAFFIC_CAPTURE, sha256="0" * 64)
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", cap)
    assert bench.factor_traffic(bop) is None
