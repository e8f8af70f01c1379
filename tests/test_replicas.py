"""The host-side logic of several ranks (replicas, split of independent
units, max-over-ranks timing, host gather) with two gloo ranks on the CPU."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")

from paper_1706_02205_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    r, w = replicas.init("gloo")
    costs = [5.0, 1.0, 7.0, 3.0, 3.0, 2.0, 9.0, 4.0]
    parts = replicas.partition(costs, w)
    res = {
        "rank_world": [r, w],
        "max": replicas.max_over_ranks([1.5 + r, 10.0 - r]),
        "sum": replicas.sum_over_ranks([r + 1.0]),
        "parts": parts,
        "gather": replicas.gather({"rank": r, "units": len(parts[r])}),
        "throughput": replicas.throughput([100.0, 300.0], [2.0, 4.0]),
    }
    replicas.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    for k, r in enumerate(res):
        assert r["rank_world"] == [k, 2]
        assert r["max"] == [2.5, 10.0]
        assert r["sum"] == [3.0]
        assert r["gather"] == [{"rank": 0, "units": len(res[0]["parts"][0])},
                               {"rank": 1, "units": len(res[0]["parts"][1])}]
        assert r["throughput"] == 100.0
    assert res[0]["parts"] == res[1]["parts"]  # the same split without communicating


def test_partition_is_a_balanced_split():
    costs = [5.0, 1.0, 7.0, 3.0, 3.0, 2.0, 9.0, 4.0, 0.5]
    for world in (1, 2, 3, 4):
        parts = replicas.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
        assert parts == replicas.partition(costs, world)


def test_single_process_fallbacks():
    assert replicas.max_over_ranks([3.0]) == [3.0]
    assert replicas.gather(7) == [7]
    replicas.barrier()
