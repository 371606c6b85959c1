"""Sharding of the batched problem set across ranks: LPT balance on the host,
and a two-rank gloo run (CPU) in which every rank picks its subset with no
data exchange, the subsets partition the global set and the step time is the
maximum over ranks."""
import json
import multiprocessing as mp
import socket

import pytest

from paper_1207_3392_gb300 import problems as P
from paper_1207_3392_gb300 import shard


def test_lpt_partitions_and_balances_the_batched_set():
    specs = P.batched_riemann()
    costs = [shard.spec_cost(s) for s in specs]
    for world in (1, 2, 4, 8):
        parts = shard.lpt_shards(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(specs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= (sum(loads) / world) * 1.001
        assert max(loads) - min(loads) <= max(costs)


def test_lpt_small_cases():
    assert shard.lpt_shards([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
    assert shard.lpt_shards([], 3) == [[], [], []]
    assert shard.lpt_shards([7], 2) == [[0], []]
    with pytest.raises(ValueError):
        shard.lpt_shards([1], 0)


def test_weak_scaling_set_grows_with_the_rank_count():
    one = shard.weak_scaling_specs(1, per_rank=64)
    two = shard.weak_scaling_specs(2, per_rank=64)
    assert len(two) == 2 * len(one)
    assert [(s.n, s.states) for s in two[:64]] == [(s.n, s.states) for s in one]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo_sharding(tmp_path):
    import shard_worker
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=shard_worker.run, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    g = res[0]["gathered"]
    assert res[1]["gathered"] == g
    keys = [k for part in g for k in part["keys"]]
    assert len(keys) == res[0]["total"] == 1024
    assert len(set(keys)) == len(keys)  # disjoint
    costs = [part["cost"] for part in g]
    assert max(costs) <= 1.01 * sum(costs) / 2
    assert res[0]["max_time"] == res[1]["max_time"] == 2.0
