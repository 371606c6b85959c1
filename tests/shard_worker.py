"""Rank body of the two-process gloo test of the batch sharding (CPU only)."""
import os


def run(rank, world, port, out_dir):
    import json
    import torch
    import torch.distributed as dist
    from paper_1207_3392_gb300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    specs = shard.weak_scaling_specs(world, per_rank=512)
    idx = shard.lpt_shards([shard.spec_cost(s) for s in specs], world)[rank]
    mine = shard.rank_specs(specs, rank, world)
    assert [specs[i] for i in idx] == mine
    keys = idx
    cost = sum(shard.spec_cost(s) for s in mine)
    gathered = [None] * world
    dist.all_gather_object(gathered, {"keys": keys, "cost": cost})
    # the max-over-ranks step time the bench reports
    t = torch.tensor([1.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"gathered": gathered, "max_time": float(t.item()), "total": len(specs)}, f)
    dist.destroy_process_group()
