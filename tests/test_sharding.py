"""Host-side multi-rank layout (no GPU): cost-balanced assignment of independent domains to
ranks, max-over-ranks and the diagnostics gather, run as two gloo ranks on the CPU."""
import json
import os
import socket

import pytest

from paper_2304_03306_gb300 import sharding as S


def sweep_costs():
    # the 48-domain sweep: 24 circles (12 radii x forward/backward) and 24 dumbbells on
    # 128^2..512^2 grids (costs in grid points)
    import ttsh_inputs as ti
    return [d["n"] ** 2 for d in ti.sweep_domains()]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_is_a_balanced_partition(world):
    costs = sweep_costs()
    parts = [S.shard(costs, r, world) for r in range(world)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert parts == [S.shard(costs, r, world) for r in range(world)]   # deterministic


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        S.shard([1, 2], 2, 2)


def test_single_process_fallbacks():
    assert S.max_over_ranks(2.5) == 2.5
    assert S.gather([1, 2]) == [1, 2]
    S.barrier()


def _worker(rank, world, port, out_dir, costs):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = S.shard(costs, rank, world)
    owners = S.gather([(i, rank) for i in mine])
    slowest = S.max_over_ranks(1.5 + rank)
    S.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"mine": mine, "owners": owners, "slowest": slowest}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    costs = sweep_costs()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_worker, args=(2, port, str(tmp_path), costs), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert res[0]["owners"] == res[1]["owners"]                      # same gather on both ranks
    owners = dict(tuple(x) for x in res[0]["owners"])
    assert sorted(owners) == list(range(len(costs)))
    for r in range(2):
        assert sorted(i for i, o in owners.items() if o == r) == res[r]["mine"]
        assert res[r]["slowest"] == 2.5
