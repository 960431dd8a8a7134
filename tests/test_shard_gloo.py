"""Multi-GPU host logic on CPU: LPT sharding and the gather of results over a
world-size-2 gloo process group (no GPU, no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2003_02547_gb300 import shard, workloads as W


def test_lpt_shard_properties():
    rng = np.random.default_rng(0)
    costs = rng.uniform(1, 100, 257).tolist()
    for world in (1, 2, 3, 8):
        shards = shard.lpt_shard(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))          # every QP exactly once
        loads = [sum(costs[i] for i in s) for s in shards]
        # LPT bound: makespan <= 4/3 of the optimum, optimum >= mean and >= max cost
        assert max(loads) <= 4.0 / 3.0 * max(sum(costs) / world, max(costs)) + 1e-9
        assert shards == shard.lpt_shard(costs, world)  # deterministic


def test_qp_cost_orders_sizes():
    small = W.small_random_qp(0)
    big = W.ragged_random_qp(0)
    assert shard.qp_cost(big) > shard.qp_cost(small) > 0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    from oracle import ocp_ipm as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    qps = [W.small_random_qp(i) for i in range(9)] + [W.small_random_qp(i, N=5 + i) for i in range(3)]
    costs = [shard.qp_cost(q) for q in qps]
    mine = shard.lpt_shard(costs, world)[rank]
    # each rank solves its shard (the CPU oracle stands in for the GPU solve)
    local = {i: (rank, O.solve(qps[i]).y) for i in mine}
    res = shard.gather_results(local, rank, world, dist)
    if rank == 0:
        np.savez(out_path, keys=np.array(sorted(res)), ranks=np.array([res[k][0] for k in sorted(res)]),
                 **{f"y{k}": res[k][1] for k in res})
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_solve_gathers_the_unsharded_solutions(tmp_path):
    from oracle import ocp_ipm as O
    out = str(tmp_path / "gathered.npz")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    assert got["keys"].tolist() == list(range(12))
    assert set(got["ranks"].tolist()) == {0, 1}
    qps = [W.small_random_qp(i) for i in range(9)] + [W.small_random_qp(i, N=5 + i) for i in range(3)]
    for k, q in enumerate(qps):
        # the same solve on one process: the gathered solution is identical
        assert np.array_equal(got[f"y{k}"], O.solve(q).y), k
