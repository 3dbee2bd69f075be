"""Multi-process host logic of the query sharding (world size 2, gloo, CPU).

Two ranks each interpolate their slice of the queries (with the FP64
oracle standing in for the GPU call, which this CPU test cannot make),
gather the results, and must reproduce the unsharded result exactly; the
max-over-ranks reduction used for timing is checked too.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import synthetic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_fn(data, queries, p):
    import oracle
    Z, _ = oracle.idw(data.numpy(), queries.numpy(), p)
    return torch.from_numpy(Z)


def _worker(rank, world, port, result_file):
    import torch.distributed as dist
    from paper_1402_4986_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = synthetic.uniform_problem(700, 1001, seed=8, exact_hits=5)
    data = torch.from_numpy(prob["data"])
    q = torch.from_numpy(prob["queries"])
    Z = shard.interpolate_sharded(data, q, 2.0, interpolate_fn=_oracle_fn)
    t = shard.max_over_ranks(float(rank + 1))
    if rank == 0:
        np.save(result_file, np.concatenate([Z.numpy(), [t]]))
    dist.barrier()
    dist.destroy_process_group()


def test_query_range_partitions():
    from paper_1402_4986_gb300.shard import query_range
    for m in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            parts = [query_range(m, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == m
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_sharded_equals_unsharded(tmp_path):
    import oracle
    out = str(tmp_path / "z.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    prob = synthetic.uniform_problem(700, 1001, seed=8, exact_hits=5)
    Z, _ = oracle.idw(prob["data"], prob["queries"], 2.0)
    assert np.array_equal(got[:-1], Z)
    assert got[-1] == 2.0
