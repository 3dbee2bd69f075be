"""Query sharding with the CUDA forward pass (paper's future work on
multi-GPU IDW, Sec. 4.2 closing paragraph; here one process per GPU, data
replicated, each rank a contiguous slice of the queries).

This run has one GPU, so the sharded path is exercised two ways on cuda:0:
  * world size 1 over NCCL (the launch the benchmark uses on N GPUs, with
    the all-gather on the device);
  * two gloo ranks sharing cuda:0, each running the CUDA interpolation on its
    slice (independent kernels: no rank waits on another on the GPU) and
    gathering on the host.
Each must match the FP64 oracle within the FP32 bar and the unsharded CUDA
result to the same bar.  (World size 1 reproduces the unsharded call bit for
bit; a rank's smaller query slice changes the launch plan, and with it where
each query's sum is split into pieces, so shards agree to rounding only.)
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    return synthetic.uniform_problem(20000, 9001, seed=81, exact_hits=7)


def _cuda_to_host(data, queries, p):
    import paper_1402_4986_gb300 as idw
    return idw.interpolate(data, queries, p).cpu()


def _worker(rank, world, port, backend, result_file):
    import torch.distributed as dist
    from paper_1402_4986_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    kw = {"device_id": torch.device("cuda", 0)} if backend == "nccl" else {}
    dist.init_process_group(backend, rank=rank, world_size=world, **kw)
    prob = _problem()
    data = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    fn = None if backend == "nccl" else _cuda_to_host  # None: the CUDA forward, gathered on GPU
    Z = shard.interpolate_sharded(data, q, 2.0, interpolate_fn=fn)
    if rank == 0:
        np.save(result_file, Z.cpu().numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def reference():
    from paper_1402_4986_gb300 import build
    build.build()
    import oracle
    import paper_1402_4986_gb300 as idw
    prob = _problem()
    Z = idw.interpolate(torch.from_numpy(prob["data"]).cuda(),
                        torch.from_numpy(prob["queries"]).cuda(), 2.0).cpu().numpy()
    Z64, _ = oracle.idw(prob["data"], prob["queries"], 2.0)
    return prob, Z, Z64


@pytest.mark.parametrize("backend,world", [("nccl", 1), ("gloo", 2)])
def test_sharded_cuda_path_equals_unsharded(tmp_path, reference, backend, world):
    prob, Z, Z64 = reference
    out = str(tmp_path / "z.npy")
    mp.start_processes(_worker, args=(world, _free_port(), backend, out), nprocs=world,
                       join=True, start_method="spawn")
    got = np.load(out)
    assert got.shape == Z.shape
    zmax = np.max(np.abs(prob["data"][:, 2]))
    if world == 1:
        assert np.array_equal(got, Z)
    assert np.max(np.abs(got.astype(np.float64) - Z)) / zmax <= TOL_F32C
    err = np.max(np.abs(got.astype(np.float64) - Z64)) / zmax
    assert err <= TOL_F32C
    hq = prob["hit_q"]
    assert np.array_equal(got[hq], prob["data"][prob["hit_d"], 2])
