"""The allocation-free entry point, idw_interpolate_noalloc.

It serves callers that cannot allocate device memory (and so cannot create
a handle): a host application that owns the whole device-memory budget, or a
loop that cannot afford the device synchronisation cudaMalloc/cudaFree imply.
This test calls it through the C ABI twice in a row, on two different
problems, and checks each result against the FP64 oracle within the FP32
form's tolerance (and bit-exact at exact hits); it checks that a problem too
large for the fixed scratch is refused before any launch, with real buffers
of the declared size behind the call; and it checks that a bounded wait that
gave up is reported once by idw_noalloc_sync_status.  It runs last (file
order) and passes alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6


@pytest.fixture(scope="module")
def lib():
    from paper_1402_4986_gb300 import build
    build.build()
    from paper_1402_4986_gb300 import _lib
    return _lib


def _call(L, d, q, p, out, stream=None):
    return L.load().idw_interpolate_noalloc(d.data_ptr(), d.shape[0], q.data_ptr(), q.shape[0],
                                            p, out.data_ptr(), stream)


def test_noalloc_matches_oracle_on_two_calls_in_a_row(lib):
    stream = torch.cuda.current_stream()
    a = synthetic.uniform_problem(50000, 30000, seed=71)
    b = synthetic.config_exact_hits(seed=72, n=20001, m=12345, hits=40)
    for prob, p in ((a, 2.0), (b, 3.5)):
        d = torch.from_numpy(prob["data"]).cuda()
        q = torch.from_numpy(prob["queries"]).cuda()
        out = torch.full((q.shape[0],), float("nan"), device="cuda")
        st = _call(lib, d, q, p, out, ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.STATUS.get(st)
        st = lib.load().idw_noalloc_sync_status(ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.STATUS.get(st)
        Z64, hit64 = oracle.idw(prob["data"], prob["queries"], p)
        zmax = float(np.abs(prob["data"][:, 2]).max())
        err = float(np.max(np.abs(out.cpu().numpy().astype(np.float64) - Z64))) / zmax
        assert err <= TOL_F32C, err
        if len(prob["hit_q"]):
            hq = prob["hit_q"]
            assert np.array_equal(out.cpu().numpy()[hq], prob["data"][prob["hit_d"], 2])


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    # 4M data points need 96 MiB of staged tiles: refused before any launch.
    # The buffers really hold 4M points, so even a launch would stay in bounds.
    n = 1 << 22
    d = torch.zeros(n, 3, device="cuda")
    q = torch.zeros(4, 2, device="cuda")
    out = torch.empty(4, device="cuda")
    assert lib.STATUS.get(_call(lib, d, q, 2.0, out)) == "IDW_ERR_WORKSPACE"
    small = d[:4]
    assert lib.STATUS.get(_call(lib, small, q, -1.0, out)) == "IDW_ERR_INVALID_ARG"
    torch.cuda.synchronize()


def test_noalloc_reports_a_bounded_wait_timeout_once(lib):
    L = lib.load()
    assert L.idw_noalloc_selftest_bounded_wait(None) == 0
    assert lib.STATUS.get(L.idw_noalloc_sync_status(None)) == "IDW_ERR_DEVICE_TIMEOUT"
    assert L.idw_noalloc_sync_status(None) == 0  # cleared
    # The path still computes after the reported timeout.
    d = torch.tensor([[0.0, 0.0, 1.0], [1.0, 0.0, 3.0]], device="cuda")
    q = torch.tensor([[0.5, 0.0]], device="cuda")
    out = torch.empty(1, device="cuda")
    assert _call(lib, d, q, 2.0, out) == 0
    assert L.idw_noalloc_sync_status(None) == 0
    assert abs(float(out[0]) - 2.0) < 1e-6
