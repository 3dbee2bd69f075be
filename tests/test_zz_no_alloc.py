"""The allocation-free entry point, idw_interpolate_noalloc.

It serves callers that cannot allocate device memory (and so cannot create
a handle).  This test calls it through the C ABI twice in a row, on two
different problems, and checks each result against idw_interpolate's within
the FP32 form's tolerance; it also checks that a problem too large for its
fixed scratch is refused before any launch.  It runs last (file order) and
passes alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6


def test_noalloc_matches_handle_path_on_two_calls_in_a_row():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as idw
    from paper_1402_4986_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()

    a = synthetic.uniform_problem(50000, 30000, seed=71)
    b = synthetic.config_exact_hits(seed=72, n=20001, m=12345, hits=40)
    for prob, p in ((a, 2.0), (b, 3.5)):
        d = torch.from_numpy(prob["data"]).cuda()
        q = torch.from_numpy(prob["queries"]).cuda()
        ref = idw.interpolate(d, q, p)
        out = torch.full((q.shape[0],), float("nan"), device="cuda")
        st = lib.idw_interpolate_noalloc(d.data_ptr(), d.shape[0], q.data_ptr(), q.shape[0],
                                         p, out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, _lib.STATUS.get(st)
        torch.cuda.synchronize()
        zmax = float(np.abs(prob["data"][:, 2]).max())
        err = float((out.double() - ref.double()).abs().max()) / zmax
        assert err <= TOL_F32C, err
        if "hit_q" in prob:
            hq = torch.from_numpy(prob["hit_q"]).cuda()
            assert torch.equal(out[hq], ref[hq])


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_1402_4986_gb300 import _lib
    lib = _lib.load()
    d = torch.zeros(4, 3, device="cuda")
    q = torch.zeros(4, 2, device="cuda")
    out = torch.empty(4, device="cuda")
    # 4M data points need 96 MiB of staged tiles: refused before any launch.
    st = lib.idw_interpolate_noalloc(d.data_ptr(), 1 << 22, q.data_ptr(), 4, 2.0,
                                     out.data_ptr(), None)
    assert _lib.STATUS.get(st) == "IDW_ERR_WORKSPACE"
    st = lib.idw_interpolate_noalloc(d.data_ptr(), 4, q.data_ptr(), 4, -1.0, out.data_ptr(), None)
    assert _lib.STATUS.get(st) == "IDW_ERR_INVALID_ARG"
