"""The paper's naive and tiled kernels (measured baselines) in each of its
layouts and both precisions, against the FP64 oracle.

They sum plainly, so the FP32 bar is looser than the library's compensated
form: plain sequential summation of n terms has relative error up to
(n - 1) u; at n = 3001 that is <= 1.8e-4 worst case, and 5e-5 of max|z| is
used here.  FP64 keeps the 1e-13 bar.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    return m


@pytest.fixture(scope="module")
def problem():
    prob = synthetic.config_exact_hits(seed=80, n=3001, m=2049, hits=6)
    Z = {p: oracle.idw(prob["data"], prob["queries"], p)[0] for p in (2.0, 3.5)}
    return prob, Z


@pytest.mark.parametrize("kernel", ["naive", "tiled"])
@pytest.mark.parametrize("layout", ["soa", "aos", "aoas", "hybrid"])
@pytest.mark.parametrize("precision,tol", [("f32c", 5e-5), ("f64", 1e-13)])
@pytest.mark.parametrize("p", [2.0, 3.5])
def test_paper_kernel_matches_oracle(idw, problem, kernel, layout, precision, tol, p):
    prob, Zref = problem
    dt = torch.float32 if precision == "f32c" else torch.float64
    d = torch.from_numpy(prob["data"]).to(dt).cuda()
    q = torch.from_numpy(prob["queries"]).to(dt).cuda()
    Z = idw.paper_interpolate(d, q, p, kernel=kernel, layout=layout, precision=precision)
    idw.sync_status()
    Zc = Z.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(Zc - Zref[p])) / np.max(np.abs(prob["data"][:, 2]))
    assert err <= tol, (kernel, layout, precision, p, err)
    hq = prob["hit_q"]
    assert np.array_equal(Zc[hq], prob["data"][prob["hit_d"], 2].astype(np.float64))


def test_paper_kernel_argument_errors(idw):
    d = torch.zeros(10, 3, device="cuda")
    q = torch.zeros(4, 2, device="cuda")
    out = torch.empty(4, device="cuda")
    h = idw.get_handle()
    assert h.lib.idw_paper_interpolate(h.ptr, 7, 0, d.data_ptr(), 10, q.data_ptr(), 4, 2.0, 0,
                                       out.data_ptr(), None) == 1
    assert h.lib.idw_paper_interpolate(h.ptr, 0, 9, d.data_ptr(), 10, q.data_ptr(), 4, 2.0, 0,
                                       out.data_ptr(), None) == 1
