"""GPU adjoint of Eq. 1 against the FP64 oracle's analytic gradient.

The oracle's gradient is pinned to central finite differences on the CPU
(test_oracle_pins); here the CUDA adjoint (FP32 pair arithmetic,
compensated sums, FP64 combine) must match it to 1e-4 of each gradient's
largest magnitude, and a direct FP64 central difference of the oracle's
forward pass at N = M = 512 (eps = 1e-6) is checked too.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    return m


def _gpu_grads(idw, data, q, p, g, **need):
    d = torch.from_numpy(data).cuda()
    qq = torch.from_numpy(q).cuda()
    Z, s0, hit = idw.interpolate_saved(d, qq, p)
    gz, gxy, gq, gp = idw.backward(d, qq, p, Z, s0, hit, torch.from_numpy(g).cuda(), **need)
    idw.sync_status()
    cpu = lambda t: None if t is None else t.cpu().numpy().astype(np.float64)
    return cpu(gz), cpu(gxy), cpu(gq), (None if gp is None else float(gp.cpu()[0]))


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _compare(G, gz, gxy, gq, gp):
    errs = {"z": _rel(gz, G["grad_z"]), "xy": _rel(gxy, G["grad_xy"]),
            "q": _rel(gq, G["grad_q"]), "p": abs(gp - G["grad_p"]) / max(abs(G["grad_p"]), 1e-12)}
    for k, e in errs.items():
        assert e <= TOL, (k, errs)
    return errs


@pytest.mark.parametrize("p", [2.0, 2.5, 1.5])
def test_adjoint_matches_oracle_gradient_512(idw, p):
    prob = synthetic.config_adjoint(n=512, m=512, p=p)
    data, q, g = prob["data"], prob["queries"], prob["grad_out"]
    G = oracle.idw_grad(data, q, p, g)
    _compare(G, *_gpu_grads(idw, data, q, p, g))


def test_adjoint_matches_fp64_central_differences(idw):
    """Direct FD of the FP64 forward (eps = 1e-6) at sampled coordinates."""
    rng = np.random.default_rng(41)
    n = m = 512
    data = np.empty((n, 3), np.float32)
    data[:, :2] = synthetic.separated_xy(rng, n, 1e-3)
    data[:, 2] = rng.standard_normal(n).astype(np.float32)
    q = synthetic.separated_xy(rng, m, 1e-3)
    g = rng.standard_normal(m).astype(np.float32)
    p = 2.5
    gz, gxy, gq, gp = _gpu_grads(idw, data, q, p, g)
    d64, q64, g64 = data.astype(np.float64), q.astype(np.float64), g.astype(np.float64)
    eps = 1e-6

    def loss(dd, qq, pp):
        return float(np.dot(g64, oracle.idw(dd, qq, pp)[0]))

    for i in rng.choice(n, 6, replace=False):
        for c, ref in ((2, gz), (0, gxy[:, 0]), (1, gxy[:, 1])):
            a = d64.copy(); a[i, c] += eps
            b = d64.copy(); b[i, c] -= eps
            fd = (loss(a, q64, p) - loss(b, q64, p)) / (2 * eps)
            assert abs(fd - ref[i]) <= TOL * np.max(np.abs(ref)), (i, c, fd, ref[i])
    for j in rng.choice(m, 6, replace=False):
        for c in (0, 1):
            a = q64.copy(); a[j, c] += eps
            b = q64.copy(); b[j, c] -= eps
            fd = (loss(d64, a, p) - loss(d64, b, p)) / (2 * eps)
            assert abs(fd - gq[j, c]) <= TOL * np.max(np.abs(gq)), (j, c, fd, gq[j, c])
    fd = (loss(d64, q64, p + eps) - loss(d64, q64, p - eps)) / (2 * eps)
    assert abs(fd - gp) <= TOL * max(1.0, abs(fd))


@pytest.mark.parametrize("n,m,p", [(3000, 5000, 2.0), (7001, 2049, 2.5), (1, 300, 2.5),
                                   (257, 1, 2.0)])
def test_adjoint_ragged_sizes(idw, n, m, p):
    prob = synthetic.uniform_problem(n, m, seed=n + 3 * m)
    g = np.random.default_rng(n).standard_normal(m).astype(np.float32)
    G = oracle.idw_grad(prob["data"], prob["queries"], p, g)
    gz, gxy, gq, gp = _gpu_grads(idw, prob["data"], prob["queries"], p, g)
    assert _rel(gz, G["grad_z"]) <= TOL
    if n > 1:  # with one data point Z is constant: every other gradient is 0
        assert _rel(gxy, G["grad_xy"]) <= TOL
        assert _rel(gq, G["grad_q"]) <= TOL
        assert abs(gp - G["grad_p"]) <= TOL * abs(G["grad_p"])


def test_adjoint_with_exact_hits_and_fp64_queries(idw):
    prob = synthetic.config_exact_hits(seed=44, n=2000, m=1500, hits=20)
    data, q = prob["data"], prob["queries"]
    # One query whose squared distance to a data point is below FP32's range.
    data[9, :2] = (1e-30, 0.25)
    q[3] = (4e-30, 0.25)
    g = np.random.default_rng(2).standard_normal(q.shape[0]).astype(np.float32)
    for p in (2.0, 2.5):
        G = oracle.idw_grad(data, q, p, g)
        _compare(G, *_gpu_grads(idw, data, q, p, g))


def test_adjoint_partial_outputs_and_empty_queries(idw):
    prob = synthetic.uniform_problem(800, 600, seed=45)
    g = np.random.default_rng(3).standard_normal(600).astype(np.float32)
    G = oracle.idw_grad(prob["data"], prob["queries"], 2.0, g)
    gz, gxy, gq, gp = _gpu_grads(idw, prob["data"], prob["queries"], 2.0, g,
                                 need_data_xy=False, need_query_xy=False, need_p=False)
    assert gxy is None and gq is None and gp is None
    assert _rel(gz, G["grad_z"]) <= TOL
    d = torch.from_numpy(prob["data"]).cuda()
    empty = torch.empty(0, 2, device="cuda")
    gz, gxy, gq, gp = idw.backward(d, empty, 2.0, torch.empty(0, device="cuda"),
                                   torch.empty(0, dtype=torch.float64, device="cuda"),
                                   torch.empty(0, dtype=torch.int32, device="cuda"),
                                   torch.empty(0, device="cuda"))
    assert float(gz.abs().max()) == 0.0 and float(gxy.abs().max()) == 0.0
    assert float(gp[0]) == 0.0


def test_autograd_function(idw):
    prob = synthetic.config_adjoint(n=700, m=900, p=2.5)
    data = torch.from_numpy(prob["data"]).cuda().requires_grad_(True)
    q = torch.from_numpy(prob["queries"]).cuda().requires_grad_(True)
    p = torch.tensor(2.5, device="cuda", requires_grad=True)
    g = torch.from_numpy(prob["grad_out"]).cuda()
    Z = idw.idw(data, q, p)
    (Z * g).sum().backward()
    G = oracle.idw_grad(prob["data"], prob["queries"], 2.5, prob["grad_out"])
    gd = data.grad.cpu().numpy().astype(np.float64)
    assert _rel(gd[:, 2], G["grad_z"]) <= TOL
    assert _rel(gd[:, :2], G["grad_xy"]) <= TOL
    assert _rel(q.grad.cpu().numpy().astype(np.float64), G["grad_q"]) <= TOL
    assert abs(float(p.grad) - G["grad_p"]) <= TOL * abs(G["grad_p"])
