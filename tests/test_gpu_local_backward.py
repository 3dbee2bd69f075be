"""GPU parity of the radius form's gradients against the FP64 oracle.

``idw_local_backward`` holds each query's FP32 membership set fixed, as the
oracle does (``oracle.idw_local_grad``, itself pinned by central differences
and invariants).  Each gradient must match the oracle's to 1e-4 of its
largest magnitude, the bar of the global adjoint.
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _dev(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / scale) if scale > 0 else float(np.max(np.abs(a)))


def _compare(idw, data, q, p, radius, g, tol=TOL):
    gz, gxy, gq, gp = idw.local_backward(_dev(data), _dev(q), p, radius, _dev(g))
    torch.cuda.synchronize()
    G = oracle.idw_local_grad(data, q, p, radius, g)
    errs = {"z": _rel(gz.cpu().numpy(), G["grad_z"]),
            "xy": _rel(gxy.cpu().numpy(), G["grad_xy"]),
            "q": _rel(gq.cpu().numpy(), G["grad_q"]),
            "p": abs(float(gp.cpu()[0]) - G["grad_p"]) / max(abs(G["grad_p"]), 1e-300)}
    for k, e in errs.items():
        assert e <= tol, (k, errs)
    return G, (gz, gxy, gq, gp)


@pytest.mark.parametrize("p", [2.0, 3.5, 1.5])
def test_uniform_ragged(idw, p):
    """N = 5003, M = 3001, R for 40 members, with exact hits."""
    prob = synthetic.config_local(n=5003, m=3001, members=40.0, seed=111)
    data, q = prob["data"], prob["queries"].copy()
    q[::500] = data[:7 * 500:500, :2][: q[::500].shape[0]]  # exact hits
    g = np.random.default_rng(112).standard_normal(q.shape[0]).astype(np.float32)
    G, _ = _compare(idw, data, q, p, prob["radius"], g)
    assert np.isfinite(G["Z"]).all()


def test_clustered_with_empty_neighbourhoods(idw):
    prob = synthetic.config_local(n=20000, m=4000, members=16.0, clustered=True, seed=113)
    g = np.random.default_rng(114).standard_normal(4000).astype(np.float32)
    G, _ = _compare(idw, prob["data"], prob["queries"], 2.0, prob["radius"], g)
    assert np.isnan(G["Z"]).any()


def test_exact_hits_pass_the_gradient_to_z(idw):
    data = np.array([[0.1, 0.2, 1.5], [0.7, 0.4, -1.0], [0.3, 0.9, 2.0], [0.72, 0.41, 4.0],
                     [0.7, 0.4, 9.0]], np.float32)  # index 4 duplicates index 1
    q = np.array([[0.7, 0.4], [5.0, 5.0], [0.71, 0.405]], np.float32)
    g = np.array([3.0, 7.0, -2.0], np.float32)
    G, (gz, gxy, gq, gp) = _compare(idw, data, q, 2.0, 0.2, g)
    # The hit goes to the lowest coincident index only; the hit query and
    # the query without members have no coordinate gradient.
    assert G["grad_z"][1] - G["grad_z"][4] == pytest.approx(3.0)
    assert np.all(gq.cpu().numpy()[:2] == 0)


def test_fp64_path_for_tiny_distances(idw):
    """Coordinates near 1e-18: d^2 near 1e-36, below the FP32 path's 2^-100
    floor, so both kernels take their FP64 branch."""
    rng = np.random.default_rng(115)
    xy = (rng.random((400, 2)) * 1e-17).astype(np.float32)
    data = np.concatenate([xy, rng.standard_normal((400, 1)).astype(np.float32)], 1)
    q = (rng.random((150, 2)) * 1e-17).astype(np.float32)
    g = rng.standard_normal(150).astype(np.float32)
    _compare(idw, data, q, 2.5, 2e-18, g)


def test_large_power_and_non_finite_points(idw):
    prob = synthetic.config_local(n=3000, m=800, members=30.0, seed=116)
    data = prob["data"].copy()
    data[::13, 0] = np.nan
    data[5::17, 1] = np.inf
    g = np.random.default_rng(117).standard_normal(800).astype(np.float32)
    for p in (2.0, 12.0):
        G, (gz, gxy, _, _) = _compare(idw, data, prob["queries"], p, prob["radius"], g)
        bad = ~np.isfinite(data[:, :2]).all(1)
        assert np.all(gz.cpu().numpy()[bad] == 0) and np.all(gxy.cpu().numpy()[bad] == 0)


def test_partial_outputs_and_errors(idw):
    prob = synthetic.config_local(n=2000, m=500, members=20.0, seed=118)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    g = _dev(np.ones(500))
    full = idw.local_backward(d, q, 2.0, prob["radius"], g)
    only_q = idw.local_backward(d, q, 2.0, prob["radius"], g, need_z=False, need_data_xy=False,
                                need_p=False)
    only_z = idw.local_backward(d, q, 2.0, prob["radius"], g, need_data_xy=False,
                                need_query_xy=False, need_p=False)
    assert only_q[0] is None and only_q[1] is None and only_q[3] is None
    assert torch.allclose(only_q[2], full[2], rtol=0, atol=1e-5 * float(full[2].abs().max()))
    assert torch.allclose(only_z[0], full[0], rtol=0, atol=1e-6 * float(full[0].abs().max()))
    with pytest.raises(idw.IDWError):
        idw.local_backward(d, q, 2.0, 0.0, g)
    with pytest.raises(idw.IDWError):
        idw.local_backward(d, q, -1.0, 0.1, g)
    gz, gxy, gq, gp = idw.local_backward(d, q[:0], 2.0, 0.1, g[:0])
    assert float(gz.abs().max()) == 0 and float(gxy.abs().max()) == 0 and float(gp[0]) == 0


def test_autograd_function(idw):
    prob = synthetic.config_local(n=4000, m=1500, members=25.0, seed=119)
    data, q, R = prob["data"], prob["queries"], prob["radius"]
    d = _dev(data).requires_grad_(True)
    qq = _dev(q).requires_grad_(True)
    p = torch.tensor(2.5, device="cuda", requires_grad=True)
    Z = idw.idw_local(d, qq, p, R)
    w = torch.from_numpy(np.random.default_rng(120).standard_normal(1500).astype(np.float32)).cuda()
    ok = torch.isfinite(Z)
    (Z[ok] * w[ok]).sum().backward()
    g = np.where(ok.cpu().numpy(), w.cpu().numpy(), 0).astype(np.float32)
    G = oracle.idw_local_grad(data, q, 2.5, R, g)
    gd = d.grad.cpu().numpy().astype(np.float64)
    assert _rel(gd[:, 2], G["grad_z"]) <= TOL
    assert _rel(gd[:, :2], G["grad_xy"]) <= TOL
    assert _rel(qq.grad.cpu().numpy(), G["grad_q"]) <= TOL
    assert abs(float(p.grad) - G["grad_p"]) <= TOL * abs(G["grad_p"])


def test_full_size_sampled_and_sum_rules(idw):
    """N = M = 2^20, R for 32 members: dL/dq on 128 sampled queries against
    the oracle; over all queries, dL/dz sums to sum_j g_j over the queries
    with a value, and the coordinate gradients cancel (translation)."""
    prob = synthetic.config_local()
    data, q, R = prob["data"], prob["queries"], prob["radius"]
    m = q.shape[0]
    g = np.random.default_rng(121).standard_normal(m).astype(np.float32)
    d, qd = _dev(data), _dev(q)
    gz, gxy, gq, gp = idw.local_backward(d, qd, 2.0, R, _dev(g))
    Z = idw.interpolate_local(d, qd, 2.0, R)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(122).choice(m, 128, replace=False))
    G = oracle.idw_local_grad(data, q[idx], 2.0, R, g[idx])
    assert _rel(gq.cpu().numpy()[idx], G["grad_q"]) <= TOL
    fin = np.isfinite(Z.cpu().numpy())
    want = float(np.sum(g[fin].astype(np.float64)))
    got = float(gz.double().sum())
    assert abs(got - want) <= 1e-4 * float(np.sum(np.abs(g))), (got, want)
    tot = gxy.double().sum(0) + gq.double().sum(0)
    assert float(tot.abs().max()) <= 1e-4 * float(gq.double().abs().sum(0).max())
