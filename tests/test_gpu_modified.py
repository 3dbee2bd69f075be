"""GPU parity of modified Shepard interpolation against the FP64 oracle.

``idw_interpolate_modified`` weights the radius form's members by
((R - d)/(R d))^p (Franke and Nielson's local weights).  Member counts must
equal the oracle's (the FP32 test is the radius form's), values within 2e-6
of max |z|, NaN where no member has a positive weight, exact z at hits.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _compare(idw, data, q, p, radius, tol=TOL):
    Z, cnt = idw.interpolate_modified(_dev(data), _dev(q), p, radius, counts=True)
    torch.cuda.synchronize()
    Z, cnt = Z.cpu().numpy(), cnt.cpu().numpy()
    Z64, hit64, cnt64 = oracle.idw_modified(data, q, p, radius)
    assert np.array_equal(cnt, cnt64), np.nonzero(cnt != cnt64)[0][:10]
    assert np.array_equal(np.isnan(Z), np.isnan(Z64))
    h = hit64 >= 0
    assert np.array_equal(Z[h], data[hit64[h], 2])
    ok = ~np.isnan(Z64)
    if ok.any():
        err = np.max(np.abs(Z[ok].astype(np.float64) - Z64[ok])) / np.max(np.abs(data[:, 2]))
        assert err <= tol, err
    return Z, cnt


@pytest.mark.parametrize("p", [1.0, 2.0, 3.5])
@pytest.mark.parametrize("members", [8.0, 40.0])
def test_uniform_ragged_with_hits(idw, p, members):
    prob = synthetic.config_local(n=5003, m=3001, members=members, seed=161)
    data, q = prob["data"], prob["queries"].copy()
    q[::400] = data[:8 * 400:400, :2][: q[::400].shape[0]]
    _compare(idw, data, q, p, prob["radius"])


def test_clustered(idw):
    prob = synthetic.config_local(n=20000, m=4000, members=16.0, clustered=True, seed=162)
    _, cnt = _compare(idw, prob["data"], prob["queries"], 2.0, prob["radius"])
    assert (cnt == 0).any() and cnt.max() > 100


def test_infinite_radius_is_the_global_form(idw):
    prob = synthetic.uniform_problem(3000, 800, seed=163, exact_hits=4)
    for p in (2.0, 3.5):
        Z = idw.interpolate_modified(_dev(prob["data"]), _dev(prob["queries"]), p,
                                     float("inf")).cpu().numpy()
        Zg, _ = oracle.idw(prob["data"], prob["queries"], p)
        assert np.max(np.abs(Z - Zg)) / np.max(np.abs(prob["data"][:, 2])) <= TOL


def test_range_edges_take_the_fp64_pass(idw):
    """3e-19 coordinates (weights near 1e38 overflow the FP32 sums) and 1e17
    coordinates (weights below 2^-100 per member): the FP64 pass computes the
    scaled modified weights."""
    rng = np.random.default_rng(164)
    for scale, R in ((3e-19, 1e-19), (1e17, 3e16)):
        xy = (rng.random((400, 2)) * scale).astype(np.float32)
        data = np.concatenate([xy, rng.standard_normal((400, 1)).astype(np.float32)], 1)
        q = (rng.random((120, 2)) * scale).astype(np.float32)
        _compare(idw, data, q, 2.0, R)


def test_matches_the_radius_form_membership_and_errors(idw):
    prob = synthetic.config_local(n=4000, m=1000, members=20.0, seed=165)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    _, cm = idw.interpolate_modified(d, q, 2.0, prob["radius"], counts=True)
    _, cl = idw.interpolate_local(d, q, 2.0, prob["radius"], counts=True)
    assert torch.equal(cm, cl)
    for bad in ((2.0, 0.0), (0.0, 0.1), (2.0, float("nan"))):
        with pytest.raises(idw.IDWError):
            idw.interpolate_modified(d, q, bad[0], bad[1])


def test_full_size_sampled(idw):
    prob = synthetic.config_local()
    data, q = prob["data"], prob["queries"]
    Z = idw.interpolate_modified(_dev(data), _dev(q), 2.0, prob["radius"]).cpu().numpy()
    idx = np.sort(np.random.default_rng(166).choice(q.shape[0], 256, replace=False))
    Z64, _, _ = oracle.idw_modified(data, q[idx], 2.0, prob["radius"])
    ok = ~np.isnan(Z64)
    assert np.array_equal(np.isnan(Z[idx]), ~ok)
    assert np.max(np.abs(Z[idx][ok] - Z64[ok])) / np.max(np.abs(data[:, 2])) <= TOL


def test_prepared_index(idw):
    """The radius index serves modified Shepard queries too, at the build
    radius and below it."""
    prob = synthetic.config_local(n=6000, m=2000, members=30.0, seed=167)
    data, q = prob["data"], prob["queries"]
    ix = idw.LocalIndex(_dev(data), radius=prob["radius"])
    for r in (prob["radius"], prob["radius"] / 2):
        Z, cnt = ix.interpolate(_dev(q), 2.5, r, counts=True, modified=True)
        Z64, _, c64 = oracle.idw_modified(data, q, 2.5, r)
        assert np.array_equal(cnt.cpu().numpy(), c64)
        ok = ~np.isnan(Z64)
        Zc = Z.cpu().numpy()
        assert np.array_equal(np.isnan(Zc), ~ok)
        assert np.max(np.abs(Zc[ok] - Z64[ok])) / np.max(np.abs(data[:, 2])) <= TOL



def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / scale) if scale > 0 else float(np.max(np.abs(a)))


def _grad_compare(idw, data, q, p, radius, g, tol=1e-4):
    gz, gxy, gq, gp = idw.local_backward(_dev(data), _dev(q), p, radius, _dev(g), modified=True)
    torch.cuda.synchronize()
    G = oracle.idw_modified_grad(data, q, p, radius, g)
    errs = {"z": _rel(gz.cpu().numpy(), G["grad_z"]), "xy": _rel(gxy.cpu().numpy(), G["grad_xy"]),
            "q": _rel(gq.cpu().numpy(), G["grad_q"]),
            "p": abs(float(gp.cpu()[0]) - G["grad_p"]) / max(abs(G["grad_p"]), 1e-300)}
    for key, e in errs.items():
        assert e <= tol, (key, errs)


@pytest.mark.parametrize("p", [2.0, 3.5, 1.5])
def test_gradients_match_the_oracle(idw, p):
    """All four gradients of modified Shepard, within 1e-4 of each one's
    largest magnitude, with exact hits among the queries."""
    prob = synthetic.config_local(n=5003, m=3001, members=40.0, seed=168)
    data, q = prob["data"], prob["queries"].copy()
    q[::500] = data[:7 * 500:500, :2][: q[::500].shape[0]]
    g = np.random.default_rng(169).standard_normal(q.shape[0]).astype(np.float32)
    _grad_compare(idw, data, q, p, prob["radius"], g)


def test_gradients_clustered_and_fp64_path(idw):
    prob = synthetic.config_local(n=20000, m=3000, members=16.0, clustered=True, seed=170)
    g = np.random.default_rng(171).standard_normal(3000).astype(np.float32)
    _grad_compare(idw, prob["data"], prob["queries"], 2.0, prob["radius"], g)
    rng = np.random.default_rng(172)
    xy = (rng.random((400, 2)) * 3e-19).astype(np.float32)
    data = np.concatenate([xy, rng.standard_normal((400, 1)).astype(np.float32)], 1)
    q = (rng.random((150, 2)) * 3e-19).astype(np.float32)
    _grad_compare(idw, data, q, 2.5, 1e-19, rng.standard_normal(150).astype(np.float32))


def test_gradients_at_infinite_radius_are_the_global_adjoint(idw):
    prob = synthetic.uniform_problem(2000, 700, seed=173)
    g = np.random.default_rng(174).standard_normal(700).astype(np.float32)
    gz, gxy, gq, gp = idw.local_backward(_dev(prob["data"]), _dev(prob["queries"]), 2.5,
                                         float("inf"), _dev(g), modified=True)
    G = oracle.idw_grad(prob["data"], prob["queries"], 2.5, g)
    assert _rel(gz.cpu().numpy(), G["grad_z"]) <= 1e-4
    assert _rel(gxy.cpu().numpy(), G["grad_xy"]) <= 1e-4
    assert _rel(gq.cpu().numpy(), G["grad_q"]) <= 1e-4
    assert abs(float(gp.cpu()[0]) - G["grad_p"]) <= 1e-4 * abs(G["grad_p"])


def test_autograd_function(idw):
    prob = synthetic.config_local(n=4000, m=1500, members=25.0, seed=175)
    data, q, R = prob["data"], prob["queries"], prob["radius"]
    d = _dev(data).requires_grad_(True)
    qq = _dev(q).requires_grad_(True)
    p = torch.tensor(2.5, device="cuda", requires_grad=True)
    Z = idw.idw_modified(d, qq, p, R)
    w = torch.from_numpy(np.random.default_rng(176).standard_normal(1500).astype(np.float32)).cuda()
    ok = torch.isfinite(Z)
    (Z[ok] * w[ok]).sum().backward()
    g = np.where(ok.cpu().numpy(), w.cpu().numpy(), 0).astype(np.float32)
    G = oracle.idw_modified_grad(data, q, 2.5, R, g)
    gd = d.grad.cpu().numpy().astype(np.float64)
    assert _rel(gd[:, 2], G["grad_z"]) <= 1e-4
    assert _rel(gd[:, :2], G["grad_xy"]) <= 1e-4
    assert _rel(qq.grad.cpu().numpy(), G["grad_q"]) <= 1e-4
    assert abs(float(p.grad) - G["grad_p"]) <= 1e-4 * abs(G["grad_p"])
