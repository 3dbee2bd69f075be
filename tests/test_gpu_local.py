"""GPU parity of the local (radius-limited) form against the FP64 oracle.

The local form is Eq. 1 over the data points within distance R of each
query (the local Shepard interpolation of the paper's related work, Sec. 1).
Membership is decided by the same FP32 expression on both sides, so the
member counts must be identical; values are compared as for the global form
(error = max_j |Z_gpu - Z_64| / max_i |z_i| <= 2e-6), NaN where a query has
no member, and bit-exact z at exact hits.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _run(idw, data, q, p, radius):
    Z, cnt = idw.interpolate_local(_dev(data), _dev(q), p, radius, counts=True)
    torch.cuda.synchronize()
    return Z.cpu().numpy(), cnt.cpu().numpy()


def _compare(idw, data, q, p, radius, tol=TOL_F32C):
    Z, cnt = _run(idw, data, q, p, radius)
    Z64, hit64, cnt64 = oracle.idw_local(data, q, p, radius)
    assert np.array_equal(cnt, cnt64), np.nonzero(cnt != cnt64)[0][:10]
    assert np.array_equal(np.isnan(Z), np.isnan(Z64))
    h = hit64 >= 0
    assert np.array_equal(Z[h], data[hit64[h], 2])
    ok = ~np.isnan(Z64)
    if ok.any():
        zmax = np.max(np.abs(data[:, 2]))
        err = np.max(np.abs(Z[ok].astype(np.float64) - Z64[ok])) / zmax
        assert err <= tol, err
    return Z, cnt, Z64, cnt64


@pytest.mark.parametrize("p", [2.0, 3.5, 1.0])
@pytest.mark.parametrize("members", [8.0, 40.0, 300.0])
def test_uniform_ragged(idw, p, members):
    """N = 5003, M = 3001 (no size a multiple of a warp or block); R for 8,
    40 or 300 members on average, so lanes take 1 to 10+ candidates."""
    prob = synthetic.config_local(n=5003, m=3001, members=members)
    _, cnt, _, _ = _compare(idw, prob["data"], prob["queries"], p, prob["radius"])
    assert cnt.max() > 0


def test_clustered(idw):
    """Gaussian-mixture data (dense blobs: cells with hundreds of points,
    empty space between them, so many queries have no member)."""
    prob = synthetic.config_local(n=20000, m=4000, members=16.0, clustered=True)
    for p in (2.0, 2.5):
        _, cnt, _, _ = _compare(idw, prob["data"], prob["queries"], p, prob["radius"])
        assert (cnt == 0).any() and cnt.max() > 100


def test_infinite_radius_is_the_global_form(idw):
    prob = synthetic.uniform_problem(3000, 777, seed=11)
    data, q = prob["data"], prob["queries"]
    for p in (2.0, 3.0):
        Z, cnt = _run(idw, data, q, p, float("inf"))
        assert np.all(cnt == data.shape[0])
        Zg, _ = oracle.idw(data, q, p)
        assert np.max(np.abs(Z - Zg)) / np.max(np.abs(data[:, 2])) <= TOL_F32C
        # Huge finite R (R^2 overflows FP32 to +inf): the same.
        Z2, cnt2 = _run(idw, data, q, p, 1e30)
        assert np.array_equal(cnt2, cnt)


def test_exact_hits_and_tiny_radius(idw):
    """Planted exact hits return the data z bit for bit at any R, even when
    fl32(R^2) underflows to 0 and no other query has a member."""
    prob = synthetic.uniform_problem(4000, 1000, seed=12, exact_hits=50)
    data, q = prob["data"], prob["queries"]
    # Append a copy of a hit point's (x, y) with another z: the lower index wins.
    extra = np.array([[*data[prob["hit_d"][0], :2], 123.0]], np.float32)
    data = np.concatenate([data, extra])
    for radius in (0.05, 1e-6, 1e-30, 1e-60):
        Z, cnt, _, _ = _compare(idw, data, q, 2.0, radius)
        hq = prob["hit_q"]
        assert np.all(cnt[hq] == -1)
        assert np.array_equal(Z[hq], data[prob["hit_d"], 2])
    assert np.isnan(Z[np.setdiff1d(np.arange(q.shape[0]), hq)]).all()


def test_queries_outside_the_box(idw):
    prob = synthetic.config_local(n=2000, m=16, members=20.0)
    data = prob["data"]
    R = prob["radius"]
    q = np.array([[-0.5, 0.5], [1.5, 0.5], [0.5, -3.0], [0.5, 9.0], [1e30, 0.0], [-1e30, -1e30],
                  [-R / 2, 0.5], [0.5, 1 + R / 2], [-R / 2, -R / 2], [1 + R / 3, 1 + R / 3],
                  [np.nan, 0.5], [0.5, np.inf]], np.float32)
    Z, cnt, _, _ = _compare(idw, data, q, 2.0, R)
    assert np.all(cnt[:6] == 0) and np.isnan(Z[:6]).all()
    assert np.all(cnt[10:] == 0) and np.isnan(Z[10:]).all()


def test_boundary_points_at_distance_r(idw):
    """A lattice of spacing 1/8 with R = 1/4, queries on removed lattice
    nodes: the four axis neighbours lie exactly R away (d^2 == fl32(R^2)) and
    are not members (strict <), leaving the 8 nodes of the 3 x 3 block."""
    g = np.arange(17, dtype=np.float32) / 8
    xx, yy = np.meshgrid(g, g, indexing="xy")
    xy = np.stack([xx.ravel(), yy.ravel()], 1)
    q = np.array([[0.5, 0.5], [1.0, 0.75], [0.25, 1.875]], np.float32)
    keep = ~np.any(np.all(xy[:, None, :] == q[None, :, :], axis=2), axis=1)
    xy = xy[keep]
    data = np.concatenate([xy, xy[:, :1] * 3 - xy[:, 1:]], 1).astype(np.float32)
    qn = np.concatenate([q, q + np.float32(1e-7), q - np.float32(3e-8)]).astype(np.float32)
    _, cnt, _, _ = _compare(idw, data, qn, 2.0, 0.25)
    assert np.all(cnt[:3] == 8)


def test_fp32_range_edges_take_the_fp64_path(idw):
    """Neighbours 1e-30 apart (d^2 underflows to 0 in FP32, so the FP32
    weights overflow) and neighbours ~1e16 apart (weights below 2^-100, or
    flushed to 0 at p = 8) are redone in FP64."""
    rng = np.random.default_rng(13)
    tiny = (rng.random((300, 2)) * 1e-30).astype(np.float32)
    data = np.concatenate([tiny, rng.standard_normal((300, 1)).astype(np.float32)], 1)
    qt = (rng.random((64, 2)) * 1e-30).astype(np.float32)
    for p in (2.0, 3.0):
        _, cnt, _, _ = _compare(idw, data, qt, p, 1e-20)
        assert np.all(cnt == 300)
    huge = (rng.random((300, 2)) * 1e17).astype(np.float32)
    data2 = np.concatenate([huge, rng.standard_normal((300, 1)).astype(np.float32)], 1)
    qh = (rng.random((64, 2)) * 1e17).astype(np.float32)
    for p in (2.0, 8.0):
        _, cnt, _, _ = _compare(idw, data2, qh, p, 3e16)
        assert cnt.max() > 20


def test_large_p(idw):
    prob = synthetic.config_local(n=3000, m=500, members=50.0)
    _compare(idw, prob["data"], prob["queries"], 40.0, prob["radius"])


def test_non_finite_data_points_are_ignored(idw):
    prob = synthetic.config_local(n=3000, m=600, members=30.0)
    data = prob["data"].copy()
    data[::7, 0] = np.nan
    data[3::11, 1] = np.inf
    data[5::13, 0] = -np.inf
    _compare(idw, data, prob["queries"], 2.0, prob["radius"])
    data[:, 0] = np.nan  # no finite point at all
    Z, cnt = _run(idw, data, prob["queries"], 2.0, prob["radius"])
    assert np.all(cnt == 0) and np.isnan(Z).all()


def test_single_point_and_degenerate_box(idw):
    prob = synthetic.config_local(n=1000, m=300, members=30.0)
    d1 = prob["data"][:1]
    _compare(idw, d1, prob["queries"], 2.0, 0.3)
    line = prob["data"].copy()
    line[:, 0] = 0.25  # zero-width box in x
    _compare(idw, line, prob["queries"], 2.0, 0.05)
    same = prob["data"].copy()
    same[:, :2] = 0.5  # every point coincides
    q = np.concatenate([prob["queries"], [[0.5, 0.5]]]).astype(np.float32)
    Z, cnt, _, _ = _compare(idw, same, q, 2.0, 0.2)
    assert cnt[-1] == -1 and Z[-1] == same[0, 2]


def test_counts_optional_and_repeatable(idw):
    prob = synthetic.config_local(n=20000, m=5000, members=32.0)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    Z1 = idw.interpolate_local(d, q, 2.0, prob["radius"])
    Z2, _ = idw.interpolate_local(d, q, 2.0, prob["radius"], counts=True)
    a, b = Z1.cpu().numpy(), Z2.cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a)
    # Scatter order may change the FP64 sums' rounding; the FP32 results
    # agree to within one ulp.
    assert np.all(np.abs(a[ok] - b[ok]) <= np.spacing(np.abs(a[ok])))


def test_argument_errors(idw):
    prob = synthetic.config_local(n=100, m=10, members=5.0)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(idw.IDWError):
            idw.interpolate_local(d, q, 2.0, bad)
    with pytest.raises(idw.IDWError):
        idw.interpolate_local(d, q, -2.0, 0.1)
    empty = torch.empty(0, 2, dtype=torch.float32, device="cuda")
    assert idw.interpolate_local(d, empty, 2.0, 0.1).shape == (0,)


def test_graph_capture_and_replay(idw):
    """The whole local form (box, grid plan, sorts, gather) is captured into
    one CUDA graph; replays on new inputs in the same buffers match the
    oracle."""
    prob = synthetic.config_local(n=4000, m=1500, members=20.0)
    R = prob["radius"]
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    out = torch.empty(q.shape[0], dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        idw.interpolate_local(d, q, 2.0, R, out=out)  # workspace sized before capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        idw.interpolate_local(d, q, 2.0, R, out=out)
    for seed in (21, 22):
        p2 = synthetic.config_local(seed=seed, n=4000, m=1500, members=20.0)
        d.copy_(_dev(p2["data"]))
        q.copy_(_dev(p2["queries"]))
        g.replay()
        torch.cuda.synchronize()
        Z = out.cpu().numpy()
        Z64, _, _ = oracle.idw_local(p2["data"], p2["queries"], 2.0, R)
        assert np.array_equal(np.isnan(Z), np.isnan(Z64))
        ok = ~np.isnan(Z64)
        err = np.max(np.abs(Z[ok] - Z64[ok])) / np.max(np.abs(p2["data"][:, 2]))
        assert err <= TOL_F32C, err


def test_full_size_sampled(idw):
    """N = M = 2^20, R for 32 members: the benchmarked launch, checked on 256
    sampled queries the oracle computes one by one."""
    prob = synthetic.config_local()
    data, q, R = prob["data"], prob["queries"], prob["radius"]
    Z, cnt = _run(idw, data, q, 2.0, R)
    idx = np.sort(np.random.default_rng(14).choice(q.shape[0], 256, replace=False))
    Z64, _, cnt64 = oracle.idw_local(data, q[idx], 2.0, R)
    assert np.array_equal(cnt[idx], cnt64)
    ok = ~np.isnan(Z64)
    assert np.array_equal(np.isnan(Z[idx]), ~ok)
    err = np.max(np.abs(Z[idx][ok].astype(np.float64) - Z64[ok])) / np.max(np.abs(data[:, 2]))
    assert err <= TOL_F32C, err
    assert 20 < cnt[cnt >= 0].mean() < 40
