"""GPU parity of the prepared local index against the FP64 oracle.

A ``LocalIndex`` builds the data side of a local form once (grid plan and
counting sort, plus the count tables for k-NN); each query call sorts only
its queries.  Its results must be those of the one-shot calls: radius
members and k-NN neighbour lists bit for bit against the oracle, values
within the global form's bar (error = max_j |Z_gpu - Z_64| / max_i |z_i|
<= 2e-6), NaN where nothing is selected, exact z at hits.
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


def _check_values(data, Z, Z64, hit64):
    assert np.array_equal(np.isnan(Z), np.isnan(Z64))
    h = hit64 >= 0
    assert np.array_equal(Z[h], data[hit64[h], 2])
    ok = ~np.isnan(Z64)
    if ok.any():
        err = np.max(np.abs(Z[ok].astype(np.float64) - Z64[ok])) / np.max(np.abs(data[:, 2]))
        assert err <= TOL_F32C, err


def _radius_query(ix, data, q, p, radius):
    Z, cnt = ix.interpolate(_dev(q), p, radius, counts=True)
    torch.cuda.synchronize()
    Z, cnt = Z.cpu().numpy(), cnt.cpu().numpy()
    Z64, hit64, cnt64 = oracle.idw_local(data, q, p, radius)
    assert np.array_equal(cnt, cnt64), np.nonzero(cnt != cnt64)[0][:10]
    _check_values(data, Z, Z64, hit64)
    return Z, cnt


def _knn_query(ix, data, q, p, k):
    Z, nbr, kd2 = ix.knn(_dev(q), p, k, neighbours=True, kth_d2=True)
    torch.cuda.synchronize()
    Z, nbr, kd2 = Z.cpu().numpy(), nbr.cpu().numpy(), kd2.cpu().numpy()
    r = oracle.idw_knn(data, q, p, k)
    bad = np.nonzero(np.any(nbr != r["nbr"], axis=1))[0]
    assert bad.size == 0, (bad[:5], nbr[bad[:2]], r["nbr"][bad[:2]])
    assert np.array_equal(np.isnan(kd2), np.isnan(r["kd2"]))
    ok = ~np.isnan(kd2)
    assert np.array_equal(kd2[ok], r["kd2"][ok])
    _check_values(data, Z, r["Z"], r["hit"])
    return Z, nbr


@pytest.mark.parametrize("p", [2.0, 3.5])
def test_radius_index_many_batches_and_smaller_radii(idw, p):
    """One index, several query batches (ragged sizes, one with exact hits),
    at the build radius and below it."""
    prob = synthetic.uniform_problem(5003, 2001, seed=91, exact_hits=7)
    data = prob["data"]
    R = 0.03
    ix = idw.LocalIndex(_dev(data), radius=R)
    for seed, m in ((92, 2001), (93, 1), (94, 777)):
        q = prob["queries"] if seed == 92 else synthetic.uniform_problem(10, m, seed=seed)["queries"]
        for r in (R, R / 2, R / 7):
            _radius_query(ix, data, q, p, r)
    ix.close()


@pytest.mark.parametrize("build_k", [1, 16, 64])
def test_knn_index_any_k(idw, build_k):
    """Cells sized for build_k, queried at every k: the selection does not
    depend on the cell size."""
    prob = synthetic.uniform_problem(5003, 1501, seed=95, exact_hits=5)
    ix = idw.LocalIndex(_dev(prob["data"]), k=build_k)
    for k in (1, 5, 16, 33, 64):
        _knn_query(ix, prob["data"], prob["queries"], 2.0, k)
    ix.close()


def test_clustered_both_forms(idw):
    prob = synthetic.config_local(seed=96, n=20000, m=3000, members=16.0, clustered=True)
    data, q = prob["data"], prob["queries"]
    rix = idw.LocalIndex(_dev(data), radius=prob["radius"])
    _, cnt = _radius_query(rix, data, q, 2.0, prob["radius"])
    assert (cnt == 0).any() and cnt.max() > 100
    kix = idw.LocalIndex(_dev(data), k=32)
    for k in (1, 8, 32):
        _knn_query(kix, data, q, 2.0, k)


def test_index_keeps_its_own_copy(idw):
    """The data tensor is overwritten after the build: queries still see the
    data the index was built from."""
    prob = synthetic.uniform_problem(3000, 800, seed=97)
    data = prob["data"]
    d = _dev(data)
    rix = idw.LocalIndex(d, radius=0.05)
    kix = idw.LocalIndex(d, k=8)
    torch.cuda.synchronize()
    d.fill_(123.0)
    _radius_query(rix, data, prob["queries"], 2.0, 0.05)
    _knn_query(kix, data, prob["queries"], 2.0, 8)


def test_degenerate_data(idw):
    """n = 1, every point coincident, a line, non-finite points, an infinite
    radius (one cell: the global form) and far or non-finite queries."""
    prob = synthetic.uniform_problem(3000, 300, seed=98, exact_hits=4)
    far = np.array([[-5, 0.5], [0.5, 9], [1e6, -1e6], [np.nan, 0.1]], np.float32)
    q = np.concatenate([prob["queries"], far]).astype(np.float32)
    one = prob["data"][:1]
    same = prob["data"][:200].copy()
    same[:, :2] = 0.5
    line = prob["data"].copy()
    line[:, 0] = 0.25
    nf = prob["data"].copy()
    nf[::7, 1] = np.inf
    for data in (one, same, line, nf):
        _radius_query(idw.LocalIndex(_dev(data), radius=0.05), data, q, 2.0, 0.05)
        _knn_query(idw.LocalIndex(_dev(data), k=9), data, q, 2.0, 9)
    gix = idw.LocalIndex(_dev(prob["data"]), radius=float("inf"))
    _radius_query(gix, prob["data"], q, 2.0, float("inf"))
    _radius_query(gix, prob["data"], q, 2.0, 0.02)


def test_argument_errors(idw):
    prob = synthetic.uniform_problem(2000, 100, seed=99)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    rix = idw.LocalIndex(d, radius=0.05)
    kix = idw.LocalIndex(d, k=8)
    for call in (lambda: rix.interpolate(q, 2.0, 0.051),  # above the build radius
                 lambda: rix.interpolate(q, 2.0, 0.0),
                 lambda: rix.interpolate(q, 2.0, float("nan")),
                 lambda: rix.interpolate(q, 0.0),
                 lambda: rix.knn(q, 2.0, 8),  # the other form
                 lambda: kix.interpolate(q, 2.0, 0.01),
                 lambda: kix.knn(q, 2.0, 0),
                 lambda: kix.knn(q, 2.0, 65),
                 lambda: idw.LocalIndex(d, k=0),
                 lambda: idw.LocalIndex(d, k=65),
                 lambda: idw.LocalIndex(d, radius=-1.0)):
        with pytest.raises(idw.IDWError) as e:
            call()
        assert e.value.name == "IDW_ERR_INVALID_ARG"
    assert rix.interpolate(q[:0], 2.0).shape == (0,)


def test_graph_capture_and_replay(idw):
    prob = synthetic.uniform_problem(4000, 1500, seed=100)
    data = prob["data"]
    rix = idw.LocalIndex(_dev(data), radius=0.04)
    kix = idw.LocalIndex(_dev(data), k=16)
    q = _dev(prob["queries"])
    zr = torch.empty(q.shape[0], dtype=torch.float32, device="cuda")
    zk = torch.empty_like(zr)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # grows the workspace outside the capture
        rix.interpolate(q, 2.0, out=zr)
        kix.knn(q, 2.0, out=zk)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rix.interpolate(q, 2.0, out=zr)
        kix.knn(q, 2.0, out=zk)
    zmax = np.max(np.abs(data[:, 2]))
    for seed in (101, 102):
        qn = synthetic.uniform_problem(10, 1500, seed=seed)["queries"]
        q.copy_(_dev(qn))
        g.replay()
        torch.cuda.synchronize()
        Zr, _, _ = oracle.idw_local(data, qn, 2.0, 0.04)
        rk = oracle.idw_knn(data, qn, 2.0, 16)
        ok = ~np.isnan(Zr)
        assert np.max(np.abs(zr.cpu().numpy()[ok] - Zr[ok])) / zmax <= TOL_F32C
        assert np.max(np.abs(zk.cpu().numpy() - rk["Z"])) / zmax <= TOL_F32C


def test_two_handles_on_two_streams(idw):
    """Queries only read the index: two handles on two streams use it at
    the same time."""
    prob = synthetic.uniform_problem(6000, 3000, seed=103)
    data = prob["data"]
    ix = idw.LocalIndex(_dev(data), k=12)
    torch.cuda.synchronize()
    qa, qb = _dev(prob["queries"][:1500]), _dev(prob["queries"][1500:])
    ha, hb = idw.Handle(0), idw.Handle(0)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    sa.wait_stream(torch.cuda.current_stream())
    sb.wait_stream(torch.cuda.current_stream())
    outs = []
    for h, s, qq in ((ha, sa, qa), (hb, sb, qb)):
        with torch.cuda.stream(s):
            outs.append(ix.knn(qq, 2.0, neighbours=True, handle=h))
    torch.cuda.synchronize()
    nbr = np.concatenate([outs[0][1].cpu().numpy(), outs[1][1].cpu().numpy()])
    r = oracle.idw_knn(data, prob["queries"], 2.0, 12)
    assert np.array_equal(nbr, r["nbr"])
    ha.close()
    hb.close()


def test_full_size_matches_one_shot(idw):
    """N = M = 2^20, R for 32 members and k = 32 (the benchmarked sizes): the
    index's members and neighbour lists equal the one-shot calls' for every
    query, and 128 sampled queries match the oracle."""
    prob = synthetic.config_local()
    data, q = prob["data"], prob["queries"]
    d, qd = _dev(data), _dev(q)
    R = prob["radius"]
    Z1, c1 = idw.interpolate_local(d, qd, 2.0, R, counts=True)
    rix = idw.LocalIndex(d, radius=R)
    Z2, c2 = rix.interpolate(qd, 2.0, counts=True)
    assert torch.equal(c1, c2)
    K1, n1 = idw.interpolate_knn(d, qd, 2.0, 32, neighbours=True)
    kix = idw.LocalIndex(d, k=32)
    K2, n2 = kix.knn(qd, 2.0, 32, neighbours=True)
    assert torch.equal(n1, n2)
    idx = np.sort(np.random.default_rng(104).choice(q.shape[0], 128, replace=False))
    zmax = np.max(np.abs(data[:, 2]))
    Zo, _, co = oracle.idw_local(data, q[idx], 2.0, R)
    assert np.array_equal(c2.cpu().numpy()[idx], co)
    assert np.nanmax(np.abs(Z2.cpu().numpy()[idx] - Zo)) / zmax <= TOL_F32C
    ro = oracle.idw_knn(data, q[idx], 2.0, 32)
    assert np.array_equal(n2.cpu().numpy()[idx], ro["nbr"])
    assert np.max(np.abs(K2.cpu().numpy()[idx] - ro["Z"])) / zmax <= TOL_F32C
