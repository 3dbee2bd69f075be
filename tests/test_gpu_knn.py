"""GPU parity of the k-nearest-neighbour form against the FP64 oracle.

Eq. 1 over the k data points nearest to each query, nearness being the key
(FP32 d^2, index), the local form of the paper's related work (Sec. 1).
Both sides rank by the same FP32 expression, so the neighbour lists and the
k-th keys must be identical; values are compared as for the global form
(error = max_j |Z_gpu - Z_64| / max_i |z_i| <= 2e-6), NaN where nothing is
selected, and bit-exact z at exact hits.  Each test runs under both k-NN searches
(one thread per query, one warp per slice of a row's queries).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6


@pytest.fixture(scope="module", params=[0, 1], ids=["thread_search", "warp_search"])
def idw(request):
    """The library with the default handle's k-NN search set to one thread
    per query (0) or one warp per row slice of queries (1); every test runs
    under both, and both must select the same neighbours."""
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    before = m.get_option("knn_search")
    m.set_option("knn_search", request.param)
    yield m
    m.set_option("knn_search", before)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _compare(idw, data, q, p, k, tol=TOL_F32C):
    Z, nbr, kd2 = idw.interpolate_knn(_dev(data), _dev(q), p, k, neighbours=True, kth_d2=True)
    torch.cuda.synchronize()
    Z, nbr, kd2 = Z.cpu().numpy(), nbr.cpu().numpy(), kd2.cpu().numpy()
    r = oracle.idw_knn(data, q, p, k)
    bad = np.nonzero(np.any(nbr != r["nbr"], axis=1))[0]
    assert bad.size == 0, (bad[:5], nbr[bad[:2]], r["nbr"][bad[:2]])
    assert np.array_equal(np.isnan(kd2), np.isnan(r["kd2"]))
    ok = ~np.isnan(kd2)
    assert np.array_equal(kd2[ok], r["kd2"][ok])
    assert np.array_equal(np.isnan(Z), np.isnan(r["Z"]))
    h = r["hit"] >= 0
    assert np.array_equal(Z[h], data[r["hit"][h], 2])
    fin = ~np.isnan(r["Z"])
    if fin.any():
        zmax = np.nanmax(np.abs(data[:, 2]))
        err = np.max(np.abs(Z[fin].astype(np.float64) - r["Z"][fin])) / zmax
        assert err <= tol, err
    return Z, nbr, r


@pytest.mark.parametrize("k", [1, 5, 16, 32, 64])
@pytest.mark.parametrize("p", [2.0, 3.5])
def test_uniform_ragged(idw, k, p):
    prob = synthetic.uniform_problem(5003, 2001, seed=51, exact_hits=7)
    _compare(idw, prob["data"], prob["queries"], p, k)


def test_clustered(idw):
    prob = synthetic.config_local(seed=52, n=20000, m=3000, clustered=True)
    for k in (1, 8, 32):
        _compare(idw, prob["data"], prob["queries"], 2.0, k)


def test_ties_on_a_lattice(idw):
    """Queries at lattice nodes and cell centres: many exactly equal keys,
    decided by the lower index on both sides."""
    g = np.arange(40, dtype=np.float32) / 32
    xx, yy = np.meshgrid(g, g, indexing="xy")
    xy = np.stack([xx.ravel(), yy.ravel()], 1)
    perm = np.random.default_rng(53).permutation(xy.shape[0])
    data = np.concatenate([xy[perm], np.arange(xy.shape[0], dtype=np.float32)[:, None]], 1)
    q = np.concatenate([xy[::13] + np.float32(1 / 64), xy[::17]]).astype(np.float32)
    for k in (1, 2, 4, 5, 9, 13):
        _compare(idw, data, q, 2.0, k)


def test_fewer_points_than_k_and_tiny_inputs(idw):
    prob = synthetic.uniform_problem(40, 100, seed=54)
    for n in (1, 2, 7, 40):
        _, nbr, _ = _compare(idw, prob["data"][:n], prob["queries"], 2.0, 32)
        assert np.all(nbr[:, n:] == -1)


def test_queries_far_outside_and_non_finite(idw):
    prob = synthetic.uniform_problem(3000, 50, seed=55)
    data = prob["data"].copy()
    data[::9, 0] = np.nan
    data[4::11, 1] = np.inf
    q = np.concatenate([prob["queries"], np.array(
        [[-0.5, 0.5], [1.5, 0.5], [0.5, -3.0], [2.0, 9.0], [1e6, 0.0], [-1e30, 1e30],
         [np.nan, 0.2], [0.3, np.inf]], np.float32)]).astype(np.float32)
    Z, nbr, r = _compare(idw, data, q, 2.0, 8)
    assert np.isnan(Z[-2:]).all() and np.all(nbr[-2:] == -1)


def test_degenerate_layouts(idw):
    prob = synthetic.uniform_problem(3000, 400, seed=56, exact_hits=5)
    line = prob["data"].copy()
    line[:, 0] = 0.25  # a vertical line: one column of cells
    _compare(idw, line, prob["queries"], 2.0, 8)
    same = prob["data"][:200].copy()
    same[:, :2] = 0.5  # every point coincides
    q = np.concatenate([prob["queries"], [[0.5, 0.5]]]).astype(np.float32)
    Z, _, _ = _compare(idw, same, q, 2.0, 16)
    assert Z[-1] == same[0, 2]


def test_fp32_range_edges(idw):
    rng = np.random.default_rng(57)
    tiny = (rng.random((300, 2)) * 1e-30).astype(np.float32)
    data = np.concatenate([tiny, rng.standard_normal((300, 1)).astype(np.float32)], 1)
    _compare(idw, data, (rng.random((64, 2)) * 1e-30).astype(np.float32), 2.0, 8)
    huge = (rng.random((300, 2)) * 1e17).astype(np.float32)
    data2 = np.concatenate([huge, rng.standard_normal((300, 1)).astype(np.float32)], 1)
    for p in (2.0, 8.0):
        _compare(idw, data2, (rng.random((64, 2)) * 1e17).astype(np.float32), p, 8)


def test_outputs_optional_and_argument_errors(idw):
    prob = synthetic.uniform_problem(2000, 500, seed=58)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    Z1 = idw.interpolate_knn(d, q, 2.0, 12)
    Z2, nbr = idw.interpolate_knn(d, q, 2.0, 12, neighbours=True)
    a, b = Z1.cpu().numpy(), Z2.cpu().numpy()
    assert np.all(np.abs(a - b) <= np.spacing(np.abs(a)))
    for bad_k in (0, -1, 65):
        with pytest.raises(idw.IDWError):
            idw.interpolate_knn(d, q, 2.0, bad_k)
    with pytest.raises(idw.IDWError):
        idw.interpolate_knn(d, q, 0.0, 4)


def test_graph_capture_and_replay(idw):
    prob = synthetic.uniform_problem(4000, 1500, seed=59)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    out = torch.empty(q.shape[0], dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        idw.interpolate_knn(d, q, 2.0, 16, out=out)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        idw.interpolate_knn(d, q, 2.0, 16, out=out)
    for seed in (60, 61):
        p2 = synthetic.uniform_problem(4000, 1500, seed=seed)
        d.copy_(_dev(p2["data"]))
        q.copy_(_dev(p2["queries"]))
        g.replay()
        torch.cuda.synchronize()
        r = oracle.idw_knn(p2["data"], p2["queries"], 2.0, 16)
        err = np.max(np.abs(out.cpu().numpy() - r["Z"])) / np.max(np.abs(p2["data"][:, 2]))
        assert err <= TOL_F32C, err


def test_full_size_sampled(idw):
    """N = M = 2^20, k = 32: the benchmarked launch, checked on 128 sampled
    queries (neighbour lists, k-th keys and values)."""
    prob = synthetic.config_local()
    data, q = prob["data"], prob["queries"]
    Z, nbr, kd2 = idw.interpolate_knn(_dev(data), _dev(q), 2.0, 32, neighbours=True, kth_d2=True)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(62).choice(q.shape[0], 128, replace=False))
    r = oracle.idw_knn(data, q[idx], 2.0, 32)
    assert np.array_equal(nbr.cpu().numpy()[idx], r["nbr"])
    assert np.array_equal(kd2.cpu().numpy()[idx], r["kd2"])
    err = np.max(np.abs(Z.cpu().numpy()[idx] - r["Z"])) / np.max(np.abs(data[:, 2]))
    assert err <= TOL_F32C, err


def test_option_values(idw):
    assert idw.get_option("knn_search") in (0, 1)
    for bad in (-1, 2):
        with pytest.raises(idw.IDWError):
            idw.set_option("knn_search", bad)


def test_rows_of_many_queries(idw):
    """Rows of cells holding many queries (several warps per row, the last
    one partial) and rows holding none: dense query bands across sparse
    data, so a warp's queries span few columns and its rectangle is wide."""
    rng = np.random.default_rng(63)
    data = np.concatenate([rng.random((6000, 2)), rng.standard_normal((6000, 1))], 1)
    data = data.astype(np.float32)
    band = np.stack([rng.random(4000), 0.5 + 0.002 * rng.random(4000)], 1)
    corner = 0.05 * rng.random((37, 2))
    q = np.concatenate([band, corner]).astype(np.float32)
    for k in (1, 16, 64):
        _compare(idw, data, q, 2.0, k)
