"""IDW_OPT_LOCAL_QUERY_ORDER: the local forms keep the caller's query order
instead of sorting the queries into cells.  The results must not change:
member counts and neighbour lists bit for bit against the oracle, values
within 2e-6, on random and on raster (row-major grid) queries, for the
one-shot calls, the prepared index and the k-NN gradients.  The radius
form's gradients sort regardless.
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


@pytest.fixture()
def kept(idw):
    h = idw.Handle(torch.cuda.current_device())
    idw.set_option("local_query_order", 1, handle=h)
    yield h
    h.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _raster(g):
    c = (np.arange(g, dtype=np.float64) + 0.5) / g
    xx, yy = np.meshgrid(c, c, indexing="xy")
    return np.stack([xx.ravel(), yy.ravel()], 1).astype(np.float32)


def _values(Z, Z64, data):
    Z = Z.cpu().numpy()
    assert np.array_equal(np.isnan(Z), np.isnan(Z64))
    ok = ~np.isnan(Z64)
    if ok.any():
        assert np.max(np.abs(Z[ok] - Z64[ok])) / np.max(np.abs(data[:, 2])) <= TOL


@pytest.mark.parametrize("queries", ["random", "raster"])
def test_results_do_not_depend_on_the_order(idw, kept, queries):
    prob = synthetic.uniform_problem(6000, 2500, seed=151, exact_hits=6)
    data = prob["data"]
    q = prob["queries"] if queries == "random" else _raster(48)
    d, qq = _dev(data), _dev(q)
    assert idw.get_option("local_query_order", handle=kept) == 1
    R = 0.04
    Zl64, _, c64 = oracle.idw_local(data, q, 2.0, R)
    rk = oracle.idw_knn(data, q, 2.0, 12)
    Z, cnt = idw.interpolate_local(d, qq, 2.0, R, counts=True, handle=kept)
    assert np.array_equal(cnt.cpu().numpy(), c64)
    _values(Z, Zl64, data)
    Zk, nbr = idw.interpolate_knn(d, qq, 2.0, 12, neighbours=True, handle=kept)
    assert np.array_equal(nbr.cpu().numpy(), rk["nbr"])
    _values(Zk, rk["Z"], data)
    rix = idw.LocalIndex(d, radius=R, handle=kept)
    Zi, ci = rix.interpolate(qq, 2.0, counts=True)
    assert np.array_equal(ci.cpu().numpy(), c64)
    _values(Zi, Zl64, data)
    kix = idw.LocalIndex(d, k=12, handle=kept)
    Zki, ni = kix.knn(qq, 2.0, neighbours=True)
    assert np.array_equal(ni.cpu().numpy(), rk["nbr"])
    _values(Zki, rk["Z"], data)


def test_gradients_with_the_caller_order(idw, kept):
    prob = synthetic.uniform_problem(5000, 2000, seed=152, exact_hits=4)
    data, q = prob["data"], prob["queries"]
    g = np.random.default_rng(153).standard_normal(2000).astype(np.float32)
    d, qq, gt = _dev(data), _dev(q), _dev(g)
    for fn, ref in ((lambda: idw.knn_backward(d, qq, 2.0, 10, gt, handle=kept),
                     lambda: oracle.idw_knn_grad(data, q, 2.0, 10, g)),
                    (lambda: idw.local_backward(d, qq, 2.0, 0.05, gt, handle=kept),
                     lambda: oracle.idw_local_grad(data, q, 2.0, 0.05, g))):
        gz, gxy, gq, _ = fn()
        G = ref()
        for got, want in ((gz, G["grad_z"]), (gxy, G["grad_xy"]), (gq, G["grad_q"])):
            assert np.max(np.abs(got.cpu().numpy() - want)) <= 1e-4 * np.max(np.abs(want))


def test_option_values(idw, kept):
    with pytest.raises(idw.IDWError):
        idw.set_option("local_query_order", 2, handle=kept)
    idw.set_option("local_query_order", 0, handle=kept)
    assert idw.get_option("local_query_order", handle=kept) == 0
