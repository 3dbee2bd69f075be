"""Input validation (IDW_OPT_VALIDATE_INPUTS) and the autotune cache given
at handle creation (idw_create_ex).

With validation on, every entry point scans its inputs first and refuses
NaN or infinite values with IDW_ERR_NOT_FINITE_INPUT, computing nothing;
clean inputs give the same results as without validation.
"""
import json

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


@pytest.fixture()
def vh(idw):
    h = idw.Handle(torch.cuda.current_device())
    idw.set_option("validate_inputs", 1, handle=h)
    yield h
    h.close()


def _prob(seed=71, n=3000, m=700):
    p = synthetic.uniform_problem(n, m, seed=seed)
    return torch.from_numpy(p["data"]).cuda(), torch.from_numpy(p["queries"]).cuda()


def _expect_not_finite(idw, fn):
    with pytest.raises(idw.IDWError) as e:
        fn()
    assert e.value.name == "IDW_ERR_NOT_FINITE_INPUT"


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), float("-inf")])
def test_every_entry_point_refuses_non_finite_inputs(idw, vh, bad):
    d, q = _prob()
    dbad = d.clone()
    dbad[1234, 2] = bad          # a value
    qbad = q.clone()
    qbad[321, 0] = bad           # a query coordinate
    assert idw.get_option("validate_inputs", handle=vh) == 1
    for dd, qq in ((dbad, q), (d, qbad)):
        _expect_not_finite(idw, lambda: idw.interpolate(dd, qq, 2.0, handle=vh))
        _expect_not_finite(idw, lambda: idw.interpolate(dd.double(), qq.double(), 2.0, "f64",
                                                        handle=vh))
        _expect_not_finite(idw, lambda: idw.interpolate_local(dd, qq, 2.0, 0.05, handle=vh))
        _expect_not_finite(idw, lambda: idw.interpolate_knn(dd, qq, 2.0, 8, handle=vh))
        _expect_not_finite(idw, lambda: idw.paper_interpolate(dd, qq, 2.0, handle=vh))
        _expect_not_finite(idw, lambda: idw.interpolate_batched([d, dd], [q, qq], 2.0, handle=vh))
        _expect_not_finite(idw, lambda: idw.local_backward(dd, qq, 2.0, 0.05, torch.ones(
            qq.shape[0], device="cuda"), handle=vh))
        _expect_not_finite(idw, lambda: idw.knn_backward(dd, qq, 2.0, 8, torch.ones(
            qq.shape[0], device="cuda"), handle=vh))
    # The prepared index scans its data when built and its queries per call.
    _expect_not_finite(idw, lambda: idw.LocalIndex(dbad, radius=0.05, handle=vh))
    _expect_not_finite(idw, lambda: idw.LocalIndex(dbad, k=8, handle=vh))
    rix = idw.LocalIndex(d, radius=0.05, handle=vh)
    kix = idw.LocalIndex(d, k=8, handle=vh)
    _expect_not_finite(idw, lambda: rix.interpolate(qbad, 2.0))
    _expect_not_finite(idw, lambda: kix.knn(qbad, 2.0))
    Z, s0, hit = idw.interpolate_saved(d, q, 2.0, handle=vh)
    g = torch.ones(q.shape[0], device="cuda")
    g[7] = bad
    _expect_not_finite(idw, lambda: idw.backward(d, q, 2.0, Z, s0, hit, g, handle=vh))
    _expect_not_finite(idw, lambda: idw.local_backward(d, q, 2.0, 0.05, g, handle=vh))
    _expect_not_finite(idw, lambda: idw.knn_backward(d, q, 2.0, 8, g, handle=vh))


def test_clean_inputs_give_the_same_results(idw, vh):
    d, q = _prob(seed=72)
    plain = idw.Handle(torch.cuda.current_device())
    for fn in (lambda h: idw.interpolate(d, q, 2.0, handle=h),
               lambda h: idw.interpolate_local(d, q, 2.0, 0.05, handle=h),
               lambda h: idw.interpolate_knn(d, q, 2.0, 8, handle=h),
               lambda h: idw.LocalIndex(d, radius=0.05, handle=h).interpolate(q, 2.0),
               lambda h: idw.LocalIndex(d, k=8, handle=h).knn(q, 2.0)):
        a = fn(vh).cpu().numpy()
        b = fn(plain).cpu().numpy()
        assert np.array_equal(np.isnan(a), np.isnan(b))
        ok = ~np.isnan(a)
        assert np.all(np.abs(a[ok] - b[ok]) <= np.spacing(np.abs(b[ok])))
    plain.close()


# The refused call leaves nothing in the graph, which torch reports.
@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_validation_refuses_stream_capture(idw, vh):
    d, q = _prob(seed=73)
    out = torch.empty(q.shape[0], device="cuda")
    idw.interpolate(d, q, 2.0, out=out, handle=vh)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(idw.IDWError, match="UNSUPPORTED"):
        with torch.cuda.graph(g):
            idw.interpolate(d, q, 2.0, out=out, handle=vh)
    torch.cuda.synchronize()
    idw.set_option("validate_inputs", 0, handle=vh)
    assert idw.get_option("validate_inputs", handle=vh) == 0


def test_autotune_cache_given_at_creation(idw, tmp_path):
    path = str(tmp_path / "tune.json")
    d, q = _prob(seed=74, n=20000, m=20000)
    h = idw.Handle(torch.cuda.current_device(), autotune_cache=path)
    idw.set_option("autotune", 1, handle=h)
    idw.interpolate(d, q, 2.0, handle=h)
    torch.cuda.synchronize()
    assert idw.get_option("tuned_classes", handle=h) >= 1
    h.close()
    with open(path) as f:
        table = json.load(f)
    assert len(table) >= 1
    h2 = idw.Handle(torch.cuda.current_device(), autotune_cache=path)
    assert idw.get_option("tuned_classes", handle=h2) == len(table)
    h2.close()


def test_misaligned_pointers_are_refused(idw):
    """Every device pointer is checked for its element alignment on the host,
    before any launch (IDW_ERR_ALIGNMENT)."""
    import ctypes
    h = idw.get_handle()
    lib = h.lib
    buf = torch.zeros(4096, dtype=torch.float64, device="cuda")
    base = buf.data_ptr()
    ok32, bad32 = base, base + 2          # float32 needs 4-byte alignment
    ok64, bad64 = base, base + 4          # float64 needs 8-byte alignment
    s = torch.cuda.current_stream().cuda_stream
    P = ctypes.c_void_p

    def fwd(prec, d, q, o):
        return lib.idw_interpolate(h.ptr, P(d), 16, P(q), 16, 2.0, prec, P(o), P(s))

    assert fwd(0, bad32, ok32, ok32) == 2
    assert fwd(0, ok32, bad32, ok32) == 2
    assert fwd(0, ok32, ok32, bad32) == 2
    assert fwd(1, bad64, ok64, ok64) == 2
    assert fwd(1, ok64, ok64, bad64) == 2
    assert lib.idw_interpolate_saved(h.ptr, P(ok32), 16, P(ok32), 16, 2.0, 0, P(ok32), P(bad64),
                                     P(ok32), P(s)) == 2
    assert lib.idw_interpolate_local(h.ptr, P(ok32), 16, P(ok32), 16, 2.0, 0.1, P(ok32),
                                     P(bad32), P(s)) == 2
    assert lib.idw_interpolate_knn(h.ptr, P(ok32), 16, P(ok32), 16, 2.0, 4, P(ok32), P(bad32),
                                   P(ok32), P(s)) == 2
    torch.cuda.synchronize()
    assert torch.count_nonzero(buf) == 0  # nothing was launched


def test_binding_refuses_bad_output_buffers(idw):
    """Every caller-supplied output or saved-state buffer is checked (size,
    dtype, device, layout) before the library is called."""
    d, q = _prob(seed=72, n=500, m=300)
    m = q.shape[0]
    short = torch.empty(m - 1, device="cuda")
    with pytest.raises(ValueError, match="hold"):
        idw.interpolate(d, q, 2.0, out=short)
    with pytest.raises(ValueError, match="float64"):
        idw.interpolate(d.double(), q.double(), 2.0, "f64", out=torch.empty(m, device="cuda"))
    with pytest.raises(ValueError, match="must be on"):
        idw.interpolate(d, q, 2.0, out=torch.empty(m))
    with pytest.raises(ValueError, match="contiguous"):
        idw.interpolate(d, q, 2.0, out=torch.empty(m, 2, device="cuda")[:, 0])
    with pytest.raises(ValueError, match="hold"):
        idw.interpolate_saved(d, q, 2.0, out=short)
    with pytest.raises(ValueError, match="hold"):
        idw.interpolate_batched([d, d], [q, q[:10].contiguous()], 2.0,
                                outs=[torch.empty(m, device="cuda"), torch.empty(9, device="cuda")])
    with pytest.raises(ValueError, match="outs must hold 2"):
        idw.interpolate_batched([d, d], [q, q], 2.0, outs=[torch.empty(m, device="cuda")])
    with pytest.raises(ValueError, match="hold"):
        idw.interpolate_local(d, q, 2.0, 0.1, out=short)
    with pytest.raises(ValueError, match="hold"):
        idw.interpolate_modified(d, q, 2.0, 0.1, out=short)
    with pytest.raises(ValueError, match="hold"):
        idw.interpolate_knn(d, q, 2.0, 8, out=short)
    with pytest.raises(ValueError, match="hold"):
        idw.paper_interpolate(d, q, 2.0, out=short)
    ix = idw.LocalIndex(d, k=8)
    with pytest.raises(ValueError, match="hold"):
        ix.knn(q, 2.0, out=short)
    ix.close()
    Z, s0, hit = idw.interpolate_saved(d, q, 2.0)
    g = torch.ones(m, device="cuda")
    with pytest.raises(ValueError, match="s0 must be torch.float64"):
        idw.backward(d, q, 2.0, Z, s0.float(), hit, g)
    with pytest.raises(ValueError, match="grad_out must hold"):
        idw.backward(d, q, 2.0, Z, s0, hit, g[:-1])
    with pytest.raises(ValueError, match="grad_out must be a tensor on"):
        idw.knn_backward(d, q, 2.0, 8, g.cpu())
    # Nothing above reached the library: the handle still computes.
    idw.sync_status()
    assert torch.isfinite(idw.interpolate(d, q, 2.0)).all()


def test_batched_problems_must_share_one_device(idw):
    if torch.cuda.device_count() < 2:
        d, q = _prob(seed=73, n=100, m=50)
        with pytest.raises(ValueError, match="must be on"):
            idw.interpolate_batched([d, d], [q, q], 2.0,
                                    outs=[torch.empty(50, device="cuda"), torch.empty(50)])
        return
    d0, q0 = _prob(seed=73, n=100, m=50)
    d1, q1 = d0.to("cuda:1"), q0.to("cuda:1")
    with pytest.raises(ValueError, match="every problem must be on"):
        idw.interpolate_batched([d0, d1], [q0, q1], 2.0)
