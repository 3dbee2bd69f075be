"""Data sets whose 16-byte staged records pass 2^32 bytes (n > 2^28): every
byte offset and record index on the device must be 64-bit clean.  The
global, radius-limited and k-NN forms are checked on sampled queries
against the oracle, and the local forms' gradients through their hit and
sum rules.  About 12 GB of device memory and 3.3 GB of host memory.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

N = (1 << 28) + 12345
TOL = 2e-6


@pytest.fixture(scope="module")
def problem():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as idw
    rng = np.random.default_rng(2025)
    data = np.empty((N, 3), np.float32)
    data[:, :2] = rng.random((N, 2), dtype=np.float32)
    data[:, 2] = np.sin(6.283185307 * data[:, 0]) * np.cos(6.283185307 * data[:, 1])
    q = rng.random((300, 2), dtype=np.float32)
    q[7] = data[N - 3, :2]  # an exact hit near the end of the data
    d = torch.from_numpy(data).cuda()
    qq = torch.from_numpy(q).cuda()
    idx = np.sort(np.random.default_rng(3).choice(300, 24, replace=False))
    idx = np.union1d(idx, [7])
    yield idw, data, q, d, qq, idx
    del d, qq
    torch.cuda.empty_cache()


def test_global_form_past_4gb_of_staged_records(problem):
    idw, data, q, d, qq, idx = problem
    Z = idw.interpolate(d, qq, 2.0).cpu().numpy()
    Z64, hit = oracle.idw(data, q[idx], 2.0)
    assert hit[list(idx).index(7)] == N - 3
    err = np.max(np.abs(Z[idx].astype(np.float64) - Z64)) / np.max(np.abs(data[:, 2]))
    assert err <= TOL, err


def test_local_forms_past_4gb_of_sorted_records(problem):
    idw, data, q, d, qq, idx = problem
    R = 2e-4  # ~34 members per query at this density
    Z, cnt = idw.interpolate_local(d, qq, 2.0, R, counts=True)
    Zl, _, cl = oracle.idw_local(data, q[idx], 2.0, R)
    assert np.array_equal(cnt.cpu().numpy()[idx], cl)
    ok = ~np.isnan(Zl)
    err = np.max(np.abs(Z.cpu().numpy()[idx][ok] - Zl[ok])) / np.max(np.abs(data[:, 2]))
    assert err <= TOL, err
    Zk, nbr = idw.interpolate_knn(d, qq, 2.0, 16, neighbours=True)
    rk = oracle.idw_knn(data, q[idx], 2.0, 16)
    assert np.array_equal(nbr.cpu().numpy()[idx], rk["nbr"])
    assert rk["nbr"][list(idx).index(7), 0] == N - 3
    err = np.max(np.abs(Zk.cpu().numpy()[idx] - rk["Z"])) / np.max(np.abs(data[:, 2]))
    assert err <= TOL, err


def test_adjoint_past_4gb_of_staged_records(problem):
    """Query gradients on sampled queries against the oracle; the data-side
    gradients through partition of unity and translation invariance."""
    idw, data, q, d, qq, idx = problem
    p = 2.5
    keep = np.setdiff1d(np.arange(q.shape[0]), [7])  # no exact hit here
    qk = qq[torch.from_numpy(keep).cuda()].contiguous()
    g = torch.from_numpy(np.random.default_rng(4).standard_normal(keep.size).astype(np.float32))
    Z, s0, hit = idw.interpolate_saved(d, qk, p)
    gz, gxy, gq, _ = idw.backward(d, qk, p, Z, s0, hit, g.cuda(), need_p=False)
    idw.sync_status()
    sel = np.arange(0, keep.size, 25)
    G = oracle.idw_grad(data, q[keep][sel], p, g.numpy()[sel].astype(np.float64))
    gq = gq.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gq[sel] - G["grad_q"])) <= 1e-4 * np.max(np.abs(G["grad_q"]))
    g64 = g.numpy().astype(np.float64)
    assert abs(float(gz.double().sum()) - g64.sum()) <= 1e-4 * np.abs(g64).sum()
    gxy = gxy.cpu().numpy().astype(np.float64)
    total = gxy.sum(0) + gq.sum(0)
    assert np.all(np.abs(total) <= 1e-4 * (np.abs(gxy).sum(0) + np.abs(gq).sum(0)))


def test_local_gradients_past_4gb_of_records(problem):
    """Both local forms' gradients at n > 2^28: the exact hit's dL/dz lands
    on data point N - 3, dL/dz sums to sum_j g_j, and the coordinate
    gradients cancel (translation)."""
    idw, data, q, d, qq, idx = problem
    g = np.random.default_rng(6).standard_normal(q.shape[0]).astype(np.float32)
    gt = torch.from_numpy(g).cuda()
    for name, fn in (("local", lambda: idw.local_backward(d, qq, 2.0, 2e-4, gt)),
                     ("knn", lambda: idw.knn_backward(d, qq, 2.0, 16, gt))):
        gz, gxy, gq, _ = fn()
        torch.cuda.synchronize()
        assert abs(float(gz[N - 3]) - float(g[7])) <= 1e-6 * abs(float(g[7])), name
        assert abs(float(gz.double().sum()) - float(g.astype(np.float64).sum())) <= \
            1e-4 * float(np.abs(g).sum()), name
        tot = gxy.double().sum(0) + gq.double().sum(0)
        assert float(tot.abs().max()) <= 1e-4 * float(gq.double().abs().sum(0).max()), name
        del gz, gxy, gq
        torch.cuda.empty_cache()


def test_large_m_past_4gb_of_partials_and_query_records():
    """m = 2^28 + 123 queries against 64 points: the 16-byte partial-sum
    slots and sorted query records pass 2^32 bytes."""
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as idw
    M = (1 << 28) + 123
    rng = np.random.default_rng(2026)
    data = np.empty((64, 3), np.float32)
    data[:, :2] = rng.random((64, 2), dtype=np.float32)
    data[:, 2] = rng.standard_normal(64).astype(np.float32)
    qd = torch.rand(M, 2, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    d = torch.from_numpy(data).cuda()
    sel = torch.tensor([0, 1, 12345, M // 2, M - 2, M - 1], device="cuda")
    qs = qd[sel].cpu().numpy()
    zmax = np.max(np.abs(data[:, 2]))
    Z = idw.interpolate(d, qd, 2.0)
    Z64, _ = oracle.idw(data, qs, 2.0)
    assert np.max(np.abs(Z[sel].cpu().numpy() - Z64)) / zmax <= TOL
    del Z
    Zl = idw.interpolate_local(d, qd, 2.0, 0.2)
    Zl64, _, _ = oracle.idw_local(data, qs, 2.0, 0.2)
    a = Zl[sel].cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(Zl64))
    ok = ~np.isnan(Zl64)
    assert np.max(np.abs(a[ok] - Zl64[ok]), initial=0.0) / zmax <= TOL
    del Zl
    Zk = idw.interpolate_knn(d, qd, 2.0, 8)
    rk = oracle.idw_knn(data, qs, 2.0, 8)
    assert np.max(np.abs(Zk[sel].cpu().numpy() - rk["Z"])) / zmax <= TOL
    del Zk, qd
    torch.cuda.empty_cache()
