"""Every entry point shares one handle's workspace.  Interleave them on one
handle, with sizes that grow and shrink the workspace, and check each
result against the oracle: nothing may depend on what an earlier call left
behind."""
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
    return m


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def _err(Z, Z64, data):
    Z = Z.cpu().numpy().astype(np.float64)
    ok = ~np.isnan(Z64)
    assert np.array_equal(np.isnan(Z), ~ok)
    return float(np.max(np.abs(Z[ok] - Z64[ok])) / np.max(np.abs(data[:, 2]))) if ok.any() else 0.0


def test_interleaved_entry_points_on_one_handle(idw):
    h = idw.Handle(torch.cuda.current_device())
    for rnd, (n, m) in enumerate([(5000, 3000), (40000, 20000), (700, 900), (25000, 1500)]):
        prob = synthetic.uniform_problem(n, m, seed=90 + rnd, exact_hits=4)
        data, q = prob["data"], prob["queries"]
        d, qq = _dev(data), _dev(q)
        Z64, _ = oracle.idw(data, q, 2.5)
        assert _err(idw.interpolate(d, qq, 2.5, handle=h), Z64, data) <= TOL

        R = 0.05
        Zl, cnt = idw.interpolate_local(d, qq, 2.0, R, counts=True, handle=h)
        Zl64, _, cnt64 = oracle.idw_local(data, q, 2.0, R)
        assert np.array_equal(cnt.cpu().numpy(), cnt64)
        assert _err(Zl, Zl64, data) <= TOL

        Zk, nbr = idw.interpolate_knn(d, qq, 3.0, 7, neighbours=True, handle=h)
        rk = oracle.idw_knn(data, q, 3.0, 7)
        assert np.array_equal(nbr.cpu().numpy(), rk["nbr"])
        assert _err(Zk, rk["Z"], data) <= TOL

        other = synthetic.uniform_problem(max(10, n // 3), max(10, m // 2), seed=190 + rnd)
        outs = idw.interpolate_batched([d, _dev(other["data"])], [qq, _dev(other["queries"])],
                                       2.0, handle=h)
        Zb64, _ = oracle.idw(other["data"], other["queries"], 2.0)
        assert _err(outs[1], Zb64, other["data"]) <= TOL

        Zs, s0, hit = idw.interpolate_saved(d, qq, 2.0, handle=h)
        g = torch.ones(m, device="cuda")
        gz, _, _, _ = idw.backward(d, qq, 2.0, Zs, s0, hit, g, handle=h)
        # Partition of unity: sum_i dL/dz_i = sum_j g_j.
        assert abs(float(gz.double().sum()) - m) <= 1e-4 * m

        Zd = idw.interpolate(_dev(data, torch.float64), _dev(q, torch.float64), 2.5, "f64",
                             handle=h)
        assert _err(Zd, Z64, data) <= 1e-13

        # The local forms' gradients and prepared indexes on the same handle.
        gl = torch.linspace(-1.0, 1.0, m, device="cuda")
        Gl = oracle.idw_local_grad(data, q, 2.0, R, gl.cpu().numpy())
        gz, _, gq, _ = idw.local_backward(d, qq, 2.0, R, gl, handle=h)
        assert np.max(np.abs(gz.cpu().numpy() - Gl["grad_z"])) <= 1e-4 * np.max(np.abs(Gl["grad_z"]))
        Gk = oracle.idw_knn_grad(data, q, 3.0, 7, gl.cpu().numpy())
        _, _, gq, _ = idw.knn_backward(d, qq, 3.0, 7, gl, handle=h)
        assert np.max(np.abs(gq.cpu().numpy() - Gk["grad_q"])) <= 1e-4 * np.max(np.abs(Gk["grad_q"]))
        rix = idw.LocalIndex(d, radius=R, handle=h)
        assert np.array_equal(rix.interpolate(qq, 2.0, counts=True)[1].cpu().numpy(), cnt64)
        kix = idw.LocalIndex(d, k=7, handle=h)
        assert np.array_equal(kix.knn(qq, 3.0, neighbours=True)[1].cpu().numpy(), rk["nbr"])
    idw.sync_status(handle=h)
    h.close()
