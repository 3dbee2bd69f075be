"""Parity at the full workload sizes, in the launch configuration the
benchmark times, on sampled outputs the FP64 oracle computes one by one
(and, for the data-side gradients, identities that hold at any size).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6
TOL_GRAD = 1e-4


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    return m


def test_clustered_full_size_sampled(idw):
    """N = 262144 Gaussian-mixture data, 1024^2 query grid, p in {1.5, 2, 3.5}."""
    prob = synthetic.config_clustered()
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    idx = np.sort(np.random.default_rng(7).choice(q.shape[0], 384, replace=False))
    zmax = np.max(np.abs(prob["data"][:, 2]))
    for p in prob["p_values"]:
        Z = idw.interpolate(d, q, p).cpu().numpy()
        Z64, _ = oracle.idw(prob["data"], prob["queries"][idx], p)
        assert np.max(np.abs(Z[idx].astype(np.float64) - Z64)) / zmax <= TOL_F32C, p


def test_adjoint_full_size_sampled(idw):
    """N = M = 262144, p = 2.5: sampled query gradients against the oracle;
    data gradients through partition of unity and translation invariance."""
    prob = synthetic.config_adjoint()
    data, q, g, p = prob["data"], prob["queries"], prob["grad_out"], prob["p"]
    d = torch.from_numpy(data).cuda()
    qq = torch.from_numpy(q).cuda()
    Z, s0, hit = idw.interpolate_saved(d, qq, p)
    gz, gxy, gq, gp = idw.backward(d, qq, p, Z, s0, hit, torch.from_numpy(g).cuda())
    idw.sync_status()
    gz = gz.cpu().numpy().astype(np.float64)
    gxy = gxy.cpu().numpy().astype(np.float64)
    gq = gq.cpu().numpy().astype(np.float64)
    idx = np.sort(np.random.default_rng(8).choice(q.shape[0], 128, replace=False))
    G = oracle.idw_grad(data, q[idx], p, g[idx])
    scale = np.max(np.abs(G["grad_q"]))
    assert np.max(np.abs(gq[idx] - G["grad_q"])) <= TOL_GRAD * scale
    # sum_i dZ_j/dz_i = 1 for every query j, so sum_i dL/dz_i = sum_j g_j.
    g64 = g.astype(np.float64)
    assert abs(gz.sum() - g64.sum()) <= TOL_GRAD * np.abs(g64).sum()
    # Moving every point and query together leaves Z unchanged.
    total = gxy.sum(0) + gq.sum(0)
    assert np.all(np.abs(total) <= TOL_GRAD * (np.abs(gxy).sum(0) + np.abs(gq).sum(0)))
    assert np.isfinite(float(gp.cpu()[0]))


def test_batch_full_size_sampled(idw):
    """256 problems, N_i and M_i log-uniform in [1024, 262144], one call."""
    batch = synthetic.config_batch()
    inst = batch["instances"]
    d = [torch.from_numpy(i["data"]).cuda() for i in inst]
    q = [torch.from_numpy(i["queries"]).cuda() for i in inst]
    outs = idw.interpolate_batched(d, q, 2.0)
    idw.sync_status()
    rng = np.random.default_rng(9)
    for k in rng.choice(len(inst), 16, replace=False):
        m = inst[k]["queries"].shape[0]
        idx = np.sort(rng.choice(m, min(m, 128), replace=False))
        Z64, _ = oracle.idw(inst[k]["data"], inst[k]["queries"][idx], 2.0)
        Z = outs[k].cpu().numpy()[idx].astype(np.float64)
        assert np.max(np.abs(Z - Z64)) / np.max(np.abs(inst[k]["data"][:, 2])) <= TOL_F32C, k
