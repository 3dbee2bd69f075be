"""Batched forward: many independent problems of Eq. 1 in one persistent
launch (work units of all problems split evenly over the grid).

Each problem of the batch is compared with the FP64 oracle element by
element, and with the single-problem entry point.
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
    return m


def _problems(sizes, seed):
    out = []
    for k, (n, m) in enumerate(sizes):
        out.append(synthetic.uniform_problem(int(n), int(m), seed=seed + k,
                                             exact_hits=3 if m > 10 and n > 10 else 0))
    return out


def _check(idw, probs, p, outs):
    for prob, o in zip(probs, outs):
        Z = o.cpu().numpy()
        Z64, hit64 = oracle.idw(prob["data"], prob["queries"], p)
        err = np.max(np.abs(Z.astype(np.float64) - Z64)) / np.max(np.abs(prob["data"][:, 2]))
        assert err <= TOL_F32C, (prob["data"].shape, err)
        hq = prob["hit_q"]
        assert np.array_equal(Z[hq], prob["data"][prob["hit_d"], 2])


@pytest.mark.parametrize("p", [2.0, 3.5])
def test_uneven_batch_matches_oracle(idw, p):
    rng = np.random.default_rng(5)
    sizes = np.exp(rng.uniform(np.log(1), np.log(30000), size=(40, 2))).astype(int) + 1
    sizes[3] = (1, 1)
    sizes[7] = (257, 2049)
    probs = _problems(sizes, 100)
    d = [torch.from_numpy(pr["data"]).cuda() for pr in probs]
    q = [torch.from_numpy(pr["queries"]).cuda() for pr in probs]
    outs = idw.interpolate_batched(d, q, p)
    idw.sync_status()
    _check(idw, probs, p, outs)
    # The single-problem entry point agrees within the same bound.
    for dk, qk, ok, pr in zip(d[:8], q[:8], outs[:8], probs[:8]):
        single = idw.interpolate(dk, qk, p)
        zmax = float(np.abs(pr["data"][:, 2]).max())
        assert float((single.double() - ok.double()).abs().max()) <= 2 * TOL_F32C * zmax


def test_batch_larger_than_one_launch_and_empty_members(idw):
    rng = np.random.default_rng(6)
    sizes = rng.integers(1, 700, size=(300, 2))
    probs = _problems(sizes, 500)
    d = [torch.from_numpy(pr["data"]).cuda() for pr in probs]
    q = [torch.from_numpy(pr["queries"]).cuda() for pr in probs]
    q[10] = torch.empty(0, 2, device="cuda")
    q[290] = torch.empty(0, 2, device="cuda")
    outs = idw.interpolate_batched(d, q, 2.0)
    idw.sync_status()
    keep = [k for k in range(300) if k not in (10, 290)]
    _check(idw, [probs[k] for k in keep], 2.0, [outs[k] for k in keep])
    assert outs[10].numel() == 0 and outs[290].numel() == 0


def test_batch_is_deterministic(idw):
    sizes = [(5000, 3000), (100, 9000), (20000, 500)]
    probs = _problems(sizes, 900)
    d = [torch.from_numpy(pr["data"]).cuda() for pr in probs]
    q = [torch.from_numpy(pr["queries"]).cuda() for pr in probs]
    a = [o.clone() for o in idw.interpolate_batched(d, q, 2.0)]
    b = idw.interpolate_batched(d, q, 2.0)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_batched_call_is_graph_capturable(idw):
    """The batched entry point only enqueues work on the caller's stream, so a
    CUDA graph of it replays to the same results (after one warm-up call that
    sizes the workspace)."""
    sizes = [(3000, 2000), (40, 7000), (12000, 900), (1, 5)]
    probs = _problems(sizes, 1200)
    d = [torch.from_numpy(pr["data"]).cuda() for pr in probs]
    q = [torch.from_numpy(pr["queries"]).cuda() for pr in probs]
    outs = [torch.empty(x.shape[0], device="cuda") for x in q]
    eager = [o.clone() for o in idw.interpolate_batched(d, q, 2.0)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        idw.interpolate_batched(d, q, 2.0, outs=outs)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        idw.interpolate_batched(d, q, 2.0, outs=outs)
    for o in outs:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, outs):
        assert torch.equal(a, b)


def test_fp64_batch_matches_oracle(idw):
    """The plain FP64 form through the batched entry (one call per instance)."""
    probs = _problems([(300, 200), (1, 5), (2049, 257), (50, 0), (4000, 3000)], 300)
    d = [torch.from_numpy(pr["data"]).cuda().double() for pr in probs]
    q = [torch.from_numpy(pr["queries"]).cuda().double() for pr in probs]
    outs = idw.interpolate_batched(d, q, 2.5, precision="f64")
    idw.sync_status()
    for pr, o in zip(probs, outs):
        if pr["queries"].shape[0] == 0:
            continue
        Z64, _ = oracle.idw(pr["data"], pr["queries"], 2.5)
        err = np.max(np.abs(o.cpu().numpy() - Z64)) / np.max(np.abs(pr["data"][:, 2]))
        assert err <= 1e-13, err
