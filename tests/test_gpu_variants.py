"""Every compiled sweep variant, the forced log2/exp2 form at p = 2, and the
autotuner: each is a separate code path and must meet the same parity bar
against the FP64 oracle."""
import os

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


def _err(Z, Z64, data):
    return float(np.max(np.abs(Z.cpu().numpy().astype(np.float64) - Z64)) /
                 np.max(np.abs(data[:, 2])))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("p", [2.0, 3.5])
def test_each_variant_matches_oracle(idw, variant, p):
    prob = synthetic.config_exact_hits(seed=60 + variant, n=9001, m=5003, hits=9)
    h = idw.Handle(0)
    idw.set_option("sweep_variant", variant, handle=h)
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    Z = idw.interpolate(d, q, p, handle=h)
    assert idw.get_option("last_variant", handle=h) == (variant if (variant != 5 or p == 2.0) else 0)
    Z64, _ = oracle.idw(prob["data"], prob["queries"], p)
    assert _err(Z, Z64, prob["data"]) <= TOL_F32C
    hq = torch.from_numpy(prob["hit_q"]).cuda()
    assert torch.equal(Z[hq].cpu(), torch.from_numpy(prob["data"][prob["hit_d"], 2]))
    # The batched entry point with the same variant.
    outs = idw.interpolate_batched([d, d[:777].contiguous()], [q, q[:100].contiguous()], p,
                                   handle=h)
    assert _err(outs[0], Z64, prob["data"]) <= TOL_F32C
    h.close()


def test_forced_general_form_at_p2(idw):
    prob = synthetic.uniform_problem(7000, 6000, seed=61, exact_hits=4)
    h = idw.Handle(0)
    idw.set_option("force_general_power", 1, handle=h)
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    Z = idw.interpolate(d, q, 2.0, handle=h)
    Z64, _ = oracle.idw(prob["data"], prob["queries"], 2.0)
    assert _err(Z, Z64, prob["data"]) <= TOL_F32C
    h.close()


def test_autotuner_picks_and_persists(idw, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("IDW_AUTOTUNE_CACHE", str(cache))
    prob = synthetic.uniform_problem(20000, 12000, seed=62)
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    h = idw.Handle(0)
    idw.set_option("autotune", 1, handle=h)
    Z = idw.interpolate(d, q, 2.0, handle=h)
    v = idw.get_option("last_variant", handle=h)
    assert 0 <= v < 6 and idw.get_option("tuned_classes", handle=h) == 1
    Z2 = idw.interpolate(d, q, 2.0, handle=h)      # cached: same variant, same bits
    assert idw.get_option("last_variant", handle=h) == v and torch.equal(Z, Z2)
    Z64, _ = oracle.idw(prob["data"], prob["queries"], 2.0)
    assert _err(Z, Z64, prob["data"]) <= TOL_F32C
    h.close()
    assert cache.exists() and '"sm' in cache.read_text()
    h2 = idw.Handle(0)                               # a new handle reads the cache
    assert idw.get_option("tuned_classes", handle=h2) >= 1
    idw.set_option("autotune", 1, handle=h2)
    idw.interpolate(d, q, 2.0, handle=h2)
    assert idw.get_option("last_variant", handle=h2) == v
    h2.close()


def test_option_errors(idw):
    h = idw.Handle(0)
    with pytest.raises(idw.IDWError):
        idw.set_option("sweep_variant", 9, handle=h)
    assert h.lib.idw_set_option(h.ptr, 77, 1) == 1  # unknown option
    h.close()


@pytest.mark.parametrize("p", [2.0, 3.5])
def test_fp64_staging_layouts_are_bit_identical(idw, p):
    """The plain FP64 form staged as Hybrid (default), AoaS double4 records
    or SoA: the same arithmetic in the same order, so bit-identical results,
    each within 1e-13 of the oracle (the paper's FP64 layout question,
    Sec. 4.1.2, asked of this library's sweep)."""
    prob = synthetic.config_exact_hits(seed=77, n=5003, m=2051, hits=5)
    d = torch.from_numpy(prob["data"]).cuda().double()
    q = torch.from_numpy(prob["queries"]).cuda().double()
    Z64, _ = oracle.idw(prob["data"], prob["queries"], p)
    outs = []
    for layout in (-1, 1, 2):
        h = idw.Handle(0)
        idw.set_option("staging_layout", layout, handle=h)
        Z = idw.interpolate(d, q, p, "f64", handle=h).cpu().numpy()
        h.close()
        assert np.max(np.abs(Z - Z64)) / np.max(np.abs(prob["data"][:, 2])) <= 1e-13, layout
        outs.append(Z)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("p", [2.0, 3.5])
def test_each_staging_layout_matches_oracle(idw, layout, p):
    prob = synthetic.config_exact_hits(seed=70 + layout, n=6001, m=4099, hits=7)
    h = idw.Handle(0)
    idw.set_option("staging_layout", layout, handle=h)
    assert idw.get_option("staging_layout", handle=h) == layout
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    Z = idw.interpolate(d, q, p, handle=h)
    Z64, _ = oracle.idw(prob["data"], prob["queries"], p)
    assert _err(Z, Z64, prob["data"]) <= TOL_F32C
    hq = torch.from_numpy(prob["hit_q"]).cuda()
    assert torch.equal(Z[hq].cpu(), torch.from_numpy(prob["data"][prob["hit_d"], 2]))
    h.close()
