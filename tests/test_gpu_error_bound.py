"""The FP32 form's worst-case error bound on the GPU (Eq. 1, Sec. 2.1).

* The adversarial input of ``synthetic.dominant_first`` (a near point
  followed or preceded, inside its block, by 63 points whose weights are
  below half an ulp of its weight) against the FP64 oracle, element by
  element, through every sweep variant and the log2/exp2 form.  A sequential
  64-point chunk misses the bar on it by 1.7x (tests/test_error_bound.py
  emulates that on the CPU).
* The MUFU approximations' accuracy, measured over every fp32 input: the
  reciprocal must stay within the one ulp (2^-23 relative) the bound uses.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6
U = 2.0 ** -24


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


@pytest.fixture(scope="module")
def adversarial():
    prob = synthetic.dominant_first()
    Z64, hit64 = oracle.idw(prob["data"], prob["queries"], 2.0)
    assert np.all(hit64 < 0)
    return prob, Z64


def _err(Z, Z64, data):
    return np.abs(Z.cpu().numpy().astype(np.float64) - Z64) / np.max(np.abs(data[:, 2]))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_dominant_first_each_variant(idw, adversarial, variant):
    prob, Z64 = adversarial
    h = idw.Handle(0)
    idw.set_option("sweep_variant", variant, handle=h)
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    Z = idw.interpolate(d, q, 2.0, handle=h)
    idw.sync_status(handle=h)
    e = _err(Z, Z64, prob["data"])
    h.close()
    assert e.max() <= TOL_F32C, (variant, e.max(), prob["positions"][int(e.argmax())])


def test_dominant_first_default_and_general_form(idw, adversarial):
    prob, Z64 = adversarial
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    assert _err(idw.interpolate(d, q, 2.0), Z64, prob["data"]).max() <= TOL_F32C
    h = idw.Handle(0)
    idw.set_option("force_general_power", 1, handle=h)
    e = _err(idw.interpolate(d, q, 2.0, handle=h), Z64, prob["data"])
    h.close()
    assert e.max() <= TOL_F32C, e.max()


def test_dominant_first_replicated_in_a_large_problem(idw):
    """The adversarial blocks repeated through a 2^17-point data set (far
    copies shifted by whole units), with the same queries: the near point of
    each query now sits in the middle of a long run of work units."""
    prob = synthetic.dominant_first()
    data = prob["data"]
    reps = (1 << 17) // data.shape[0] + 1
    shifted = [data.copy() for _ in range(reps)]
    for r, block in enumerate(shifted):
        block[:, 0] += np.float32(8.0 * (r // 2))
        if r % 2:
            block[:, 1] += np.float32(8.0)
    # Keep the original copy (shift 0) in the middle of the array.
    shifted[0], shifted[reps // 2] = shifted[reps // 2], shifted[0]
    big = np.ascontiguousarray(np.concatenate(shifted)[: 1 << 17])
    qs = prob["queries"]
    Z64, _ = oracle.idw(big, qs, 2.0)
    Z = idw.interpolate(torch.from_numpy(big).cuda(), torch.from_numpy(qs).cuda(), 2.0)
    assert _err(Z, Z64, big).max() <= TOL_F32C


def test_mufu_errors_exhaustive(idw):
    e = idw.measure_mufu_errors(0)
    print("MUFU accuracy over all fp32 inputs:", e,
          {k: v / U for k, v in e.items()}, "(units of u = 2^-24)")
    assert 0.0 < e["rcp_rel"] <= 2 * U       # one ulp: the constant of the bound
    assert 0.0 < e["lg2_abs"] <= 2.0 ** -21
    assert 0.0 < e["ex2_rel"] <= 2.0 ** -21
    assert 0.0 < e["lg2_rel_outer"] <= 2.0 ** -21


@pytest.mark.parametrize("p", [0.5, 1.5, 3.5, 6.0])
def test_fma_log2_option_matches_oracle(idw, p):
    """IDW_OPT_FMA_LOG2: one pair in 16 takes log2 d^2 from the FMA-pipe
    polynomial; ragged sizes (padding records), exact hits and the bar."""
    prob = synthetic.uniform_problem(9001, 4099, seed=int(10 * p) + 150, exact_hits=5)
    d = torch.from_numpy(prob["data"]).cuda()
    q = torch.from_numpy(prob["queries"]).cuda()
    h = idw.Handle(0)
    idw.set_option("fma_log2", 1, handle=h)
    Z = idw.interpolate(d, q, p, handle=h)
    idw.sync_status(handle=h)
    assert idw.get_option("last_variant", handle=h) == 4
    Z64, _ = oracle.idw(prob["data"], prob["queries"], p)
    e = _err(Z, Z64, prob["data"])
    h.close()
    assert e.max() <= TOL_F32C, e.max()
    hq = torch.from_numpy(prob["hit_q"]).cuda()
    assert torch.equal(Z[hq].cpu(), torch.from_numpy(prob["data"][prob["hit_d"], 2]))
