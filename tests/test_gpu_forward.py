"""GPU parity of the forward pass against the FP64 oracle (Eq. 1, Sec. 2.1).

Every test calls the CUDA library through its C ABI (via the thin binding)
and compares with ``oracle`` element by element on the same seeded inputs.

Bars (error = max_j |Z_gpu - Z_64| / max_i |z_i|):
  * FP32-compensated form: <= 2e-6, and bit-exact z_k at exact hits;
  * plain FP64 form: <= 1e-13, and bit-exact at exact hits;
  * exact-hit indices: identical.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32C = 2e-6
TOL_F64 = 1e-13


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    import paper_1402_4986_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _rel_err(zg, z64, zvals):
    return float(np.max(np.abs(np.asarray(zg, np.float64) - z64)) / np.max(np.abs(zvals)))


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _run(idw, data, q, p, precision="f32c"):
    dt = torch.float32 if precision == "f32c" else torch.float64
    Z, s0, hit = idw.interpolate_saved(_dev(data, dt), _dev(q, dt), p, precision)
    idw.sync_status()
    return Z.cpu().numpy(), s0.cpu().numpy(), hit.cpu().numpy()


def test_exact_hit_config_f32c_and_f64(idw):
    prob = synthetic.config_exact_hits()
    data, q, p = prob["data"], prob["queries"], prob["p"]
    Z64, hit64 = oracle.idw(data, q, p)
    for prec, tol in (("f32c", TOL_F32C), ("f64", TOL_F64)):
        Z, s0, hit = _run(idw, data, q, p, prec)
        assert np.array_equal(np.nonzero(hit >= 0)[0], np.nonzero(hit64 >= 0)[0]), prec
        assert np.array_equal(hit[hit >= 0], hit64[hit64 >= 0]), prec
        hq = prob["hit_q"]
        assert np.array_equal(Z[hq], data[prob["hit_d"], 2].astype(Z.dtype)), prec
        assert np.all(np.isinf(s0[hq]))
        err = _rel_err(Z, Z64, data[:, 2])
        assert err <= tol, (prec, err)


@pytest.mark.parametrize("n,m", [(1, 1), (2, 3), (3, 31), (31, 257), (255, 2047), (256, 2048),
                                 (257, 2049), (1000, 4099), (4097, 333), (20000, 5000)])
@pytest.mark.parametrize("p", [2.0, 3.5])
def test_ragged_sizes(idw, n, m, p):
    prob = synthetic.uniform_problem(n, m, seed=n * 7 + m)
    data, q = prob["data"], prob["queries"]
    Z64, hit64 = oracle.idw(data, q, p)
    Z, _, hit = _run(idw, data, q, p, "f32c")
    assert np.array_equal(hit >= 0, hit64 >= 0)
    assert _rel_err(Z, Z64, data[:, 2]) <= TOL_F32C
    Zd, _, _ = _run(idw, data, q, p, "f64")
    assert _rel_err(Zd, Z64, data[:, 2]) <= TOL_F64


@pytest.mark.parametrize("p", [0.5, 1.5, 2.5, 3.5, 6.0])
def test_general_power(idw, p):
    prob = synthetic.uniform_problem(6000, 7000, seed=int(p * 10))
    data, q = prob["data"], prob["queries"]
    Z64, _ = oracle.idw(data, q, p)
    Z, _, _ = _run(idw, data, q, p, "f32c")
    assert _rel_err(Z, Z64, data[:, 2]) <= TOL_F32C, p
    Zd, _, _ = _run(idw, data, q, p, "f64")
    assert _rel_err(Zd, Z64, data[:, 2]) <= TOL_F64, p


@pytest.mark.parametrize("p", [0.01, 40.0, 64.0])
def test_extreme_powers(idw, p):
    """p near 0 (weights nearly equal: the sums' compensation carries the
    result) and p = 40, 64 (FP32 weights overflow or flush for most pairs, so
    most queries take the FP64 recompute; Z tends to the nearest value)."""
    prob = synthetic.uniform_problem(2000, 600, seed=95, exact_hits=3)
    data, q = prob["data"], prob["queries"]
    Z64, _ = oracle.idw(data, q, p)
    Z, s0, hit = _run(idw, data, q, p)
    assert _rel_err(Z, Z64, data[:, 2]) <= TOL_F32C, p
    Zd, _, _ = _run(idw, data, q, p, "f64")
    assert _rel_err(Zd, Z64, data[:, 2]) <= TOL_F64, p


def test_clustered_config_sampled(idw):
    prob = synthetic.config_clustered(n=65536, grid=256)
    data, q = prob["data"], prob["queries"]
    for p in prob["p_values"]:
        Z64, _ = oracle.idw(data, q, p)
        Z, _, _ = _run(idw, data, q, p, "f32c")
        assert _rel_err(Z, Z64, data[:, 2]) <= TOL_F32C, p


def test_single_point_and_empty_queries(idw):
    data = np.array([[0.3, 0.6, -1.25]], np.float32)
    q = np.random.default_rng(0).random((5000, 2)).astype(np.float32)
    Z, _, _ = _run(idw, data, q, 2.0)
    # Z = fl(w z) / w: within the FP32 form's bound of z (not bit-exact).
    assert np.max(np.abs(Z.astype(np.float64) + 1.25)) <= 1.25 * TOL_F32C
    out = idw.interpolate(_dev(data), torch.empty(0, 2, device="cuda"), 2.0)
    assert out.numel() == 0


def test_near_coincident_takes_fp64_path(idw):
    rng = np.random.default_rng(3)
    data = np.empty((3000, 3), np.float32)
    data[:, :2] = rng.random((3000, 2))
    data[:, 2] = rng.standard_normal(3000)
    q = rng.random((600, 2)).astype(np.float32)
    # Distinct points 2e-30 apart: d^2 = 4e-60 is below FP32's range, so the
    # FP32 sums overflow and the query is recomputed in FP64.
    data[5, :2] = (1e-30, 0.5)
    q[10] = (3e-30, 0.5)
    # Duplicate locations with distinct z: the lowest index wins.
    data[100, :2] = data[50, :2]
    q[12] = data[50, :2]
    Z64, hit64 = oracle.idw(data, q, 2.0)
    Z, s0, hit = _run(idw, data, q, 2.0)
    assert hit[12] == 50 and hit64[12] == 50 and Z[12] == data[50, 2]
    assert hit[10] == -2 and hit64[10] == -1
    assert _rel_err(Z, Z64, data[:, 2]) <= TOL_F32C


def test_fp32_overflow_takes_fp64_path(idw):
    rng = np.random.default_rng(4)
    data = np.empty((2000, 3), np.float32)
    data[:, :2] = rng.random((2000, 2))
    data[:, 2] = rng.standard_normal(2000)
    data[7, 2] = np.float32(3e38)       # w * z overflows FP32 near point 7
    q = rng.random((500, 2)).astype(np.float32)
    q[11] = data[7, :2] + np.float32(1e-4)
    q[12] = data[7, :2] - np.float32(3e-5)
    Z64, _ = oracle.idw(data, q, 2.0)
    Z, _, hit = _run(idw, data, q, 2.0)
    assert np.count_nonzero(hit == -2) > 0
    rel = np.abs(Z.astype(np.float64) - Z64) / np.maximum(np.abs(Z64), 1e-30)
    assert np.all(np.isfinite(Z)) and np.max(rel) <= 1e-6


@pytest.mark.parametrize("offset,scale", [(0.0, 1e-20), (1e6, 1000.0), (-3e4, 1e-3),
                                          (0.0, 1e12), (5e-3, 1e-6)])
def test_coordinate_ranges(idw, offset, scale):
    """Eq. 1 depends only on distance ratios; the library rescales by a power
    of two internally, so any coordinate range gives the FP32 bound."""
    prob = synthetic.uniform_problem(4000, 3000, seed=17)
    data = prob["data"].astype(np.float64)
    q = prob["queries"].astype(np.float64)
    data[:, :2] = data[:, :2] * scale + offset
    q = q * scale + offset
    data = data.astype(np.float32)
    q = q.astype(np.float32)
    for p in (2.0, 2.5):
        Z64, hit64 = oracle.idw(data, q, p)
        Z, _, hit = _run(idw, data, q, p)
        assert np.array_equal(hit >= 0, hit64 >= 0)
        assert _rel_err(Z, Z64, data[:, 2]) <= TOL_F32C, (offset, scale, p)
        assert np.count_nonzero(hit == -2) <= 3


def test_permutation_and_constant_field(idw):
    prob = synthetic.uniform_problem(5000, 3000, seed=11)
    data, q = prob["data"], prob["queries"]
    perm = np.random.default_rng(2).permutation(5000)
    Za, _, _ = _run(idw, data, q, 2.0)
    Zb, _, _ = _run(idw, data[perm], q, 2.0)
    assert np.max(np.abs(Za - Zb)) <= 2 * TOL_F32C * np.abs(data[:, 2]).max()
    const = data.copy()
    const[:, 2] = np.float32(0.75)
    Zc, _, _ = _run(idw, const, q, 2.0)
    assert np.max(np.abs(Zc.astype(np.float64) - 0.75)) <= 0.75 * TOL_F32C


def test_host_entry_matches_device_entry(idw):
    prob = synthetic.uniform_problem(9000, 5000, seed=12)
    d = torch.from_numpy(prob["data"]).pin_memory()
    q = torch.from_numpy(prob["queries"]).pin_memory()
    Zh = idw.interpolate_host(d, q, 2.0)
    Zd = idw.interpolate(d.cuda(), q.cuda(), 2.0).cpu()
    assert torch.equal(Zh, Zd)


def test_deterministic_repeat(idw):
    prob = synthetic.uniform_problem(30000, 20000, seed=13)
    d, q = _dev(prob["data"]), _dev(prob["queries"])
    a = idw.interpolate(d, q, 2.0).clone()
    b = idw.interpolate(d, q, 2.0)
    assert torch.equal(a, b)


def test_argument_errors(idw):
    d = _dev(np.zeros((10, 3), np.float32))
    q = _dev(np.zeros((4, 2), np.float32))
    h = idw.get_handle()
    lib = h.lib
    out = torch.empty(4, device="cuda")
    s = None
    assert lib.idw_interpolate(h.ptr, d.data_ptr(), 10, q.data_ptr(), 4, 0.0, 0, out.data_ptr(), s) == 1
    assert lib.idw_interpolate(h.ptr, d.data_ptr(), 10, q.data_ptr(), 4, float("nan"), 0,
                               out.data_ptr(), s) == 1
    assert lib.idw_interpolate(h.ptr, None, 10, q.data_ptr(), 4, 2.0, 0, out.data_ptr(), s) == 1
    assert lib.idw_interpolate(h.ptr, d.data_ptr(), 0, q.data_ptr(), 4, 2.0, 0, out.data_ptr(), s) == 1
    assert lib.idw_interpolate(h.ptr, d.data_ptr() + 2, 10, q.data_ptr(), 4, 2.0, 0,
                               out.data_ptr(), s) == 2
    assert lib.idw_interpolate(h.ptr, d.data_ptr(), 10, q.data_ptr(), 4, 2.0, 7,
                               out.data_ptr(), s) == 1
    # m = 0 is a no-op that succeeds, even with null pointers.
    assert lib.idw_interpolate(h.ptr, None, 10, None, 0, 2.0, 0, None, s) == 0
    idw.sync_status()


def test_full_size_sampled_against_oracle(idw):
    """N = M = 2^20 in the benchmark's launch configuration; 1536 sampled queries."""
    prob = synthetic.config_scale(1 << 20)
    data, q = prob["data"], prob["queries"]
    Z = idw.interpolate(_dev(data), _dev(q), 2.0).cpu().numpy()
    idx = np.random.default_rng(5).choice(q.shape[0], 1536, replace=False)
    Z64, _ = oracle.idw(data, q[idx], 2.0)
    assert _rel_err(Z[idx], Z64, data[:, 2]) <= TOL_F32C
    # FP64 plain on a smaller sample (it is ~100x slower on this GPU).
    qs = q[idx[:256]]
    Zd = idw.interpolate(_dev(data, torch.float64), _dev(qs, torch.float64), 2.0, "f64").cpu().numpy()
    assert _rel_err(Zd, Z64[:256], data[:, 2]) <= TOL_F64
