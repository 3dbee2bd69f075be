"""Pins for the FP64 oracle: each check is fixed by the mathematics of Eq. 1
(Sec. 2.1), not by re-running the oracle's own formula.

* exact rational arithmetic (fp32 inputs are dyadic rationals, and for even p
  every weight is rational, so Eq. 1 has an exact value);
* 50-digit mpmath evaluation for non-integer p;
* closed forms (N = 1, two points, symmetric squares, bisector);
* invariants (constant field, convex hull of z, permutation, dyadic
  translation and scaling, nearest-neighbour limit as p grows, exact hits);
* central finite differences of the forward pass for the analytic gradient.

A dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of these.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic

mpmath = pytest.importorskip("mpmath")


def _tiny(seed, n, m, lo=0.0, hi=1.0):
    rng = np.random.default_rng(seed)
    data = np.empty((n, 3), np.float32)
    data[:, :2] = rng.uniform(lo, hi, (n, 2)).astype(np.float32)
    data[:, 2] = rng.standard_normal(n).astype(np.float32)
    q = rng.uniform(lo, hi, (m, 2)).astype(np.float32)
    return data, q


def _exact_z(data, q, p_even):
    """Exact rational Z of Eq. 1 for an even integer power."""
    out = []
    for qx, qy in q:
        fx, fy = Fraction(float(qx)), Fraction(float(qy))
        s0 = Fraction(0)
        s1 = Fraction(0)
        hit = None
        for i, (x, y, z) in enumerate(data):
            d2 = (fx - Fraction(float(x))) ** 2 + (fy - Fraction(float(y))) ** 2
            if d2 == 0:
                hit = i
                break
            w = 1 / d2 ** (p_even // 2)
            s0 += w
            s1 += w * Fraction(float(z))
        out.append((float(data[hit, 2]), hit) if hit is not None else (float(s1 / s0), -1))
    return out


@pytest.mark.parametrize("p", [2, 4, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_rational_even_p(p, seed):
    data, q = _tiny(seed, 23, 17)
    Z, hit = oracle.idw(data, q, float(p))
    zmax = np.abs(data[:, 2]).max()
    for j, (ze, he) in enumerate(_exact_z(data, q, p)):
        assert hit[j] == he
        assert abs(Z[j] - ze) <= 4e-16 * zmax, (j, Z[j], ze)


def test_exact_rational_with_hits_and_duplicates():
    data, q = _tiny(7, 19, 12)
    data[11, :2] = data[4, :2]          # duplicate location, different z
    q[3] = data[4, :2]                  # hit on the duplicated location
    q[8] = data[18, :2]
    Z, hit = oracle.idw(data, q, 2.0)
    exact = _exact_z(data, q, 2)
    assert hit[3] == 4 and Z[3] == np.float64(data[4, 2])
    assert hit[8] == 18 and Z[8] == np.float64(data[18, 2])
    for j, (ze, he) in enumerate(exact):
        assert hit[j] == he
        assert abs(Z[j] - ze) <= 4e-16 * np.abs(data[:, 2]).max()


@pytest.mark.parametrize("p", [0.5, 1.5, 2.5, 3.5, 7.25])
def test_mpmath_general_p(p):
    data, q = _tiny(11, 21, 13)
    Z, hit = oracle.idw(data, q, p)
    mpmath.mp.dps = 50
    for j, (qx, qy) in enumerate(q):
        s0 = mpmath.mpf(0)
        s1 = mpmath.mpf(0)
        for x, y, z in data:
            d2 = (mpmath.mpf(float(qx)) - float(x)) ** 2 + (mpmath.mpf(float(qy)) - float(y)) ** 2
            w = d2 ** (-mpmath.mpf(p) / 2)
            s0 += w
            s1 += w * float(z)
        ref = float(s1 / s0)
        assert hit[j] == -1
        assert abs(Z[j] - ref) <= 1e-15 * np.abs(data[:, 2]).max(), (p, j, Z[j], ref)


def test_single_point_gives_its_value_everywhere():
    data = np.array([[0.25, 0.75, -3.5]], np.float32)
    q = np.random.default_rng(0).random((50, 2)).astype(np.float32)
    for p in (0.3, 2.0, 5.0):
        Z, hit = oracle.idw(data, q, p)
        assert np.all(Z == -3.5)


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0, 4.5])
def test_two_points_closed_form(p):
    # Points on the x axis, query between and beyond them.
    data = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, -2.0]], np.float32)
    qs = np.array([[0.25, 0.0], [0.5, 0.0], [0.75, 0.0], [2.0, 0.0], [0.5, 0.5]], np.float32)
    Z, _ = oracle.idw(data, qs, p)
    for j, (qx, qy) in enumerate(qs.astype(np.float64)):
        a = np.hypot(qx - 0.0, qy)      # distance to point 1
        b = np.hypot(qx - 1.0, qy)      # distance to point 2
        ref = (1.0 * b ** p + (-2.0) * a ** p) / (a ** p + b ** p)
        assert abs(Z[j] - ref) <= 1e-15, (p, j, Z[j], ref)


def test_square_centre_is_mean_and_bisector():
    # Four corners of a square around (0.5, 0.5): all equidistant from the centre.
    data = np.array([[0.25, 0.25, 1.0], [0.75, 0.25, 2.0], [0.25, 0.75, 4.0],
                     [0.75, 0.75, 8.0]], np.float32)
    for p in (0.7, 2.0, 3.5):
        Z, _ = oracle.idw(data, np.array([[0.5, 0.5]], np.float32), p)
        assert Z[0] == pytest.approx(15.0 / 4.0, abs=1e-15)
    # On the perpendicular bisector of two points the result is their mean.
    two = np.array([[0.0, 0.0, 3.0], [1.0, 0.0, 5.0]], np.float32)
    qs = np.array([[0.5, y] for y in (-2.0, 0.1, 0.5, 7.0)], np.float32)
    Z, _ = oracle.idw(two, qs, 2.0)
    assert np.all(np.abs(Z - 4.0) <= 1e-15)


def test_constant_field_is_reproduced():
    data, q = _tiny(3, 300, 200)
    data[:, 2] = np.float32(0.3)
    for p in (1.5, 2.0, 3.5):
        Z, _ = oracle.idw(data, q, p)
        assert np.all(np.abs(Z - np.float64(np.float32(0.3))) <= 2 * np.spacing(0.3))


def test_result_inside_range_of_z():
    prob = synthetic.uniform_problem(2000, 500, seed=5)
    for p in (0.5, 2.0, 6.0):
        Z, _ = oracle.idw(prob["data"], prob["queries"], p)
        zmin, zmax = prob["data"][:, 2].min(), prob["data"][:, 2].max()
        assert np.all(Z >= zmin - 1e-15) and np.all(Z <= zmax + 1e-15)


def test_permutation_invariance():
    prob = synthetic.uniform_problem(1500, 300, seed=6)
    perm = np.random.default_rng(1).permutation(1500)
    for p in (2.0, 3.5):
        Za, _ = oracle.idw(prob["data"], prob["queries"], p)
        Zb, _ = oracle.idw(prob["data"][perm], prob["queries"], p)
        assert np.max(np.abs(Za - Zb)) <= 1e-15


def test_dyadic_translation_and_scaling_are_exact():
    prob = synthetic.uniform_problem(800, 200, seed=8)
    d64 = prob["data"].astype(np.float64)
    q64 = prob["queries"].astype(np.float64)
    for p in (2.0, 3.5):
        Z0, _ = oracle.idw(d64, q64, p)
        # Translation by 0.5 and scaling by 2^5 are exact in FP64 on fp32
        # inputs, and Eq. 1 depends only on distance ratios.
        dt = d64.copy(); dt[:, :2] += 0.5
        Zt, _ = oracle.idw(dt, q64 + 0.5, p)
        ds = d64.copy(); ds[:, :2] *= 32.0
        Zs, _ = oracle.idw(ds, q64 * 32.0, p)
        assert np.array_equal(Z0, Zt)
        assert np.array_equal(Z0, Zs)
        # Non-dyadic scaling re-rounds the inputs: agreement to rounding level.
        dn = d64.copy(); dn[:, :2] *= 3.7
        Zn, _ = oracle.idw(dn, q64 * 3.7, p)
        assert np.max(np.abs(Z0 - Zn)) <= 1e-12


def test_nearest_neighbour_limit_large_p():
    data, q = _tiny(12, 200, 60)
    d = data[:, :2].astype(np.float64)
    for p in (64.0, 300.0):
        Z, _ = oracle.idw(data, q, p)
        for j, (qx, qy) in enumerate(q.astype(np.float64)):
            dist = np.hypot(d[:, 0] - qx, d[:, 1] - qy)
            k = np.argmin(dist)
            ratio = (dist[k] / np.delete(dist, k)) ** p
            bound = np.sum(ratio * np.abs(np.delete(data[:, 2], k) - data[k, 2])) + 1e-15
            assert abs(Z[j] - data[k, 2]) <= bound


def test_exact_hit_rule_reproduces_data_values():
    prob = synthetic.config_exact_hits(n=4096, m=1024, hits=64)
    Z, hit = oracle.idw(prob["data"], prob["queries"], 2.0)
    assert np.array_equal(np.sort(np.nonzero(hit >= 0)[0]), prob["hit_q"])
    assert np.array_equal(hit[prob["hit_q"]], prob["hit_d"])
    assert np.array_equal(Z[prob["hit_q"]], prob["data"][prob["hit_d"], 2].astype(np.float64))


def test_shared_single_coordinate_is_not_a_hit():
    # Queries that share exactly one coordinate with a data point are ordinary
    # points of Eq. 1; only both coordinates equal make d = 0.
    data = np.array([[0.5, 0.125, 7.0], [0.25, 0.875, 1.0], [0.75, 0.5, -2.0]], np.float32)
    q = np.array([[0.5, 0.375], [0.625, 0.875], [0.75, 0.5]], np.float32)
    Z, hit = oracle.idw(data, q, 2.0)
    exact = _exact_z(data, q, 2)
    assert list(hit) == [-1, -1, 2]
    for j, (ze, he) in enumerate(exact):
        assert abs(Z[j] - ze) <= 4e-16 * 7.0


def test_negative_zero_counts_as_coincident():
    data = np.array([[0.0, 0.5, 2.0], [1.0, 1.0, 9.0]], np.float32)
    q = np.array([[-0.0, 0.5]], np.float32)
    Z, hit = oracle.idw(data, q, 2.0)
    assert hit[0] == 0 and Z[0] == 2.0


def test_rejects_bad_p():
    data, q = _tiny(0, 4, 2)
    for p in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(ValueError):
            oracle.idw(data, q, p)


# ---------------------------------------------------------------- gradients

def _loss(data, q, p, g):
    Z, _ = oracle.idw(data, q, p)
    return float(np.dot(g, Z))


@pytest.mark.parametrize("p", [2.0, 2.5])
def test_gradient_matches_central_differences(p):
    rng = np.random.default_rng(21)
    n = m = 96
    data = np.empty((n, 3), np.float64)
    data[:, :2] = synthetic.separated_xy(rng, n, 2e-3)
    data[:, 2] = rng.standard_normal(n)
    q = synthetic.separated_xy(rng, m, 2e-3).astype(np.float64) + 1e-3 * rng.random((m, 2))
    g = rng.standard_normal(m)
    G = oracle.idw_grad(data, q, p, g)
    eps = 1e-6

    def fd(arr, idx):
        a = arr.copy(); a[idx] += eps
        b = arr.copy(); b[idx] -= eps
        if arr is data:
            return (_loss(a, q, p, g) - _loss(b, q, p, g)) / (2 * eps)
        return (_loss(data, a, p, g) - _loss(data, b, p, g)) / (2 * eps)

    scale_d = max(np.abs(G["grad_xy"]).max(), np.abs(G["grad_z"]).max())
    for i in rng.choice(n, 12, replace=False):
        assert abs(fd(data, (i, 2)) - G["grad_z"][i]) <= 1e-6 * scale_d
        assert abs(fd(data, (i, 0)) - G["grad_xy"][i, 0]) <= 1e-6 * scale_d
        assert abs(fd(data, (i, 1)) - G["grad_xy"][i, 1]) <= 1e-6 * scale_d
    scale_q = np.abs(G["grad_q"]).max()
    for j in rng.choice(m, 12, replace=False):
        assert abs(fd(q, (j, 0)) - G["grad_q"][j, 0]) <= 1e-6 * scale_q
        assert abs(fd(q, (j, 1)) - G["grad_q"][j, 1]) <= 1e-6 * scale_q
    dp = (_loss(data, q, p + eps, g) - _loss(data, q, p - eps, g)) / (2 * eps)
    assert abs(dp - G["grad_p"]) <= 1e-6 * max(1.0, abs(dp))
    assert np.allclose(G["Z"], oracle.idw(data, q, p)[0], rtol=0, atol=0)


def test_gradient_z_is_partition_of_unity():
    # sum_i dZ/dz_i = 1 for every query (weights normalised by S0), so with
    # g = 1 the data-side z-gradient sums to m.
    prob = synthetic.uniform_problem(300, 120, seed=31)
    G = oracle.idw_grad(prob["data"], prob["queries"], 2.0, np.ones(120))
    assert abs(G["grad_z"].sum() - 120.0) <= 1e-11
    # Translating every point and query together changes nothing, so the
    # coordinate gradients cancel: sum_i dZ/dx_i + dZ/dq = 0.
    assert np.abs(G["grad_xy"].sum(0) + G["grad_q"].sum(0)).max() <= 1e-9 * np.abs(G["grad_q"]).max()


def test_gradient_at_exact_hit():
    data = np.array([[0.1, 0.2, 1.5], [0.7, 0.4, -1.0], [0.3, 0.9, 2.0]], np.float64)
    q = np.array([[0.7, 0.4]], np.float64)
    G = oracle.idw_grad(data, q, 2.0, np.array([3.0]))
    assert np.array_equal(G["grad_z"], [0.0, 3.0, 0.0])
    assert np.all(G["grad_xy"] == 0) and np.all(G["grad_q"] == 0) and G["grad_p"] == 0


# ------------------------------------------------------- local variant

def _round_f32(frac):
    """Round an exact Fraction to the nearest float32 (ties to even)."""
    d = np.float32(float(frac))
    best = None
    for c in (np.nextafter(d, np.float32(-np.inf)), d, np.nextafter(d, np.float32(np.inf))):
        if not np.isfinite(c):
            continue
        err = abs(Fraction(float(c)) - frac)
        key = (err, int(np.frombuffer(np.float32(c).tobytes(), np.uint32)[0]) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


def _local_exact(data, q, radius, p_even=2):
    """Exact Z of Eq. 1 over the members decided by the FP32 test
    fmaf(dy, dy, fl32(dx dx)) < fl32(R^2), emulated without rounding slips."""
    r2f = np.float32(radius * radius)
    out = []
    for qx, qy in q.astype(np.float32):
        hit = None
        members = []
        for i, (x, y, z) in enumerate(data.astype(np.float32)):
            if x == qx and y == qy:
                hit = i
                break
            dx = np.float32(qx - x)
            dy = np.float32(qy - y)
            dxx = np.float32(dx * dx)
            d2 = _round_f32(Fraction(float(dy)) ** 2 + Fraction(float(dxx)))
            if d2 < r2f:
                members.append(i)
        if hit is not None:
            out.append((float(data[hit, 2]), hit, -1))
            continue
        if not members:
            out.append((float("nan"), -1, 0))
            continue
        s0 = Fraction(0)
        s1 = Fraction(0)
        for i in members:
            d2 = (Fraction(float(qx)) - Fraction(float(data[i, 0]))) ** 2 + \
                 (Fraction(float(qy)) - Fraction(float(data[i, 1]))) ** 2
            w = 1 / d2 ** (p_even // 2)
            s0 += w
            s1 += w * Fraction(float(data[i, 2]))
        out.append((float(s1 / s0), -1, len(members)))
    return out


@pytest.mark.parametrize("radius", [0.05, 0.2, 0.6])
def test_local_exact_rational(radius):
    data, q = _tiny(31, 60, 25)
    q[4] = data[17, :2]
    Z, hit, count = oracle.idw_local(data, q, 2.0, radius)
    for j, (ze, he, ce) in enumerate(_local_exact(data, q, radius)):
        assert hit[j] == he and count[j] == ce, (j, hit[j], he, count[j], ce)
        if np.isnan(ze):
            assert np.isnan(Z[j])
        else:
            assert abs(Z[j] - ze) <= 4e-16 * np.abs(data[:, 2]).max()


def test_local_membership_at_the_boundary():
    # Points placed so that d^2 sits next to R^2: the FP32 test decides.
    data = np.array([[0.0, 0.0, 1.0], [0.3, 0.4, 2.0], [0.30000001, 0.4, 3.0],
                     [0.6, 0.8, 4.0], [0.5, 0.0, 5.0]], np.float32)
    # The last query is exactly 0.5 from (0.5, 0): d^2 = R^2 = 0.25 exactly,
    # so the strict test excludes that point at R = 0.5.
    q = np.array([[0.0, 0.0001], [0.0, 0.0], [1.0, 0.0]], np.float32)
    for radius in (0.5, 0.49999999, 0.5000001, 1.0):
        Z, hit, count = oracle.idw_local(data, q, 2.0, radius)
        for j, (ze, he, ce) in enumerate(_local_exact(data, q, radius)):
            assert hit[j] == he and count[j] == ce, (radius, j, count[j], ce)
        if radius == 0.5:
            assert count[2] == 0 and np.isnan(Z[2])


def test_local_with_huge_radius_is_the_global_form():
    prob = synthetic.uniform_problem(700, 300, seed=33, exact_hits=4)
    for p in (2.0, 3.5):
        Zg, hg = oracle.idw(prob["data"], prob["queries"], p)
        Zl, hl, cl = oracle.idw_local(prob["data"], prob["queries"], p, 1e30)
        assert np.array_equal(Zg, Zl) and np.array_equal(hg, hl)
        assert np.all(cl[hl < 0] == 700)


def test_local_no_member_is_nan():
    data = np.array([[0.0, 0.0, 1.0], [1.0, 1.0, 2.0]], np.float32)
    q = np.array([[0.5, 0.5], [0.01, 0.0]], np.float32)
    Z, hit, count = oracle.idw_local(data, q, 2.0, 0.1)
    assert np.isnan(Z[0]) and count[0] == 0
    assert Z[1] == 1.0 and count[1] == 1


def test_local_membership_is_decided_in_fp32():
    """Find points where the FP32 test and an exact test disagree; the oracle
    must follow the FP32 decision (a GPU makes it the same way)."""
    rng = np.random.default_rng(35)
    radius = 0.3
    r2f = np.float32(radius * radius)
    q = np.array([[0.5, 0.5]], np.float32)
    found = []
    for _ in range(20000):
        ang = rng.uniform(0, 2 * np.pi)
        rad = radius * (1 + rng.uniform(-3e-7, 3e-7))
        pt = np.array([0.5 + rad * np.cos(ang), 0.5 + rad * np.sin(ang)], np.float32)
        dx = np.float32(q[0, 0] - pt[0])
        dy = np.float32(q[0, 1] - pt[1])
        d2f = _round_f32(Fraction(float(dy)) ** 2 + Fraction(float(np.float32(dx * dx))))
        exact = (Fraction(float(q[0, 0])) - Fraction(float(pt[0]))) ** 2 + \
                (Fraction(float(q[0, 1])) - Fraction(float(pt[1]))) ** 2
        if (d2f < r2f) != (exact < Fraction(float(r2f))):
            found.append((pt, bool(d2f < r2f)))
        if len(found) >= 4:
            break
    assert found, "no disagreeing point found"
    for pt, member in found:
        data = np.array([[pt[0], pt[1], 7.0], [0.9, 0.9, 1.0]], np.float32)
        Z, hit, count = oracle.idw_local(data, q, 2.0, radius)
        assert count[0] == (1 if member else 0)


# ---------------------------------------------------------------- k-NN form

def _fp32_key(qx, qy, x, y):
    """FP32 d^2 = fmaf(dy, dy, fl32(dx dx)), emulated exactly."""
    dx = np.float32(np.float32(qx) - np.float32(x))
    dy = np.float32(np.float32(qy) - np.float32(y))
    dxx = np.float32(dx * dx)
    return _round_f32(Fraction(float(dy)) ** 2 + Fraction(float(dxx)))


def _knn_exact(data, q, k, p_even=2):
    """Exact selection by the key (FP32 d^2, index) and exact rational Z."""
    out = []
    for qx, qy in q.astype(np.float32):
        fin = [i for i in range(data.shape[0])
               if np.isfinite(data[i, 0]) and np.isfinite(data[i, 1])]
        if not (np.isfinite(qx) and np.isfinite(qy)):
            out.append((float("nan"), -1, [], 0))
            continue
        hit = next((i for i in fin if data[i, 0] == qx and data[i, 1] == qy), -1)
        keys = sorted((float(_fp32_key(qx, qy, data[i, 0], data[i, 1])), i) for i in fin)
        sel = [i for _, i in keys[:k]]
        if hit >= 0:
            out.append((float(data[hit, 2]), hit, sel, len(sel)))
            continue
        s0 = Fraction(0)
        s1 = Fraction(0)
        for i in sel:
            d2 = (Fraction(float(qx)) - Fraction(float(data[i, 0]))) ** 2 + \
                 (Fraction(float(qy)) - Fraction(float(data[i, 1]))) ** 2
            w = 1 / d2 ** (p_even // 2)
            s0 += w
            s1 += w * Fraction(float(data[i, 2]))
        out.append((float(s1 / s0) if sel else float("nan"), -1, sel, len(sel)))
    return out


def _check_knn(data, q, k, p_even=2):
    r = oracle.idw_knn(data, q, float(p_even), k)
    zmax = np.nanmax(np.abs(data[:, 2]))
    for j, (ze, he, sel, ce) in enumerate(_knn_exact(data, q, k, p_even)):
        assert r["hit"][j] == he and r["count"][j] == ce, (j, r["hit"][j], he, r["count"][j], ce)
        got = [int(i) for i in r["nbr"][j] if i >= 0]
        assert got == sel, (j, got, sel)
        assert np.all(r["nbr"][j][len(sel):] == -1)
        if np.isnan(ze):
            assert np.isnan(r["Z"][j])
        else:
            assert abs(r["Z"][j] - ze) <= 4e-16 * zmax, (j, r["Z"][j], ze)
    return r


@pytest.mark.parametrize("k", [1, 3, 7, 16])
def test_knn_exact_rational(k):
    data, q = _tiny(41, 40, 20)
    q[3] = data[11, :2]  # an exact hit
    for p_even in (2, 4):
        _check_knn(data, q, k, p_even)


def test_knn_ties_go_to_the_lower_index():
    # Four points exactly 1/4 from the query (FP32 keys equal), one nearer,
    # one farther; indices arranged so that the tie order is visible.
    data = np.array([[0.75, 0.5, 1.0], [0.5, 0.25, 2.0], [0.5, 0.5625, 3.0],
                     [0.25, 0.5, 4.0], [0.5, 0.75, 5.0], [0.9, 0.9, 6.0]], np.float32)
    q = np.array([[0.5, 0.5]], np.float32)
    for k, sel in ((1, [2]), (2, [2, 0]), (3, [2, 0, 1]), (4, [2, 0, 1, 3]), (6, [2, 0, 1, 3, 4, 5])):
        r = _check_knn(data, q, k)
        assert [int(i) for i in r["nbr"][0] if i >= 0] == sel
    r = oracle.idw_knn(data, q, 2.0, 2)
    # Z over {2, 0} at distances 1/16 and 1/4: weights 256 and 16.
    assert r["Z"][0] == (256 * 3.0 + 16 * 1.0) / (256 + 16)
    assert r["kd2"][0] == np.float32(0.0625)


def test_knn_with_k_at_least_n_is_the_global_form():
    prob = synthetic.uniform_problem(300, 120, seed=43, exact_hits=3)
    for p in (2.0, 3.5):
        Zg, hg = oracle.idw(prob["data"], prob["queries"], p)
        for k in (300, 305):
            r = oracle.idw_knn(prob["data"], prob["queries"], p, k)
            assert np.array_equal(r["hit"], hg)
            assert np.all(r["count"] == 300)
            assert np.max(np.abs(r["Z"] - Zg)) <= 1e-15 * np.abs(prob["data"][:, 2]).max()


def test_knn_k1_is_the_nearest_neighbour():
    data, q = _tiny(44, 500, 200)
    r = oracle.idw_knn(data, q, 2.0, 1)
    for j in range(q.shape[0]):
        keys = [(float(_fp32_key(q[j, 0], q[j, 1], x, y)), i) for i, (x, y, _) in enumerate(data)]
        i = min(keys)[1]
        assert r["nbr"][j, 0] == i and r["Z"][j] == np.float64(data[i, 2])


def test_knn_selection_is_decided_in_fp32():
    """Find two points whose FP32 keys rank differently from their exact
    distances; the oracle must follow the FP32 key (a GPU ranks the same)."""
    rng = np.random.default_rng(45)
    q = np.array([[0.5, 0.5]], np.float32)
    found = 0
    for _ in range(40000):
        r0 = 0.3 * (1 + rng.uniform(-2e-7, 2e-7))
        a0, a1 = rng.uniform(0, 2 * np.pi, 2)
        pa = np.array([0.5 + r0 * np.cos(a0), 0.5 + r0 * np.sin(a0)], np.float32)
        pb = np.array([0.5 + 0.3 * np.cos(a1), 0.5 + 0.3 * np.sin(a1)], np.float32)
        ka, kb = _fp32_key(q[0, 0], q[0, 1], *pa), _fp32_key(q[0, 0], q[0, 1], *pb)
        ea = (Fraction(float(q[0, 0])) - Fraction(float(pa[0]))) ** 2 + \
             (Fraction(float(q[0, 1])) - Fraction(float(pa[1]))) ** 2
        eb = (Fraction(float(q[0, 0])) - Fraction(float(pb[0]))) ** 2 + \
             (Fraction(float(q[0, 1])) - Fraction(float(pb[1]))) ** 2
        fp32_first = (float(ka), 0) < (float(kb), 1)
        if ea == eb or fp32_first == (ea < eb):
            continue
        # pa at index 0, pb at index 1: the FP32 key order (ties: index 0
        # first) disagrees with the exact order.
        data = np.array([[pa[0], pa[1], 1.0], [pb[0], pb[1], 2.0]], np.float32)
        r = oracle.idw_knn(data, q, 2.0, 1)
        want = 0 if fp32_first else 1
        assert r["nbr"][0, 0] == want
        found += 1
        if found >= 4:
            break
    assert found, "no disagreeing pair found"


def test_knn_non_finite_inputs():
    data = np.array([[np.nan, 0.5, 9.0], [0.5, np.inf, 9.0], [0.1, 0.1, 1.0],
                     [0.9, 0.9, 2.0], [0.2, 0.2, 3.0]], np.float32)
    q = np.array([[0.15, 0.15], [np.nan, 0.5], [0.5, np.inf]], np.float32)
    r = _check_knn(data, q, 4)
    assert r["count"][0] == 3 and np.all(r["count"][1:] == 0)
    assert np.isnan(r["Z"][1]) and np.isnan(r["Z"][2]) and np.isnan(r["kd2"][1])


def test_local_ignores_non_finite_points():
    # A data point with a non-finite coordinate is neither a hit nor a
    # member, even for a query with the same (non-finite) coordinates.
    data = np.array([[np.inf, 0.5, 9.0], [np.nan, 0.2, 8.0], [0.1, 0.1, 1.0]], np.float32)
    q = np.array([[np.inf, 0.5], [0.1, 0.12]], np.float32)
    Z, hit, count = oracle.idw_local(data, q, 2.0, 0.5)
    assert np.isnan(Z[0]) and hit[0] == -1 and count[0] == 0
    assert Z[1] == 1.0 and count[1] == 1


# ------------------------------------------------- local-form gradients

def _local_loss(data, q, p, radius, g, ok):
    Z, _, _ = oracle.idw_local(data, q, p, radius)
    return float(np.dot(g[ok], Z[ok]))


@pytest.mark.parametrize("p", [2.0, 3.0])
def test_local_gradient_matches_central_differences(p):
    """Central differences of the local oracle's loss, for coordinates whose
    perturbation leaves every membership set unchanged (the sets are held
    fixed by definition), against the analytic local gradient."""
    rng = np.random.default_rng(41)
    n = m = 96
    data = np.empty((n, 3), np.float64)
    data[:, :2] = synthetic.separated_xy(rng, n, 2e-3)
    data[:, 2] = rng.standard_normal(n)
    q = synthetic.separated_xy(rng, m, 2e-3).astype(np.float64) + 1e-3 * rng.random((m, 2))
    data[:, :2] = data[:, :2].astype(np.float32)
    q = q.astype(np.float32).astype(np.float64)
    R = 0.2
    g = rng.standard_normal(m)
    _, _, c0 = oracle.idw_local(data, q, p, R)
    ok = c0 > 0
    assert 0 < ok.sum() < m or ok.all()
    G = oracle.idw_local_grad(data, q, p, R, g)
    eps = 1e-6

    def fd(arr, idx):
        a = arr.copy(); a[idx] += eps
        b = arr.copy(); b[idx] -= eps
        args = ((a, q), (b, q)) if arr is data else ((data, a), (data, b))
        for d_, q_ in args:  # the membership sets must not move
            if not np.array_equal(oracle.idw_local(d_, q_, p, R)[2], c0):
                return None
        return (_local_loss(*args[0], p, R, g, ok) - _local_loss(*args[1], p, R, g, ok)) / (2 * eps)

    scale_d = max(np.abs(G["grad_xy"]).max(), np.abs(G["grad_z"]).max())
    checked = 0
    for i in rng.choice(n, 16, replace=False):
        for col, ref in ((2, G["grad_z"][i]), (0, G["grad_xy"][i, 0]), (1, G["grad_xy"][i, 1])):
            v = fd(data, (i, col))
            if v is not None:
                assert abs(v - ref) <= 1e-6 * scale_d, (i, col, v, ref)
                checked += 1
    scale_q = np.abs(G["grad_q"]).max()
    for j in rng.choice(m, 16, replace=False):
        for col in (0, 1):
            v = fd(q, (j, col))
            if v is not None:
                assert abs(v - G["grad_q"][j, col]) <= 1e-6 * scale_q, (j, col)
                checked += 1
    assert checked >= 40
    dp = (_local_loss(data, q, p + eps, R, g, ok) - _local_loss(data, q, p - eps, R, g, ok)) / (2 * eps)
    assert abs(dp - G["grad_p"]) <= 1e-6 * max(1.0, abs(dp))
    Zl, _, _ = oracle.idw_local(data, q, p, R)
    assert np.array_equal(np.isnan(G["Z"]), np.isnan(Zl))
    assert np.array_equal(G["Z"][ok], Zl[ok])


def test_local_gradient_with_huge_radius_is_the_global_gradient():
    prob = synthetic.uniform_problem(300, 120, seed=42)
    g = np.random.default_rng(43).standard_normal(120)
    L = oracle.idw_local_grad(prob["data"], prob["queries"], 2.5, 1e30, g)
    G = oracle.idw_grad(prob["data"], prob["queries"], 2.5, g)
    for k in ("grad_z", "grad_xy", "grad_q"):
        assert np.abs(L[k] - G[k]).max() <= 1e-12 * np.abs(G[k]).max(), k
    assert abs(L["grad_p"] - G["grad_p"]) <= 1e-12 * abs(G["grad_p"])


def test_local_gradient_sums_and_translation():
    """With g = 1 the z-gradient sums to the number of queries with a value
    (each query's weights are normalised over its members), and moving every
    point and query together changes nothing, so the coordinate gradients
    cancel.  Clustered data leave some queries without members."""
    prob = synthetic.config_local(seed=44, n=600, m=400, members=6.0, clustered=True)
    data, q, R = prob["data"], prob["queries"], prob["radius"]
    G = oracle.idw_local_grad(data, q, 2.0, R, np.ones(q.shape[0]))
    Zl, _, cnt = oracle.idw_local(data, q, 2.0, R)
    assert (cnt == 0).any() and (cnt > 0).any()
    assert abs(G["grad_z"].sum() - np.isfinite(Zl).sum()) <= 1e-10
    assert np.abs(G["grad_xy"].sum(0) + G["grad_q"].sum(0)).max() <= 1e-9 * np.abs(G["grad_q"]).max()


def test_local_gradient_at_hits_and_empty_neighbourhoods():
    data = np.array([[0.1, 0.2, 1.5], [0.7, 0.4, -1.0], [0.3, 0.9, 2.0], [0.75, 0.45, 4.0]],
                    np.float64)
    q = np.array([[0.7, 0.4], [5.0, 5.0]], np.float64)  # a hit, and no member at all
    G = oracle.idw_local_grad(data, q, 2.0, 0.2, np.array([3.0, 7.0]))
    assert np.array_equal(G["grad_z"], [0.0, 3.0, 0.0, 0.0])
    assert np.all(G["grad_xy"] == 0) and np.all(G["grad_q"] == 0) and G["grad_p"] == 0
    assert G["Z"][0] == -1.0 and np.isnan(G["Z"][1])


# --------------------------------------------------- k-NN gradients

def _knn_loss(data, q, p, k, g, ok):
    return float(np.dot(g[ok], oracle.idw_knn(data, q, p, k)["Z"][ok]))


@pytest.mark.parametrize("p", [2.0, 3.0])
def test_knn_gradient_matches_central_differences(p):
    """Central differences of the k-NN oracle's loss, for coordinates whose
    perturbation changes no selection, against the analytic gradient."""
    rng = np.random.default_rng(51)
    n = m = 96
    k = 9
    data = np.empty((n, 3), np.float64)
    data[:, :2] = synthetic.separated_xy(rng, n, 2e-3).astype(np.float32)
    data[:, 2] = rng.standard_normal(n)
    q = (synthetic.separated_xy(rng, m, 2e-3) + 1e-3 * rng.random((m, 2))).astype(np.float32)
    q = q.astype(np.float64)
    g = rng.standard_normal(m)
    base = oracle.idw_knn(data, q, p, k)["nbr"]
    ok = np.ones(m, bool)
    G = oracle.idw_knn_grad(data, q, p, k, g)
    eps = 1e-6

    def fd(arr, idx):
        a = arr.copy(); a[idx] += eps
        b = arr.copy(); b[idx] -= eps
        args = ((a, q), (b, q)) if arr is data else ((data, a), (data, b))
        for d_, q_ in args:  # the selections must not move
            if not np.array_equal(oracle.idw_knn(d_, q_, p, k)["nbr"], base):
                return None
        return (_knn_loss(*args[0], p, k, g, ok) - _knn_loss(*args[1], p, k, g, ok)) / (2 * eps)

    scale_d = max(np.abs(G["grad_xy"]).max(), np.abs(G["grad_z"]).max())
    checked = 0
    for i in rng.choice(n, 16, replace=False):
        for col, ref in ((2, G["grad_z"][i]), (0, G["grad_xy"][i, 0]), (1, G["grad_xy"][i, 1])):
            v = fd(data, (i, col))
            if v is not None:
                assert abs(v - ref) <= 1e-6 * scale_d, (i, col, v, ref)
                checked += 1
    scale_q = np.abs(G["grad_q"]).max()
    for j in rng.choice(m, 16, replace=False):
        for col in (0, 1):
            v = fd(q, (j, col))
            if v is not None:
                assert abs(v - G["grad_q"][j, col]) <= 1e-6 * scale_q, (j, col)
                checked += 1
    assert checked >= 40
    dp = (_knn_loss(data, q, p + eps, k, g, ok) - _knn_loss(data, q, p - eps, k, g, ok)) / (2 * eps)
    assert abs(dp - G["grad_p"]) <= 1e-6 * max(1.0, abs(dp))


def test_knn_gradient_with_k_at_least_n_is_the_global_gradient():
    prob = synthetic.uniform_problem(300, 120, seed=52)
    g = np.random.default_rng(53).standard_normal(120)
    K = oracle.idw_knn_grad(prob["data"], prob["queries"], 2.5, 300, g)
    G = oracle.idw_grad(prob["data"], prob["queries"], 2.5, g)
    for key in ("grad_z", "grad_xy", "grad_q"):
        assert np.abs(K[key] - G[key]).max() <= 1e-12 * np.abs(G[key]).max(), key
    assert abs(K["grad_p"] - G["grad_p"]) <= 1e-12 * abs(G["grad_p"])


def test_knn_gradient_sums_and_translation():
    prob = synthetic.config_local(seed=54, n=600, m=400, clustered=True)
    data, q = prob["data"], prob["queries"]
    K = oracle.idw_knn_grad(data, q, 2.0, 12, np.ones(q.shape[0]))
    assert abs(K["grad_z"].sum() - q.shape[0]) <= 1e-10
    assert np.abs(K["grad_xy"].sum(0) + K["grad_q"].sum(0)).max() <= 1e-9 * np.abs(K["grad_q"]).max()


def test_knn_gradient_at_hits_and_empty_selections():
    data = np.array([[0.1, 0.2, 1.5], [0.7, 0.4, -1.0], [0.3, 0.9, 2.0], [0.7, 0.4, 9.0]],
                    np.float64)  # index 3 duplicates index 1
    q = np.array([[0.7, 0.4], [np.nan, 0.5], [0.5, 0.5]], np.float64)
    g = np.array([3.0, 7.0, -2.0])
    K = oracle.idw_knn_grad(data, q, 2.0, 8, g)  # k > n: all finite points
    G = oracle.idw_grad(data, q[2:], 2.0, g[2:])
    assert np.allclose(K["grad_z"] - np.array([0.0, 3.0, 0.0, 0.0]), G["grad_z"], rtol=0, atol=1e-14)
    assert np.all(K["grad_q"][:2] == 0) and np.isnan(K["Z"][1]) and K["Z"][0] == -1.0


# ------------------------------------------------- modified Shepard

def test_modified_closed_form_two_points():
    """Points at d = 1/2 and 1/4 from the query with R = 1: the bases
    1/d - 1/R are 1 and 3, so Z = (z1 + 3^p z2) / (1 + 3^p) exactly; a point
    beyond R takes no part."""
    data = np.array([[0.5, 0.0, 1.0], [0.0, 0.25, 3.0], [0.0, -1.5, 100.0]], np.float64)
    q = np.array([[0.0, 0.0]], np.float64)
    for p in (1, 2, 3):
        Z, hit, cnt = oracle.idw_modified(data, q, float(p), 1.0)
        want = Fraction(1) * 1 + Fraction(3) ** p * 3
        want = want / (1 + Fraction(3) ** p)
        # FP64 with weights scaled by the largest: within a few ulps.
        assert abs(Z[0] - float(want)) <= 4 * np.spacing(float(want))
        assert cnt[0] == 2 and hit[0] == -1


def test_modified_with_infinite_radius_is_the_global_form():
    prob = synthetic.uniform_problem(400, 150, seed=61, exact_hits=3)
    for p in (2.0, 3.5):
        Zg, _ = oracle.idw(prob["data"], prob["queries"], p)
        for R in (float("inf"), 1e30):
            Zm, _, _ = oracle.idw_modified(prob["data"], prob["queries"], p, R)
            assert np.max(np.abs(Zm - Zg)) <= 1e-12 * np.max(np.abs(prob["data"][:, 2]))


def test_modified_is_continuous_at_the_radius():
    """A point just inside R carries a weight of order (1e-7)^p, so moving it
    out of the neighbourhood changes Z by almost nothing; the standard local
    form jumps."""
    rng = np.random.default_rng(62)
    data = np.concatenate([rng.random((30, 2)) * 0.2 - 0.1, rng.standard_normal((30, 1))], 1)
    data = data.astype(np.float32).astype(np.float64)
    q = np.array([[0.0, 0.0]], np.float64)
    R = 0.25
    inside = np.array([[np.float32(R * (1 - 1e-6)), 0.0, 50.0]])
    outside = np.array([[np.float32(R * (1 + 1e-6)), 0.0, 50.0]])
    Zin, _, cin = oracle.idw_modified(np.concatenate([data, inside]), q, 2.0, R)
    Zout, _, cout = oracle.idw_modified(np.concatenate([data, outside]), q, 2.0, R)
    assert cin[0] == cout[0] + 1
    assert abs(Zin[0] - Zout[0]) <= 1e-9
    Lin, _, _ = oracle.idw_local(np.concatenate([data, inside]), q, 2.0, R)
    Lout, _, _ = oracle.idw_local(np.concatenate([data, outside]), q, 2.0, R)
    assert abs(Lin[0] - Lout[0]) > 1e-3


def test_modified_members_and_hits_are_the_radius_form_s():
    prob = synthetic.uniform_problem(2000, 500, seed=63, exact_hits=6)
    R = 0.06
    _, hm, cm = oracle.idw_modified(prob["data"], prob["queries"], 2.0, R)
    _, hl, cl = oracle.idw_local(prob["data"], prob["queries"], 2.0, R)
    assert np.array_equal(hm, hl) and np.array_equal(cm, cl)


def _modified_loss(data, q, p, radius, g, ok):
    Z, _, _ = oracle.idw_modified(data, q, p, radius)
    return float(np.dot(g[ok], Z[ok]))


@pytest.mark.parametrize("p", [2.0, 3.0])
def test_modified_gradient_matches_central_differences(p):
    """Central differences of the modified Shepard oracle's loss, for
    coordinates whose perturbation moves no membership set, against the
    analytic gradient (the weights' derivative involves 1/(t d^3))."""
    rng = np.random.default_rng(64)
    n = m = 96
    data = np.empty((n, 3), np.float64)
    data[:, :2] = synthetic.separated_xy(rng, n, 2e-3).astype(np.float32)
    data[:, 2] = rng.standard_normal(n)
    q = (synthetic.separated_xy(rng, m, 2e-3) + 1e-3 * rng.random((m, 2))).astype(np.float32)
    q = q.astype(np.float64)
    R = 0.2
    g = rng.standard_normal(m)
    _, _, c0 = oracle.idw_modified(data, q, p, R)
    ok = c0 > 0
    G = oracle.idw_modified_grad(data, q, p, R, g)
    eps = 1e-6

    def fd(arr, idx):
        a = arr.copy(); a[idx] += eps
        b = arr.copy(); b[idx] -= eps
        args = ((a, q), (b, q)) if arr is data else ((data, a), (data, b))
        for d_, q_ in args:
            if not np.array_equal(oracle.idw_modified(d_, q_, p, R)[2], c0):
                return None
        return (_modified_loss(*args[0], p, R, g, ok) -
                _modified_loss(*args[1], p, R, g, ok)) / (2 * eps)

    scale_d = max(np.abs(G["grad_xy"]).max(), np.abs(G["grad_z"]).max())
    checked = 0
    for i in rng.choice(n, 16, replace=False):
        for col, ref in ((2, G["grad_z"][i]), (0, G["grad_xy"][i, 0]), (1, G["grad_xy"][i, 1])):
            v = fd(data, (i, col))
            if v is not None:
                assert abs(v - ref) <= 1e-6 * scale_d, (i, col, v, ref)
                checked += 1
    scale_q = np.abs(G["grad_q"]).max()
    for j in rng.choice(m, 16, replace=False):
        for col in (0, 1):
            v = fd(q, (j, col))
            if v is not None:
                assert abs(v - G["grad_q"][j, col]) <= 1e-6 * scale_q, (j, col)
                checked += 1
    assert checked >= 40
    dp = (_modified_loss(data, q, p + eps, R, g, ok) -
          _modified_loss(data, q, p - eps, R, g, ok)) / (2 * eps)
    assert abs(dp - G["grad_p"]) <= 1e-6 * max(1.0, abs(dp))


def test_modified_gradient_at_infinite_radius_is_the_global_gradient():
    prob = synthetic.uniform_problem(300, 120, seed=65)
    g = np.random.default_rng(66).standard_normal(120)
    M = oracle.idw_modified_grad(prob["data"], prob["queries"], 2.5, float("inf"), g)
    G = oracle.idw_grad(prob["data"], prob["queries"], 2.5, g)
    for key in ("grad_z", "grad_xy", "grad_q"):
        assert np.abs(M[key] - G[key]).max() <= 1e-12 * np.abs(G[key]).max(), key
    assert abs(M["grad_p"] - G["grad_p"]) <= 1e-12 * abs(G["grad_p"])


def test_modified_gradient_sums_translation_and_hits():
    prob = synthetic.config_local(seed=67, n=600, m=400, members=6.0, clustered=True)
    data, q, R = prob["data"], prob["queries"].copy(), prob["radius"]
    q[5] = data[17, :2]  # an exact hit
    M = oracle.idw_modified_grad(data, q, 2.0, R, np.ones(q.shape[0]))
    Zm, hit, _ = oracle.idw_modified(data, q, 2.0, R)
    assert hit[5] >= 0 and np.all(M["grad_q"][5] == 0)
    assert abs(M["grad_z"].sum() - np.isfinite(Zm).sum()) <= 1e-10
    assert np.abs(M["grad_xy"].sum(0) + M["grad_q"].sum(0)).max() <= 1e-9 * np.abs(M["grad_q"]).max()


@pytest.mark.parametrize("p", [1.5, 2.5, 3.7])
def test_modified_mpmath_general_p(p):
    """Modified Shepard at general p against 50-digit evaluation of its
    definition over the oracle's own FP32 membership sets."""
    data, q = _tiny(11, 21, 13)
    R = 0.45
    Z, hit, cnt = oracle.idw_modified(data, q, p, R)
    _, _, cl = oracle.idw_local(data, q, p, R)
    assert np.array_equal(cnt, cl)
    mpmath.mp.dps = 50
    r2f = np.float32(R * R)
    for j, (qx, qy) in enumerate(q):
        s0 = mpmath.mpf(0)
        s1 = mpmath.mpf(0)
        for x, y, z in data:
            if not _fp32_key(qx, qy, x, y) < r2f:
                continue  # the radius form's FP32 membership test, emulated exactly
            d = mpmath.sqrt((mpmath.mpf(float(qx)) - float(x)) ** 2 +
                            (mpmath.mpf(float(qy)) - float(y)) ** 2)
            t = 1 / d - 1 / mpmath.mpf(R)
            w = t ** mpmath.mpf(p) if t > 0 else mpmath.mpf(0)
            s0 += w
            s1 += w * float(z)
        assert hit[j] == -1
        if s0 == 0:
            assert np.isnan(Z[j])
            continue
        ref = float(s1 / s0)
        assert abs(Z[j] - ref) <= 1e-14 * np.abs(data[:, 2]).max(), (p, j, Z[j], ref)
