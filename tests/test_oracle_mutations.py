"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source
(on the CPU), compiles it, swaps it in, and checks that at least one pin of
``test_oracle_pins`` fails.  The real oracle is untouched.
"""
import ctypes
import os

import pytest

import oracle
import test_oracle_pins as pins

MUTATIONS = [
    ("transposed operand in d^2", "return dx * dx + dy * dy;", "return dx * dx + dx * dy;"),
    ("sign of dy", "double dy = qy - y;\n    return", "double dy = qy + y;\n    return"),
    ("power not halved", "return pow(r, 0.5 * p);", "return pow(r, p);"),
    ("p = 2 path uses 1/d instead of 1/d^2", "        return r;\n    return pow",
     "        return sqrt(r);\n    return pow"),
    ("value index off by one", "nsum_add(&s1, w * data[3 * i + 2]);",
     "nsum_add(&s1, w * data[3 * i + 1]);"),
    ("dropped weight in S1", "nsum_add(&s1, w * data[3 * i + 2]);", "nsum_add(&s1, data[3 * i + 2]);"),
    ("exact hit on x only", "if (x == qx && y == qy)\n            return i;",
     "if (x == qx)\n            return i;"),
    ("last hit instead of first", "if (x == qx && y == qy)\n            return i;",
     "if (x == qx && y == qy && i + 1 < n && !(data[3*(i+1)] == qx && data[3*(i+1)+1] == qy))\n"
     "            return i;"),
    ("Neumaier correction sign", "a->c += (a->s - t) + x;", "a->c += (a->s - t) - x;"),
    ("query-gradient sign", "c->grad_q[2 * j] = -gj * (c->p / S0) * nsum_value(&gx);",
     "c->grad_q[2 * j] = gj * (c->p / S0) * nsum_value(&gx);"),
    ("p-gradient factor 1/2 dropped", "c->grad_p_part[j] = -gj * nsum_value(&gp) / (2.0 * S0);",
     "c->grad_p_part[j] = -gj * nsum_value(&gp) / S0;"),
    ("data-gradient uses dy for x", "nsum_add(&gx, a * dx);\n            nsum_add(&gy, a * dy);",
     "nsum_add(&gx, a * dy);\n            nsum_add(&gy, a * dy);"),
    ("z-gradient not normalised", "nsum_add(&gz, gj * w / S0);", "nsum_add(&gz, gj * w);"),
    ("local membership not strict", "    return d2 < r2f;", "    return d2 <= r2f;"),
    ("local membership in FP64", "    float d2 = fmaf(dy, dy, dxx);\n    return d2 < r2f;",
     "    float d2 = fmaf(dy, dy, dxx);\n    return (double)(qx - x) * (qx - x) + (double)(qy - y) * (qy - y) < r2f;"),
    ("local weights over all points", "            if (!local_member(qxf, qyf, (float)x, (float)y, c->r2f))\n                continue;",
     "            (void)local_member;"),
    ("local empty neighbourhood not NaN", "        if (count == 0) {\n            c->Z[j] = NAN;",
     "        if (count == 0) {\n            c->Z[j] = 0.0;"),
    ("knn ties to the higher index", "return da < db || (da == db && ia < ib);",
     "return da < db || (da == db && ia > ib);"),
    ("knn keys in FP64", "    float dxx = dx * dx;\n    return fmaf(dy, dy, dxx);",
     "    float dxx = dx * dx;\n    (void)dxx;\n    return (float)((double)(qx - x) * (qx - x) + (double)(qy - y) * (qy - y));"),
    ("knn keeps k - 1", "                if (size < k) {", "                if (size < k - 1) {"),
    ("knn hit loses precedence", "        if (hit >= 0) {\n            c->Z[j] = c->data[3 * hit + 2];",
     "        if (hit >= 0 && 0) {\n            c->Z[j] = c->data[3 * hit + 2];"),
    ("local hit on non-finite points", "            if (!isfinite(x) || !isfinite(y))\n                continue; /* ignored: neither a hit nor a member */",
     "            if (0)\n                continue;"),
    ("knn ignores non-finite check", "                if (!isfinite(x) || !isfinite(y))\n                    continue;\n                if (hit < 0",
     "                if (hit < 0"),
    ("exact-hit gradient dropped", "                if (c->hit[j] == i)\n                    nsum_add(&gz, gj);",
     "                if (c->hit[j] == i)\n                    nsum_add(&gz, 0.0);"),
    ("local query gradient over all points", "                continue; /* members only: the query-side sums */",
     "                ; /* members only: the query-side sums */"),
    ("local data gradient outside the neighbourhood",
     "                continue; /* i is outside query j's neighbourhood */",
     "                ; /* i is outside query j's neighbourhood */"),
    ("local p-gradient factor 1/2 dropped", "c->grad_p_part[j] = -0.5 * gj * nsum_value(&sp) / S0;",
     "c->grad_p_part[j] = -gj * nsum_value(&sp) / S0;"),
    ("local data-gradient sign", "const double a = gj * (c->p / S0) * (z - c->Z[j]) * w / d2;",
     "const double a = gj * (c->p / S0) * (c->Z[j] - z) * w / d2;"),
    ("knn gradient over one point fewer",
     "            for (int s = 0; s < cnt; s++) {\n                const double *x = data + 3 * sel[s];\n                const double ex",
     "            for (int s = 0; s < cnt - 1; s++) {\n                const double *x = data + 3 * sel[s];\n                const double ex"),
    ("knn query-gradient sign", "grad_q[2 * j] = -gj * (p / S0) * nsum_value(&qsx);",
     "grad_q[2 * j] = gj * (p / S0) * nsum_value(&qsx);"),
    ("knn p-gradient factor 1/2 dropped", "nsum_add(&ptot, -gj * nsum_value(&qsp) / (2.0 * S0));",
     "nsum_add(&ptot, -gj * nsum_value(&qsp) / S0);"),
    ("knn data-gradient uses dy for x", "nsum_add(&acc[3 * sel[s] + 1], f * ex);",
     "nsum_add(&acc[3 * sel[s] + 1], f * ey);"),
    ("modified weight without the radius term",
     "const double t = isinf(radius) ? 1.0 / d : (radius - d) / (radius * d);",
     "const double t = 1.0 / d;"),
    ("modified weight with R + d", "const double t = isinf(radius) ? 1.0 / d : (radius - d) / (radius * d);",
     "const double t = isinf(radius) ? 1.0 / d : (radius + d) / (radius * d);"),
    ("modified power halved", "const double w = pow(t / tmax, c->p);",
     "const double w = pow(t / tmax, 0.5 * c->p);"),
    ("modified gradient with 1/d^2 in place of 1/(t d^3)",
     "const double f = b / (tt * d * d * d); /* (z_i - Z) w_i / (t_i d_i^3) */",
     "const double f = b / (d * d); /* (z_i - Z) w_i / (t_i d_i^3) */"),
    ("modified p-gradient with the global factor -1/2",
     "nsum_add(&ptot, gj * nsum_value(&vp) / S0);",
     "nsum_add(&ptot, -0.5 * gj * nsum_value(&vp) / S0);"),
]

PINS = [
    lambda: pins.test_exact_rational_even_p(2, 0),
    lambda: pins.test_exact_rational_even_p(4, 1),
    pins.test_exact_rational_with_hits_and_duplicates,
    lambda: pins.test_mpmath_general_p(1.5),
    lambda: pins.test_two_points_closed_form(3.0),
    pins.test_square_centre_is_mean_and_bisector,
    pins.test_constant_field_is_reproduced,
    pins.test_permutation_invariance,
    pins.test_exact_hit_rule_reproduces_data_values,
    pins.test_shared_single_coordinate_is_not_a_hit,
    lambda: pins.test_gradient_matches_central_differences(2.5),
    pins.test_gradient_z_is_partition_of_unity,
    pins.test_gradient_at_exact_hit,
    lambda: pins.test_local_exact_rational(0.2),
    pins.test_local_membership_at_the_boundary,
    pins.test_local_with_huge_radius_is_the_global_form,
    pins.test_local_no_member_is_nan,
    pins.test_local_membership_is_decided_in_fp32,
    lambda: pins.test_knn_exact_rational(3),
    pins.test_knn_ties_go_to_the_lower_index,
    pins.test_knn_with_k_at_least_n_is_the_global_form,
    pins.test_knn_k1_is_the_nearest_neighbour,
    pins.test_knn_selection_is_decided_in_fp32,
    pins.test_knn_non_finite_inputs,
    pins.test_local_ignores_non_finite_points,
    lambda: pins.test_local_gradient_matches_central_differences(3.0),
    pins.test_local_gradient_with_huge_radius_is_the_global_gradient,
    pins.test_local_gradient_sums_and_translation,
    pins.test_local_gradient_at_hits_and_empty_neighbourhoods,
    lambda: pins.test_knn_gradient_matches_central_differences(3.0),
    pins.test_knn_gradient_with_k_at_least_n_is_the_global_gradient,
    pins.test_knn_gradient_sums_and_translation,
    pins.test_knn_gradient_at_hits_and_empty_selections,
    pins.test_modified_closed_form_two_points,
    pins.test_modified_with_infinite_radius_is_the_global_form,
    pins.test_modified_is_continuous_at_the_radius,
    pins.test_modified_members_and_hits_are_the_radius_form_s,
    lambda: pins.test_modified_mpmath_general_p(2.5),
    lambda: pins.test_modified_gradient_matches_central_differences(3.0),
    pins.test_modified_gradient_at_infinite_radius_is_the_global_gradient,
    pins.test_modified_gradient_sums_translation_and_hits,
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path, monkeypatch):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found uniquely: {name}"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.bind(ctypes.CDLL(oracle.compile_source(str(mutated), str(tmp_path / "mutant.so"))))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = None
    for pin in PINS:  # the first pin that fails is enough
        try:
            pin()
        except AssertionError:
            caught = pin.__name__
            break
    assert caught is not None, f"no pin caught: {name}"


def test_unmutated_source_passes_every_pin(tmp_path, monkeypatch):
    lib = oracle.bind(ctypes.CDLL(oracle.compile_source(oracle._SRC, str(tmp_path / "clean.so"))))
    monkeypatch.setattr(oracle, "_lib", lib)
    for pin in PINS:
        pin()
    assert os.path.exists(oracle._SRC)
