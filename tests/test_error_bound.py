"""The FP32 form's worst-case error bound (Eq. 1), checked on the CPU.

At p = 2 the GPU sweep sums each chunk of 64 points as a balanced tree
(S0, 6 levels) and as FMA chains of 4 products joined by a 4-level tree
(S1), then folds the chunk sums error-free (TwoSum).  The first-order bound
at p = 2, relative to max |z|, is

    E <= 2 delta_w + gamma_S0 + gamma_S1 + u
       = 2 (4 + 2 + 2) u + 6 u + (4 + 4) u + u = 31 u ~ 1.85e-6   (u = 2^-24)

with delta_w the weight error of a shared reciprocal (d^2: 4u, two
products: 2u, rcp.approx: one ulp = 2u).  A long sequential chunk has no
such bound: a near point entering first makes the following far points'
weights round away one by one.  ``synthetic.dominant_first`` builds that
case; these tests emulate both summation orders in exactly rounded float32
(numpy) and compare each with the FP64 oracle.  The same input runs on the
GPU in tests/test_gpu_error_bound.py.
"""
import math

import numpy as np

import oracle
import synthetic

U = 2.0 ** -24
BOUND_P2 = 31 * U
CHUNK, CHAIN = 64, 4  # the p = 2 chunk shape
TOL = 2e-6


def _weights_f32(data, q):
    """w_i = fl(1 / d_i^2) with d^2 rounded as the kernel forms it."""
    f = np.float32
    dx = (f(q[0]) - data[:, 0]).astype(np.float32)
    dy = (f(q[1]) - data[:, 1]).astype(np.float32)
    dx2 = (dx * dx).astype(np.float32)
    d2 = (dy.astype(np.float64) ** 2 + dx2.astype(np.float64)).astype(np.float32)  # one FMA
    return (np.float32(1.0) / d2).astype(np.float32)


def _sequential(v, chunk):
    """Chunk sums accumulated left to right in float32; chunks combined exactly."""
    sums = []
    for c in range(0, len(v), chunk):
        s = np.float32(0.0)
        for x in v[c:c + chunk]:
            s = np.float32(s + x)
        sums.append(float(s))
    return math.fsum(sums)


def _tree(v):
    """Balanced pairwise sum of a power-of-two count of float32 terms."""
    v = list(v)
    while len(v) > 1:
        v = [np.float32(v[i] + v[i + 1]) for i in range(0, len(v), 2)]
    return v[0]


def _tree_chunks_s0(w):
    return math.fsum(float(_tree(w[c:c + CHUNK])) for c in range(0, len(w), CHUNK))


def _tree_chunks_s1(w, z):
    """Chains of CHAIN products (MUL, then FMAs rounded once each), joined by a tree."""
    total = []
    for c in range(0, len(w), CHUNK):
        chains = []
        for k in range(c, c + CHUNK, CHAIN):
            t = np.float32(w[k] * z[k])
            for i in range(k + 1, k + CHAIN):
                t = np.float32(float(w[i]) * float(z[i]) + float(t))
            chains.append(t)
        total.append(float(_tree(chains)))
    return math.fsum(total)


def _errors(order):
    prob = synthetic.dominant_first()
    data, qs = prob["data"], prob["queries"]
    z = data[:, 2]
    Z64, _ = oracle.idw(data, qs, 2.0)
    errs = []
    for j, q in enumerate(qs):
        w = _weights_f32(data, q)
        if order == "sequential64":
            s0 = _sequential(w, 64)
            s1 = _sequential((w * z).astype(np.float32), 64)  # products exact here: z = +-1
        else:
            s0 = _tree_chunks_s0(w)
            s1 = _tree_chunks_s1(w, z)
        errs.append(abs(s1 / s0 - Z64[j]) / np.max(np.abs(z)))
    return np.array(errs), prob["positions"]


def test_dominant_first_defeats_sequential_chunks():
    """The adversarial input is real: a sequential 64-point chunk loses
    every far point after the near one, an error of about 2 (63 - pos) 0.45 u."""
    errs, pos = _errors("sequential64")
    first = errs[list(pos).index(0)]
    assert first > TOL, first
    assert first > 0.9 * 2 * 63 * 0.45 * U, first
    # The loss shrinks with the number of far points after the near one.
    assert errs[list(pos).index(63)] < 1e-7


def test_tree_chunks_meet_the_bound_on_dominant_first():
    errs, _ = _errors("tree")
    assert np.max(errs) <= BOUND_P2, np.max(errs)
    assert np.max(errs) < TOL


def test_bound_constants():
    """The bound's arithmetic: shared-reciprocal weight error, tree depths,
    final rounding; below the 2e-6 bar with margin."""
    delta_w = (4 + 2 + 2) * U
    gamma_s0 = math.log2(CHUNK) * U                   # tree levels
    gamma_s1 = (CHAIN + math.log2(CHUNK / CHAIN)) * U  # chain (MUL + FMAs), then tree levels
    assert math.isclose(2 * delta_w + gamma_s0 + gamma_s1 + U, BOUND_P2)
    assert BOUND_P2 < 0.93 * TOL
