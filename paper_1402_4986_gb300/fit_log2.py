"""Coefficients of the FMA-pipe log2 used by the general-power sweep.

The sweep evaluates log2 d^2 on the MUFU pipe (`lg2.approx`) for most pairs
and, to balance the two arithmetic pipes, by a polynomial on the FMA pipe for
a fixed fraction of them.  For x = 2^e m with m in [1/sqrt 2, sqrt 2):

    log2 x = e + s P(s),   s = m - 1,

where P approximates log2(1 + s) / s.  P is the minimax polynomial of
degree DEGREE for the relative error on [1/sqrt 2 - 1, sqrt 2 - 1], found by
the Remez exchange algorithm (alternation at DEGREE + 2 points, refined until
the extremal errors equalise), in 40-digit arithmetic; the coefficients are
then rounded to fp32, which is what the kernel stores.

Run as a script to print the coefficients in the form the kernel source
holds them.  tests/test_log2_poly.py recomputes them and checks the kernel's
constants against this fit and the fp32 evaluation against the bound.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

DEGREE = 8
LO = float(np.sqrt(0.5)) - 1.0
HI = float(np.sqrt(2.0)) - 1.0


def _f(s):
    return mp.log(1 + s) / (mp.log(2) * s) if s != 0 else 1 / mp.log(2)


def remez(degree: int = DEGREE, lo: float = LO, hi: float = HI, iters: int = 30):
    """Minimax P (coefficients low to high) for max |P(s) / f(s) - 1|."""
    mp.mp.dps = 40
    n = degree + 2
    # Start from the Chebyshev extrema of the interval.
    xs = [mp.mpf(lo + hi) / 2 + mp.mpf(hi - lo) / 2 * mp.cos(mp.pi * k / (n - 1))
          for k in range(n)][::-1]
    coef = None
    for _ in range(iters):
        # Solve P(x_k) - f(x_k) = (-1)^k E f(x_k) for the coefficients and E.
        A = mp.matrix(n, n)
        rhs = mp.matrix(n, 1)
        for k, x in enumerate(xs):
            fx = _f(x)
            for j in range(degree + 1):
                A[k, j] = x ** j
            A[k, degree + 1] = (-1) ** k * fx
            rhs[k] = fx
        sol = mp.lu_solve(A, rhs)
        coef = [sol[j] for j in range(degree + 1)]
        # New reference: the extrema of the relative error between sign changes.
        grid = [mp.mpf(lo) + (mp.mpf(hi) - lo) * i / 4000 for i in range(4001)]
        err = [_rel_err(coef, g) for g in grid]
        xs = _extrema(grid, err, n)
    return coef


def _rel_err(coef, s):
    p = mp.mpf(0)
    for c in reversed(coef):
        p = p * s + c
    return p / _f(s) - 1


def _extrema(grid, err, n):
    # Split the grid into runs of constant sign and keep each run's largest |err|.
    runs, cur = [], [0]
    for i in range(1, len(grid)):
        if (err[i] >= 0) == (err[cur[0]] >= 0):
            cur.append(i)
        else:
            runs.append(cur)
            cur = [i]
    runs.append(cur)
    pts = [max(r, key=lambda i: abs(err[i])) for r in runs]
    while len(pts) > n:  # drop the smallest end point
        if abs(err[pts[0]]) < abs(err[pts[-1]]):
            pts = pts[1:]
        else:
            pts = pts[:-1]
    return [grid[i] for i in pts]


def coefficients_f32(degree: int = DEGREE):
    """The fp32 coefficients, low to high."""
    return [np.float32(float(c)) for c in remez(degree)]


if __name__ == "__main__":
    cs = coefficients_f32()
    print("// log2(1 + s) / s on [1/sqrt2 - 1, sqrt2 - 1], low to high (fit_log2.py)")
    for c in cs:
        print(f"  {float(c)!r:>24}f,")
