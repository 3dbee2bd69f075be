"""Seeded synthetic inputs for global Shepard IDW.

This module serves both the CUDA path and the FP64 oracle.  It draws inputs
only; it holds none of the interpolation's arithmetic and imports neither
side.  Every array it returns is C-contiguous float32 (the library's input
precision), so both sides see identical bit patterns.

The paper evaluates equal numbers of data and prediction points at sizes
10K ... 1000K with 1K = 1024 (Sec. 3.1 and Sec. 4.1) and names no dataset, so
every workload here is synthetic.  Recipes:

  field_wave      z = sin(2 pi x) cos(2 pi y) + 0.1 N(0,1)      (uniform data)
  field_bump      z = exp(-4 r^2) + 0.05 N(0,1), r = |p - (0.5, 0.5)|
  exact-hit mix   a fixed count of queries replaced by bit-exact copies of
                  randomly chosen data points' (x, y)
  mixture         64 isotropic Gaussian blobs, centres U[0,1)^2, sigma 0.01,
                  equal weights; samples outside [0,1)^2 are kept as drawn
  grid            g x g cell centres ((i + 0.5)/g, (j + 0.5)/g)
  batch           instance sizes log-uniform in [lo, hi], drawn independently
  local           uniform data and queries, radius R chosen so that a query
                  has K data points within R on average: pi R^2 N = K
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1402

# Paper-shaped sizes: equal data and query counts.
SCALE_SWEEP = (10_000, 50_000, 100_000, 500_000, 1 << 20)
PAPER_SIZES_K1024 = (10 * 1024, 50 * 1024, 100 * 1024, 500 * 1024, 1000 * 1024)


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def uniform_xy(rng: np.random.Generator, k: int) -> np.ndarray:
    """k points uniform in [0,1)^2 as float32 (k, 2)."""
    return rng.random((k, 2), dtype=np.float64).astype(np.float32)


def field_wave(rng: np.random.Generator, xy: np.ndarray) -> np.ndarray:
    x = xy[:, 0].astype(np.float64)
    y = xy[:, 1].astype(np.float64)
    z = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.1 * rng.standard_normal(xy.shape[0])
    return z.astype(np.float32)


def field_bump(rng: np.random.Generator, xy: np.ndarray) -> np.ndarray:
    r2 = (xy[:, 0].astype(np.float64) - 0.5) ** 2 + (xy[:, 1].astype(np.float64) - 0.5) ** 2
    z = np.exp(-4.0 * r2) + 0.05 * rng.standard_normal(xy.shape[0])
    return z.astype(np.float32)


def pack_xyz(xy: np.ndarray, z: np.ndarray) -> np.ndarray:
    """(n, 3) float32 rows (x, y, z): the library's user-facing data layout."""
    out = np.empty((xy.shape[0], 3), np.float32)
    out[:, :2] = xy
    out[:, 2] = z
    return out


def mixture_xy(rng: np.random.Generator, k: int, components: int = 64,
               sigma: float = 0.01) -> np.ndarray:
    centres = rng.random((components, 2))
    which = rng.integers(0, components, size=k)
    pts = centres[which] + sigma * rng.standard_normal((k, 2))
    return pts.astype(np.float32)


def grid_xy(g: int) -> np.ndarray:
    c = (np.arange(g, dtype=np.float64) + 0.5) / g
    gx, gy = np.meshgrid(c, c, indexing="xy")
    return np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.float32)


def plant_exact_hits(rng: np.random.Generator, data_xyz: np.ndarray, queries_xy: np.ndarray,
                     count: int):
    """Overwrite ``count`` queries with bit-exact copies of data points' (x, y).

    Returns (query_indices, data_indices), both sorted by query index.
    """
    m, n = queries_xy.shape[0], data_xyz.shape[0]
    count = min(count, m, n)
    qi = np.sort(rng.choice(m, size=count, replace=False))
    di = rng.choice(n, size=count, replace=False)
    queries_xy[qi] = data_xyz[di, :2]
    return qi, di


def uniform_problem(n: int, m: int, seed: int = DEFAULT_SEED, exact_hits: int = 0):
    """Uniform data with the wave field and uniform queries.

    Returns dict(data=(n,3) f32, queries=(m,2) f32, hit_q, hit_d).
    """
    rng = _rng(seed)
    xy = uniform_xy(rng, n)
    data = pack_xyz(xy, field_wave(rng, xy))
    queries = uniform_xy(rng, m)
    hq, hd = plant_exact_hits(rng, data, queries, exact_hits) if exact_hits else (
        np.zeros(0, np.int64), np.zeros(0, np.int64))
    return {"data": data, "queries": queries, "hit_q": hq, "hit_d": hd}


def config_exact_hits(seed: int = DEFAULT_SEED + 1, n: int = 16384, m: int = 16384, hits: int = 64):
    """N = M = 16384 uniform, wave field, 64 queries placed on data points, p = 2."""
    out = uniform_problem(n, m, seed, exact_hits=hits)
    out["p"] = 2.0
    return out


def config_scale(n: int, seed: int = DEFAULT_SEED + 2):
    """One point of the equal-size scale sweep (N = M = n), wave field, p = 2."""
    out = uniform_problem(n, n, seed + n)
    out["p"] = 2.0
    return out


def config_clustered(seed: int = DEFAULT_SEED + 3, n: int = 262144, grid: int = 1024):
    """Gaussian-mixture data with the bump field, queries on a grid x grid lattice."""
    rng = _rng(seed)
    xy = mixture_xy(rng, n)
    data = pack_xyz(xy, field_bump(rng, xy))
    return {"data": data, "queries": grid_xy(grid), "p_values": (1.5, 2.0, 3.5)}


def config_adjoint(seed: int = DEFAULT_SEED + 4, n: int = 262144, m: int = 262144, p: float = 2.5):
    """Uniform data and queries, wave field, p = 2.5, upstream gradient N(0,1)."""
    rng = _rng(seed)
    xy = uniform_xy(rng, n)
    data = pack_xyz(xy, field_wave(rng, xy))
    queries = uniform_xy(rng, m)
    g = rng.standard_normal(m).astype(np.float32)
    return {"data": data, "queries": queries, "grad_out": g, "p": p}


def separated_xy(rng: np.random.Generator, k: int, min_sep: float) -> np.ndarray:
    """k points on a jittered lattice in [0,1)^2 with pairwise distance >= min_sep."""
    g = int(np.ceil(np.sqrt(k)))
    cell = 1.0 / g
    jitter = max(0.0, 0.5 * (cell - min_sep))
    idx = rng.permutation(g * g)[:k]
    cx = (idx % g + 0.5) * cell
    cy = (idx // g + 0.5) * cell
    pts = np.stack([cx, cy], 1) + rng.uniform(-jitter, jitter, (k, 2))
    return pts.astype(np.float32)


def config_batch(seed: int = DEFAULT_SEED + 5, count: int = 256, lo: int = 1024, hi: int = 262144):
    """``count`` independent instances, N_i and M_i log-uniform in [lo, hi]."""
    rng = _rng(seed)
    ln = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
    lm = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
    inst = []
    for k in range(count):
        xy = uniform_xy(rng, int(ln[k]))
        data = pack_xyz(xy, field_wave(rng, xy))
        inst.append({"data": data, "queries": uniform_xy(rng, int(lm[k]))})
    return {"instances": inst, "p": 2.0}


def batch_sizes(seed: int = DEFAULT_SEED + 5, count: int = 256, lo: int = 1024, hi: int = 262144):
    """The (N_i, M_i) of ``config_batch`` without drawing the points."""
    rng = _rng(seed)
    ln = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
    lm = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
    return ln, lm


def local_radius(n: int, members: float) -> float:
    """R with pi R^2 n = members: the mean neighbour count of uniform data on
    the unit square (ignoring the boundary)."""
    return float(np.sqrt(members / (np.pi * n)))


def config_local(seed: int = DEFAULT_SEED + 6, n: int = 1 << 20, m: int = 1 << 20,
                 members: float = 32.0, clustered: bool = False):
    """Local (radius-limited) workload: N data, M queries, R for ``members``
    neighbours on average; uniform data with the wave field, or the mixture
    with the bump field when ``clustered``.  p = 2."""
    rng = _rng(seed)
    xy = mixture_xy(rng, n) if clustered else uniform_xy(rng, n)
    z = field_bump(rng, xy) if clustered else field_wave(rng, xy)
    data = pack_xyz(xy, z)
    return {"data": data, "queries": uniform_xy(rng, m), "radius": local_radius(n, members),
            "p": 2.0}


# Positions of the dominant point inside its 64-point block, one per query of
# ``dominant_first``: chunk starts and ends, odd offsets, and both halves.
DOMINANT_POSITIONS = (0, 1, 2, 3, 5, 7, 8, 15, 16, 17, 24, 31, 32, 33, 40, 47, 48, 56, 62, 63)


def dominant_first(ratio: float = 0.45, positions=DOMINANT_POSITIONS, d0: float = 2.0 ** -20):
    """An input built to defeat long sequential sums (not drawn at random).

    Query j sits at the centre of its own unit cell; data block j (indices
    64 j ... 64 j + 63) holds one point at distance d0 from it (index
    64 j + positions[j], z = +1) and 63 points on a circle of radius
    R = d0 2^12 / sqrt(ratio) around it (z = -1).  At p = 2 each circle
    point's weight is ``ratio`` 2^-24 times the near point's, below half an
    ulp of it for ratio < 1/2, so a running FP32 sum that starts at the near
    point's weight rounds every one of them away.  The true Z_j is about
    1 - 4 * 63 * ratio * 2^-24; blocks of the other queries lie a unit or
    more away and weigh about 2^-30 of the near point or less.

    Returns dict(data=(64 m, 3) f32, queries=(m, 2) f32, positions).
    """
    m = len(positions)
    g = int(np.ceil(np.sqrt(m)))
    R = d0 * 4096.0 / np.sqrt(ratio)
    data = np.zeros((64 * m, 3), np.float32)
    queries = np.zeros((m, 2), np.float32)
    ang = 2.0 * np.pi * (np.arange(63) + 0.5) / 63.0
    for j, pos in enumerate(positions):
        c = np.array([j % g + 0.5, j // g + 0.5])  # multiples of 2^-1: d0 offsets stay exact
        queries[j] = c
        ring = np.stack([c[0] + R * np.cos(ang), c[1] + R * np.sin(ang)], 1)
        block = np.empty((64, 3))
        others = [i for i in range(64) if i != pos]
        block[others, :2] = ring
        block[others, 2] = -1.0
        block[pos] = (c[0] + d0, c[1], 1.0)
        data[64 * j:64 * j + 64] = block
    return {"data": np.ascontiguousarray(data), "queries": np.ascontiguousarray(queries),
            "positions": tuple(positions)}
