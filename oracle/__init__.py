"""FP64 CPU oracle for Shepard IDW (Sec. 2.1, Eq. 1): the global form, its
gradients, and the radius-limited and k-nearest-neighbour local forms of
the related work (Sec. 1) with their gradients.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA library
(``paper_1402_4986_gb300``) and never imports it.

The arithmetic lives in ``idw_oracle.c`` (plain C, FP64, Neumaier sums,
pthreads over queries); this module only compiles it with gcc and marshals
numpy arrays.  Inputs given as float32 are promoted to float64 exactly, so the
oracle sees the same bit patterns as the GPU path.

Parity: pinned by ``tests/test_oracle_pins.py`` (exact rationals, mpmath,
closed forms, invariants, finite differences, FP32-decision searches), and
``tests/test_oracle_mutations.py`` checks that planted mistakes fail a pin.
The ``bench.py`` CPU legs (``cpu_baseline`` and ``--impl reference``) time it
as it stands.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "idw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def bind(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    d = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.oracle_idw_forward.argtypes = [d, i64, d, i64, ctypes.c_double, d,
                                       ctypes.POINTER(ctypes.c_int64), d, ctypes.c_int]
    lib.oracle_idw_forward.restype = ctypes.c_int
    lib.oracle_idw_grad.argtypes = [d, i64, d, i64, ctypes.c_double, d, d, d, d, d, d,
                                    ctypes.c_int]
    lib.oracle_idw_grad.restype = ctypes.c_int
    lib.oracle_idw_local.argtypes = [d, i64, d, i64, ctypes.c_double, ctypes.c_double, d,
                                     ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    lib.oracle_idw_local.restype = ctypes.c_int
    lib.oracle_idw_knn.argtypes = [d, i64, d, i64, ctypes.c_double, ctypes.c_int, d,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    lib.oracle_idw_knn.restype = ctypes.c_int
    lib.oracle_idw_local_grad.argtypes = [d, i64, d, i64, ctypes.c_double, ctypes.c_double, d,
                                          d, d, d, d, d, ctypes.c_int]
    lib.oracle_idw_local_grad.restype = ctypes.c_int
    lib.oracle_idw_knn_grad.argtypes = [d, i64, d, i64, ctypes.c_double, ctypes.c_int, d, d, d, d,
                                        d, d, ctypes.c_int]
    lib.oracle_idw_knn_grad.restype = ctypes.c_int
    lib.oracle_idw_modified.argtypes = [d, i64, d, i64, ctypes.c_double, ctypes.c_double, d,
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    lib.oracle_idw_modified.restype = ctypes.c_int
    lib.oracle_idw_modified_grad.argtypes = [d, i64, d, i64, ctypes.c_double, ctypes.c_double, d,
                                             d, d, d, d, d]
    lib.oracle_idw_modified_grad.restype = ctypes.c_int
    return lib


def compile_source(src_path: str, out_path: str) -> str:
    """Compile an oracle C source to a shared library (gcc, plain IEEE FP64)."""
    subprocess.check_call([
        "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
        "-pthread", "-D_POSIX_C_SOURCE=200809L", src_path, "-o", out_path, "-lm",
    ])
    return out_path


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
    return _lib


def _f64(a, cols):
    a = np.ascontiguousarray(np.asarray(a), dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != cols:
        raise ValueError(f"expected an array of shape (k, {cols}), got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def idw(data_xyz, queries_xy, p: float, threads: int = 0, return_s0: bool = False):
    """Eq. 1 in FP64 for every query.

    data_xyz: (n, 3) array of (x, y, z); queries_xy: (m, 2) array of (x, y).
    Returns (Z float64[m], hit int64[m]) where hit is the lowest index of a
    coincident data point, or -1; with ``return_s0`` also the weight sum S0
    scaled by d2_min^(p/2) (inf at an exact hit).
    """
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    m = q.shape[0]
    Z = np.empty(m, np.float64)
    hit = np.empty(m, np.int64)
    S0 = np.empty(m, np.float64) if return_s0 else None
    rc = lib.oracle_idw_forward(_ptr(data), data.shape[0], _ptr(q), m, float(p), _ptr(Z),
                                hit.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                _ptr(S0) if S0 is not None else None, int(threads))
    if rc < 0:
        raise ValueError("oracle_idw_forward rejected its arguments")
    return (Z, hit, S0) if return_s0 else (Z, hit)


def idw_local(data_xyz, queries_xy, p: float, radius: float, threads: int = 0):
    """Eq. 1 over the data points within ``radius`` of each query (FP64).

    Membership is decided in FP32 as a GPU evaluates it (see idw_oracle.c).
    Returns (Z float64[m] (NaN where no member), hit int64[m], count int32[m]).
    """
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    m = q.shape[0]
    Z = np.empty(m, np.float64)
    hit = np.empty(m, np.int64)
    count = np.empty(m, np.int32)
    rc = lib.oracle_idw_local(_ptr(data), data.shape[0], _ptr(q), m, float(p), float(radius),
                              _ptr(Z), hit.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              count.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(threads))
    if rc < 0:
        raise ValueError("oracle_idw_local rejected its arguments")
    return Z, hit, count


def idw_knn(data_xyz, queries_xy, p: float, k: int, threads: int = 0):
    """Eq. 1 over the k data points nearest to each query (FP64 weights).

    Nearness is ranked by (FP32 d2, index) as a GPU evaluates it (see
    idw_oracle.c).  Returns a dict with Z float64[m] (NaN where nothing is
    selected), hit int64[m], kd2 float32[m], nbr int64[m, k] (key order, -1
    padded) and count int32[m].
    """
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    m = q.shape[0]
    Z = np.empty(m, np.float64)
    hit = np.empty(m, np.int64)
    kd2 = np.empty(m, np.float32)
    nbr = np.empty((m, int(k)), np.int64)
    count = np.empty(m, np.int32)
    rc = lib.oracle_idw_knn(_ptr(data), data.shape[0], _ptr(q), m, float(p), int(k), _ptr(Z),
                            hit.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            kd2.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                            nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            count.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(threads))
    if rc < 0:
        raise ValueError("oracle_idw_knn rejected its arguments")
    return {"Z": Z, "hit": hit, "kd2": kd2, "nbr": nbr, "count": count}


def idw_grad(data_xyz, queries_xy, p: float, g, threads: int = 0):
    """Gradients of L = sum_j g_j Z(q_j) in FP64 (chain rule on Eq. 1).

    Returns a dict with Z[m], grad_z[n], grad_xy[n,2], grad_q[m,2], grad_p.
    """
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    n, m = data.shape[0], q.shape[0]
    g = np.ascontiguousarray(np.asarray(g), dtype=np.float64).reshape(m)
    Z = np.empty(m, np.float64)
    gz = np.empty(n, np.float64)
    gxy = np.empty((n, 2), np.float64)
    gq = np.empty((m, 2), np.float64)
    gp = np.empty(1, np.float64)
    rc = lib.oracle_idw_grad(_ptr(data), n, _ptr(q), m, float(p), _ptr(g), _ptr(Z), _ptr(gz),
                             _ptr(gxy), _ptr(gq), _ptr(gp), int(threads))
    if rc < 0:
        raise ValueError("oracle_idw_grad rejected its arguments")
    return {"Z": Z, "grad_z": gz, "grad_xy": gxy, "grad_q": gq, "grad_p": float(gp[0])}


def idw_local_grad(data_xyz, queries_xy, p: float, radius: float, g, threads: int = 0):
    """Gradients of L = sum_j g_j Z(q_j) for the local form (FP64).

    The membership sets (FP32 test, as ``idw_local``) are held fixed, so each
    derivative is the global one summed over the members.  Returns a dict
    with Z[m], grad_z[n], grad_xy[n,2], grad_q[m,2], grad_p.
    """
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    n, m = data.shape[0], q.shape[0]
    g = np.ascontiguousarray(np.asarray(g), dtype=np.float64).reshape(m)
    Z = np.empty(m, np.float64)
    gz = np.empty(n, np.float64)
    gxy = np.empty((n, 2), np.float64)
    gq = np.empty((m, 2), np.float64)
    gp = np.empty(1, np.float64)
    rc = lib.oracle_idw_local_grad(_ptr(data), n, _ptr(q), m, float(p), float(radius), _ptr(g),
                                   _ptr(Z), _ptr(gz), _ptr(gxy), _ptr(gq), _ptr(gp), int(threads))
    if rc < 0:
        raise ValueError("oracle_idw_local_grad rejected its arguments")
    return {"Z": Z, "grad_z": gz, "grad_xy": gxy, "grad_q": gq, "grad_p": float(gp[0])}


def idw_knn_grad(data_xyz, queries_xy, p: float, k: int, g, threads: int = 0):
    """Gradients of L = sum_j g_j Z(q_j) for the k-NN form (FP64).

    Each query's selection (``idw_knn``) is held fixed, so each derivative
    is the global one summed over the selected points.  Returns a dict with
    Z[m], grad_z[n], grad_xy[n,2], grad_q[m,2], grad_p.
    """
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    n, m = data.shape[0], q.shape[0]
    g = np.ascontiguousarray(np.asarray(g), dtype=np.float64).reshape(m)
    Z = np.empty(m, np.float64)
    gz = np.empty(n, np.float64)
    gxy = np.empty((n, 2), np.float64)
    gq = np.empty((m, 2), np.float64)
    gp = np.empty(1, np.float64)
    rc = lib.oracle_idw_knn_grad(_ptr(data), n, _ptr(q), m, float(p), int(k), _ptr(g), _ptr(Z),
                                 _ptr(gz), _ptr(gxy), _ptr(gq), _ptr(gp), int(threads))
    if rc < 0:
        raise ValueError("oracle_idw_knn_grad rejected its arguments")
    return {"Z": Z, "grad_z": gz, "grad_xy": gxy, "grad_q": gq, "grad_p": float(gp[0])}


def idw_modified(data_xyz, queries_xy, p: float, radius: float, threads: int = 0):
    """Modified Shepard (FP64): Eq. 1 over the radius form's members with
    weights ((R - d)/(R d))^p.  Returns (Z, hit, count) as ``idw_local``.
    """
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    m = q.shape[0]
    Z = np.empty(m, np.float64)
    hit = np.empty(m, np.int64)
    count = np.empty(m, np.int32)
    rc = lib.oracle_idw_modified(_ptr(data), data.shape[0], _ptr(q), m, float(p), float(radius),
                                 _ptr(Z), hit.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 count.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 int(threads))
    if rc < 0:
        raise ValueError("oracle_idw_modified rejected its arguments")
    return Z, hit, count


def idw_modified_grad(data_xyz, queries_xy, p: float, radius: float, g):
    """Gradients of L = sum_j g_j Z(q_j) for modified Shepard (FP64, the
    membership sets held fixed).  Returns a dict as ``idw_local_grad``."""
    lib = _load()
    data = _f64(data_xyz, 3)
    q = _f64(queries_xy, 2)
    n, m = data.shape[0], q.shape[0]
    g = np.ascontiguousarray(np.asarray(g), dtype=np.float64).reshape(m)
    Z = np.empty(m, np.float64)
    gz = np.empty(n, np.float64)
    gxy = np.empty((n, 2), np.float64)
    gq = np.empty((m, 2), np.float64)
    gp = np.empty(1, np.float64)
    rc = lib.oracle_idw_modified_grad(_ptr(data), n, _ptr(q), m, float(p), float(radius),
                                      _ptr(g), _ptr(Z), _ptr(gz), _ptr(gxy), _ptr(gq), _ptr(gp))
    if rc < 0:
        raise ValueError("oracle_idw_modified_grad rejected its arguments")
    return {"Z": Z, "grad_z": gz, "grad_xy": gxy, "grad_q": gq, "grad_p": float(gp[0])}

