"""GB300 (sm_103a) global Shepard IDW interpolation.

Thin Python binding over the C ABI of ``include/idw.h``: it checks tensor
shapes, dtypes and devices, passes raw pointers and the current CUDA stream
to the library, and wraps the results.  Every step of the computation runs
in the library's CUDA kernels; PyTorch only provides device memory, streams
and autograd plumbing.

    Z(q) = sum_i w_i z_i / sum_i w_i,   w_i = d(q, x_i)^(-p)    (Eq. 1)
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _lib
from ._lib import IDWError, PREC_F32_COMP, PREC_F64_PLAIN, PlanInfo

__all__ = [
    "IDWError", "Handle", "get_handle", "interpolate", "interpolate_saved", "interpolate_host",
    "interpolate_batched", "interpolate_local", "interpolate_modified", "interpolate_knn",
    "LocalIndex",
    "local_backward", "LocalIDWFunction", "idw_local", "idw_modified", "knn_backward",
    "KnnIDWFunction",
    "idw_knn",
    "paper_interpolate", "backward", "IDWFunction", "idw", "plan_forward",
    "measure_pipe_rates", "measure_mufu_errors", "sync_status", "profile_enable", "profile_read",
    "selftest_bounded_wait", "set_option", "get_option", "PREC_F32_COMP", "PREC_F64_PLAIN",
]

_PREC = {"f32c": PREC_F32_COMP, "f32_comp": PREC_F32_COMP, PREC_F32_COMP: PREC_F32_COMP,
         "f64": PREC_F64_PLAIN, "f64_plain": PREC_F64_PLAIN, PREC_F64_PLAIN: PREC_F64_PLAIN}
_DTYPE = {PREC_F32_COMP: torch.float32, PREC_F64_PLAIN: torch.float64}


class Handle:
    """Owns one ``idw_handle_t`` (and its device workspace) on one device."""

    def __init__(self, device: int = 0, autotune_cache: str | None = None):
        self.lib = _lib.load()
        self.device = int(device)
        h = ctypes.c_void_p()
        if autotune_cache is None:
            _lib.check(self.lib.idw_create(ctypes.byref(h), self.device), "idw_create")
        else:
            _lib.check(self.lib.idw_create_ex(ctypes.byref(h), self.device,
                                              os.fsencode(autotune_cache)), "idw_create_ex")
        self.ptr = h

    def close(self):
        if getattr(self, "ptr", None):
            self.lib.idw_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles: dict = {}
_hlock = threading.Lock()


def get_handle(device=None) -> Handle:
    """The process-wide handle of ``device`` (current device by default)."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    with _hlock:
        if dev not in _handles:
            _handles[dev] = Handle(dev)
        return _handles[dev]


def _stream(t: torch.Tensor):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _prec(precision):
    try:
        return _PREC[precision]
    except KeyError:
        raise ValueError(f"unknown precision {precision!r}") from None


def _check_inputs(data, queries, prec):
    dt = _DTYPE[prec]
    if data.dim() != 2 or data.shape[1] != 3:
        raise ValueError(f"data must be (n, 3) rows (x, y, z), got {tuple(data.shape)}")
    if queries.dim() != 2 or queries.shape[1] != 2:
        raise ValueError(f"queries must be (m, 2) rows (x, y), got {tuple(queries.shape)}")
    for name, t in (("data", data), ("queries", queries)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt} for this precision, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if data.device != queries.device:
        raise ValueError("data and queries must be on the same device")


def _check_buf(t, numel, dtype, device, name):
    """A caller-supplied output or saved-state tensor: the library writes or
    reads exactly ``numel`` contiguous ``dtype`` values at its address on
    ``device``, so each of those must hold before the call."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} values, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _handle_for(handle, device):
    """``handle`` (or the device's process-wide one), checked to own ``device``."""
    if handle is None:
        return get_handle(device)
    if device.type != "cuda" or handle.device != (device.index or 0):
        raise ValueError(f"the handle belongs to cuda:{handle.device}, the tensors to {device}")
    return handle


def _grad_vec(grad_out, m, device):
    """The upstream gradient as contiguous float32[m] on ``device``."""
    if not isinstance(grad_out, torch.Tensor) or grad_out.device != device:
        raise ValueError(f"grad_out must be a tensor on {device}")
    if grad_out.numel() != m:
        raise ValueError(f"grad_out must hold {m} values, got {grad_out.numel()}")
    return grad_out.reshape(m).contiguous().to(torch.float32)


def interpolate_saved(data: torch.Tensor, queries: torch.Tensor, p: float = 2.0,
                      precision="f32c", out=None, handle: Handle | None = None):
    """Eq. 1 plus the state the adjoint needs.

    Returns (Z, S0, hit): Z[m] (float32 or float64), S0[m] float64 (the
    weight sum, +inf at an exact hit), hit[m] int32 (exact-hit index, -1, or
    -2 where the query was recomputed in FP64).
    """
    prec = _prec(precision)
    _check_inputs(data, queries, prec)
    m = queries.shape[0]
    h = _handle_for(handle, data.device)
    if out is None:
        out = torch.empty(m, dtype=_DTYPE[prec], device=data.device)
    _check_buf(out, m, _DTYPE[prec], data.device, "out")
    s0 = torch.empty(m, dtype=torch.float64, device=data.device)
    hit = torch.empty(m, dtype=torch.int32, device=data.device)
    st = h.lib.idw_interpolate_saved(h.ptr, _ptr(data), data.shape[0], _ptr(queries), m,
                                     float(p), prec, _ptr(out), _ptr(s0), _ptr(hit),
                                     _stream(data))
    _lib.check(st, "idw_interpolate_saved", h.ptr)
    return out, s0, hit


def interpolate(data: torch.Tensor, queries: torch.Tensor, p: float = 2.0, precision="f32c",
                out: torch.Tensor | None = None, handle: Handle | None = None) -> torch.Tensor:
    """Eq. 1 for every query: data (n,3) rows (x,y,z), queries (m,2) rows (x,y).

    ``precision`` is "f32c" (FP32 pair arithmetic, compensated sums, FP64
    combine; float32 tensors) or "f64" (plain FP64; float64 tensors).
    """
    prec = _prec(precision)
    _check_inputs(data, queries, prec)
    m = queries.shape[0]
    h = _handle_for(handle, data.device)
    if out is None:
        out = torch.empty(m, dtype=_DTYPE[prec], device=data.device)
    _check_buf(out, m, _DTYPE[prec], data.device, "out")
    st = h.lib.idw_interpolate(h.ptr, _ptr(data), data.shape[0], _ptr(queries), m, float(p), prec,
                               _ptr(out), _stream(data))
    _lib.check(st, "idw_interpolate", h.ptr)
    return out


def interpolate_host(data, queries, p: float = 2.0, precision="f32c", out=None,
                     handle: Handle | None = None, stream=None):
    """Eq. 1 on host (CPU) tensors: the library copies in, computes and copies out."""
    prec = _prec(precision)
    dt = _DTYPE[prec]
    if data.device.type != "cpu" or queries.device.type != "cpu":
        raise ValueError("interpolate_host takes host tensors")
    if data.dtype != dt or queries.dtype != dt or not data.is_contiguous() or \
            not queries.is_contiguous():
        raise ValueError(f"host inputs must be contiguous {dt}")
    if data.dim() != 2 or data.shape[1] != 3:
        raise ValueError(f"data must be (n, 3) rows (x, y, z), got {tuple(data.shape)}")
    if queries.dim() != 2 or queries.shape[1] != 2:
        raise ValueError(f"queries must be (m, 2) rows (x, y), got {tuple(queries.shape)}")
    m = queries.shape[0]
    if out is not None:
        _check_buf(out, m, dt, torch.device("cpu"), "out")
    h = handle or get_handle()
    if out is None:
        out = torch.empty(m, dtype=dt, pin_memory=True)
    s = stream if stream is not None else torch.cuda.current_stream(h.device)
    st = h.lib.idw_interpolate_host(h.ptr, _ptr(data), data.shape[0], _ptr(queries), m, float(p),
                                    prec, _ptr(out), ctypes.c_void_p(s.cuda_stream))
    _lib.check(st, "idw_interpolate_host", h.ptr)
    return out


def interpolate_batched(datas, queries_list, p: float = 2.0, outs=None,
                        handle: Handle | None = None, precision="f32c"):
    """Eq. 1 for many independent problems in one call (FP32-compensated in
    one persistent launch; "f64": the plain FP64 form, one launch each)."""
    prec = _prec(precision)
    k = len(datas)
    if len(queries_list) != k:
        raise ValueError("datas and queries_list differ in length")
    if k == 0:
        return []
    dev = datas[0].device
    for d, q in zip(datas, queries_list):
        _check_inputs(d, q, prec)
        if d.device != dev:
            raise ValueError(f"every problem must be on {dev}, got {d.device}")
    if outs is None:
        outs = [torch.empty(q.shape[0], dtype=_DTYPE[prec], device=dev) for q in queries_list]
    if len(outs) != k:
        raise ValueError(f"outs must hold {k} tensors, got {len(outs)}")
    for i, (o, q) in enumerate(zip(outs, queries_list)):
        _check_buf(o, q.shape[0], _DTYPE[prec], dev, f"outs[{i}]")
    h = _handle_for(handle, dev)
    P = ctypes.c_void_p * k
    I = ctypes.c_int64 * k
    st = h.lib.idw_interpolate_batched(
        h.ptr, k, P(*[d.data_ptr() for d in datas]), I(*[d.shape[0] for d in datas]),
        P(*[q.data_ptr() for q in queries_list]), I(*[q.shape[0] for q in queries_list]),
        float(p), prec, P(*[o.data_ptr() for o in outs]), _stream(datas[0]))
    _lib.check(st, "idw_interpolate_batched", h.ptr)
    return outs


def paper_interpolate(data, queries, p: float = 2.0, kernel: str = "tiled", layout: str = "aoas",
                      precision="f32c", out=None, handle: Handle | None = None):
    """The paper's naive or tiled kernel in one of its layouts (a baseline).

    ``kernel`` in {"naive", "tiled"}; ``layout`` in {"soa", "aos", "aoas",
    "hybrid"}; ``precision`` "f32c" runs plain FP32 here, "f64" plain FP64.
    """
    prec = _prec(precision)
    _check_inputs(data, queries, prec)
    m = queries.shape[0]
    h = _handle_for(handle, data.device)
    if out is None:
        out = torch.empty(m, dtype=_DTYPE[prec], device=data.device)
    _check_buf(out, m, _DTYPE[prec], data.device, "out")
    st = h.lib.idw_paper_interpolate(h.ptr, _lib.PAPER_KERNELS[kernel], _lib.PAPER_LAYOUTS[layout],
                                     _ptr(data), data.shape[0], _ptr(queries), m, float(p), prec,
                                     _ptr(out), _stream(data))
    _lib.check(st, "idw_paper_interpolate", h.ptr)
    return out


def interpolate_local(data, queries, p: float = 2.0, radius: float = float("inf"), out=None,
                      counts: bool = False, handle: Handle | None = None):
    """Eq. 1 over the data points within ``radius`` of each query (FP32).

    Returns ``out`` (float32[m], NaN where no data point is within R), or
    ``(out, count)`` with ``count`` int32[m] (members per query, -1 at an
    exact hit) when ``counts`` is true.  Asynchronous on the current stream
    (graph-capturable).
    """
    _check_inputs(data, queries, PREC_F32_COMP)
    m = queries.shape[0]
    h = _handle_for(handle, data.device)
    if out is None:
        out = torch.empty(m, dtype=torch.float32, device=data.device)
    _check_buf(out, m, torch.float32, data.device, "out")
    cnt = torch.empty(m, dtype=torch.int32, device=data.device) if counts else None
    st = h.lib.idw_interpolate_local(h.ptr, _ptr(data), data.shape[0], _ptr(queries), m, float(p),
                                     float(radius), _ptr(out), _ptr(cnt),
                                     _stream(data))
    _lib.check(st, "idw_interpolate_local", h.ptr)
    return (out, cnt) if counts else out


def interpolate_modified(data, queries, p: float = 2.0, radius: float = float("inf"), out=None,
                         counts: bool = False, handle: Handle | None = None):
    """Modified Shepard (``idw_interpolate_modified``): the radius form's
    members with weights ((R - d)/(R d))^p, which vanish at d = R.  Returns
    as ``interpolate_local``."""
    _check_inputs(data, queries, PREC_F32_COMP)
    m = queries.shape[0]
    h = _handle_for(handle, data.device)
    if out is None:
        out = torch.empty(m, dtype=torch.float32, device=data.device)
    _check_buf(out, m, torch.float32, data.device, "out")
    cnt = torch.empty(m, dtype=torch.int32, device=data.device) if counts else None
    st = h.lib.idw_interpolate_modified(h.ptr, _ptr(data), data.shape[0], _ptr(queries), m,
                                        float(p), float(radius), _ptr(out), _ptr(cnt),
                                        _stream(data))
    _lib.check(st, "idw_interpolate_modified", h.ptr)
    return (out, cnt) if counts else out


def interpolate_knn(data, queries, p: float = 2.0, k: int = 16, out=None,
                    neighbours: bool = False, kth_d2: bool = False,
                    handle: Handle | None = None):
    """Eq. 1 over the k data points nearest to each query (FP32).

    Returns ``out`` (float32[m]); with ``neighbours`` also int32[m, k] (the
    selected indices in key order, -1 padded) and with ``kth_d2`` also
    float32[m] (the k-th key's squared distance), in that order.
    """
    _check_inputs(data, queries, PREC_F32_COMP)
    m = queries.shape[0]
    h = _handle_for(handle, data.device)
    if out is None:
        out = torch.empty(m, dtype=torch.float32, device=data.device)
    _check_buf(out, m, torch.float32, data.device, "out")
    nbr = torch.empty(m, int(k), dtype=torch.int32, device=data.device) if neighbours else None
    kd2 = torch.empty(m, dtype=torch.float32, device=data.device) if kth_d2 else None
    st = h.lib.idw_interpolate_knn(h.ptr, _ptr(data), data.shape[0], _ptr(queries), m, float(p),
                                   int(k), _ptr(out), _ptr(nbr), _ptr(kd2), _stream(data))
    _lib.check(st, "idw_interpolate_knn", h.ptr)
    res = (out,) + ((nbr,) if neighbours else ()) + ((kd2,) if kth_d2 else ())
    return res if len(res) > 1 else out


class LocalIndex:
    """Prepared index of a local form (``idw_local_index_create``): the data
    side is built once, then each call sorts only its own queries.

    ``LocalIndex(data, radius=R)`` serves ``interpolate`` for any radius up
    to R; ``LocalIndex(data, k=K)`` serves ``knn`` for any 1 <= k <= 64 (its
    cells are sized for K).  Results equal the one-shot
    ``interpolate_local`` / ``interpolate_knn`` on the same data.  The index
    copies what it needs, so ``data`` may change after construction.
    """

    def __init__(self, data, radius: float | None = None, k: int | None = None,
                 handle: Handle | None = None):
        if (radius is None) == (k is None):
            raise ValueError("give exactly one of radius or k")
        if data.dim() != 2 or data.shape[1] != 3 or not data.is_cuda:
            raise ValueError("data must be a CUDA (n, 3) tensor")
        if data.dtype != torch.float32 or not data.is_contiguous():
            raise ValueError("data must be contiguous float32")
        self.handle = handle or get_handle(data.device)
        self.device = data.device
        self.radius = None if radius is None else float(radius)
        self.k = None if k is None else int(k)
        self.n = data.shape[0]
        ix = ctypes.c_void_p()
        st = self.handle.lib.idw_local_index_create(
            self.handle.ptr, _ptr(data), self.n, 0.0 if radius is None else float(radius),
            0 if k is None else int(k), ctypes.byref(ix), _stream(data))
        _lib.check(st, "idw_local_index_create", self.handle.ptr)
        self.ptr = ix

    def _queries(self, queries):
        if queries.dim() != 2 or queries.shape[1] != 2 or not queries.is_cuda:
            raise ValueError("queries must be a CUDA (m, 2) tensor")
        if queries.dtype != torch.float32 or not queries.is_contiguous():
            raise ValueError("queries must be contiguous float32")
        if queries.device != self.device:
            raise ValueError("queries must be on the index's device")
        return queries.shape[0]

    def interpolate(self, queries, p: float = 2.0, radius: float | None = None, out=None,
                    counts: bool = False, handle: Handle | None = None, modified: bool = False):
        """``interpolate_local`` on the indexed data (radius defaults to the
        build radius and may not exceed it); ``modified`` selects the modified
        Shepard weights (``interpolate_modified``).  ``handle`` (default: the
        build's) supplies the workspace: one handle per concurrent stream."""
        m = self._queries(queries)
        h = self.handle if handle is None else _handle_for(handle, self.device)
        r = self.radius if radius is None else float(radius)
        if out is None:
            out = torch.empty(m, dtype=torch.float32, device=self.device)
        _check_buf(out, m, torch.float32, self.device, "out")
        cnt = torch.empty(m, dtype=torch.int32, device=self.device) if counts else None
        fn = h.lib.idw_local_index_modified if modified else h.lib.idw_local_index_interpolate
        st = fn(h.ptr, self.ptr, _ptr(queries), m, float(p), 0.0 if r is None else r,
                _ptr(out), _ptr(cnt), _stream(queries))
        _lib.check(st, "idw_local_index_modified" if modified else "idw_local_index_interpolate",
                   h.ptr)
        return (out, cnt) if counts else out

    def knn(self, queries, p: float = 2.0, k: int | None = None, out=None,
            neighbours: bool = False, kth_d2: bool = False, handle: Handle | None = None):
        """``interpolate_knn`` on the indexed data (k defaults to the build k;
        ``handle`` as in ``interpolate``)."""
        m = self._queries(queries)
        h = self.handle if handle is None else _handle_for(handle, self.device)
        kk = int(k) if k is not None else (self.k or 0)  # 0: refused by the library
        if out is None:
            out = torch.empty(m, dtype=torch.float32, device=self.device)
        _check_buf(out, m, torch.float32, self.device, "out")
        nbr = torch.empty(m, max(kk, 1), dtype=torch.int32, device=self.device) if neighbours else None
        kd2 = torch.empty(m, dtype=torch.float32, device=self.device) if kth_d2 else None
        st = h.lib.idw_local_index_knn(
            h.ptr, self.ptr, _ptr(queries), m, float(p), kk, _ptr(out), _ptr(nbr),
            _ptr(kd2), _stream(queries))
        _lib.check(st, "idw_local_index_knn", h.ptr)
        res = (out,) + ((nbr,) if neighbours else ()) + ((kd2,) if kth_d2 else ())
        return res if len(res) > 1 else out

    def close(self):
        if getattr(self, "ptr", None):
            self.handle.lib.idw_local_index_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def backward(data, queries, p, Z, s0, hit, grad_out, need_z=True, need_data_xy=True,
             need_query_xy=True, need_p=True, handle: Handle | None = None):
    """Adjoint of Eq. 1 (see include/idw.h); returns (gz, gxy, gq, gp)."""
    _check_inputs(data, queries, PREC_F32_COMP)
    n, m = data.shape[0], queries.shape[0]
    dev = data.device
    gz = torch.empty(n, dtype=torch.float32, device=dev) if need_z else None
    gxy = torch.empty(n, 2, dtype=torch.float32, device=dev) if need_data_xy else None
    gq = torch.empty(m, 2, dtype=torch.float32, device=dev) if need_query_xy else None
    gp = torch.empty(1, dtype=torch.float64, device=dev) if need_p else None
    h = _handle_for(handle, dev)
    _check_buf(Z, m, torch.float32, dev, "Z")
    _check_buf(s0, m, torch.float64, dev, "s0")
    _check_buf(hit, m, torch.int32, dev, "hit")
    g = _grad_vec(grad_out, m, dev)
    st = h.lib.idw_backward(h.ptr, _ptr(data), n, _ptr(queries), m, float(p), _ptr(Z), _ptr(s0),
                            _ptr(hit), _ptr(g), _ptr(gz), _ptr(gxy), _ptr(gq), _ptr(gp),
                            _stream(data))
    _lib.check(st, "idw_backward", h.ptr)
    return gz, gxy, gq, gp


class IDWFunction(torch.autograd.Function):
    """Differentiable Eq. 1 (FP32-compensated) with the hand-written adjoint."""

    @staticmethod
    def forward(ctx, data, queries, p):
        pv = float(p.item()) if torch.is_tensor(p) else float(p)
        Z, s0, hit = interpolate_saved(data.detach().contiguous(), queries.detach().contiguous(),
                                       pv, "f32c")
        ctx.save_for_backward(data, queries, Z, s0, hit)
        ctx.p = pv
        ctx.p_is_tensor = torch.is_tensor(p)
        return Z

    @staticmethod
    def backward(ctx, grad):
        data, queries, Z, s0, hit = ctx.saved_tensors
        need_d, need_q, need_p = ctx.needs_input_grad
        gz, gxy, gq, gp = backward(data.detach().contiguous(), queries.detach().contiguous(),
                                   ctx.p, Z, s0, hit, grad, need_z=need_d, need_data_xy=need_d,
                                   need_query_xy=need_q, need_p=need_p and ctx.p_is_tensor)
        gdata = torch.cat([gxy, gz[:, None]], 1) if need_d else None
        gp_out = gp.to(torch.float32).reshape(()) if (need_p and ctx.p_is_tensor) else None
        return gdata, gq if need_q else None, gp_out


def idw(data, queries, p=2.0):
    """Autograd entry: Z = IDW(data, queries, p); p may be a tensor to get dL/dp."""
    return IDWFunction.apply(data, queries, p)


def local_backward(data, queries, p, radius, grad_out, need_z=True, need_data_xy=True,
                   need_query_xy=True, need_p=True, handle: Handle | None = None,
                   modified: bool = False):
    """Gradients of the radius form (``idw_local_backward``), or with
    ``modified`` of modified Shepard (``idw_modified_backward``); returns
    (gz, gxy, gq, gp), each None when not requested."""
    _check_inputs(data, queries, PREC_F32_COMP)
    n, m = data.shape[0], queries.shape[0]
    dev = data.device
    gz = torch.empty(n, dtype=torch.float32, device=dev) if need_z else None
    gxy = torch.empty(n, 2, dtype=torch.float32, device=dev) if need_data_xy else None
    gq = torch.empty(m, 2, dtype=torch.float32, device=dev) if need_query_xy else None
    gp = torch.empty(1, dtype=torch.float64, device=dev) if need_p else None
    h = _handle_for(handle, dev)
    g = _grad_vec(grad_out, m, dev)
    name = "idw_modified_backward" if modified else "idw_local_backward"
    st = getattr(h.lib, name)(h.ptr, _ptr(data), n, _ptr(queries), m, float(p), float(radius),
                              _ptr(g), _ptr(gz), _ptr(gxy), _ptr(gq), _ptr(gp), _stream(data))
    _lib.check(st, name, h.ptr)
    return gz, gxy, gq, gp


class LocalIDWFunction(torch.autograd.Function):
    """Differentiable radius form: Eq. 1 over the data within ``radius`` of
    each query (plain d^-p weights, or modified Shepard weights), with the
    hand-written local adjoint (membership held fixed).  Queries without
    members give NaN and pass no gradient."""

    @staticmethod
    def forward(ctx, data, queries, p, radius, modified=False):
        pv = float(p.item()) if torch.is_tensor(p) else float(p)
        fwd = interpolate_modified if modified else interpolate_local
        Z = fwd(data.detach().contiguous(), queries.detach().contiguous(), pv, float(radius))
        ctx.save_for_backward(data, queries)
        ctx.p, ctx.radius, ctx.p_is_tensor = pv, float(radius), torch.is_tensor(p)
        ctx.modified = bool(modified)
        return Z

    @staticmethod
    def backward(ctx, grad):
        data, queries = ctx.saved_tensors
        need_d, need_q, need_p = ctx.needs_input_grad[:3]
        want_p = need_p and ctx.p_is_tensor
        gz, gxy, gq, gp = local_backward(data.detach().contiguous(), queries.detach().contiguous(),
                                         ctx.p, ctx.radius, grad, need_z=need_d,
                                         need_data_xy=need_d, need_query_xy=need_q,
                                         need_p=want_p, modified=ctx.modified)
        gdata = torch.cat([gxy, gz[:, None]], 1) if need_d else None
        gp_out = gp.to(torch.float32).reshape(()) if want_p else None
        return gdata, gq if need_q else None, gp_out, None, None


def idw_local(data, queries, p=2.0, radius=1.0):
    """Autograd entry for the radius form; p may be a tensor to get dL/dp."""
    return LocalIDWFunction.apply(data, queries, p, radius, False)


def idw_modified(data, queries, p=2.0, radius=1.0):
    """Autograd entry for modified Shepard; p may be a tensor to get dL/dp."""
    return LocalIDWFunction.apply(data, queries, p, radius, True)


def knn_backward(data, queries, p, k, grad_out, need_z=True, need_data_xy=True,
                 need_query_xy=True, need_p=True, handle: Handle | None = None):
    """Gradients of the k-NN form (``idw_knn_backward``); returns
    (gz, gxy, gq, gp), each None when not requested."""
    _check_inputs(data, queries, PREC_F32_COMP)
    n, m = data.shape[0], queries.shape[0]
    dev = data.device
    gz = torch.empty(n, dtype=torch.float32, device=dev) if need_z else None
    gxy = torch.empty(n, 2, dtype=torch.float32, device=dev) if need_data_xy else None
    gq = torch.empty(m, 2, dtype=torch.float32, device=dev) if need_query_xy else None
    gp = torch.empty(1, dtype=torch.float64, device=dev) if need_p else None
    h = _handle_for(handle, dev)
    g = _grad_vec(grad_out, m, dev)
    st = h.lib.idw_knn_backward(h.ptr, _ptr(data), n, _ptr(queries), m, float(p), int(k),
                                _ptr(g), _ptr(gz), _ptr(gxy), _ptr(gq), _ptr(gp), _stream(data))
    _lib.check(st, "idw_knn_backward", h.ptr)
    return gz, gxy, gq, gp


class KnnIDWFunction(torch.autograd.Function):
    """Differentiable k-NN form with the hand-written adjoint (each query's
    selection held fixed)."""

    @staticmethod
    def forward(ctx, data, queries, p, k):
        pv = float(p.item()) if torch.is_tensor(p) else float(p)
        Z = interpolate_knn(data.detach().contiguous(), queries.detach().contiguous(), pv, int(k))
        ctx.save_for_backward(data, queries)
        ctx.p, ctx.k, ctx.p_is_tensor = pv, int(k), torch.is_tensor(p)
        return Z

    @staticmethod
    def backward(ctx, grad):
        data, queries = ctx.saved_tensors
        need_d, need_q, need_p, _ = ctx.needs_input_grad
        want_p = need_p and ctx.p_is_tensor
        gz, gxy, gq, gp = knn_backward(data.detach().contiguous(), queries.detach().contiguous(),
                                       ctx.p, ctx.k, grad, need_z=need_d, need_data_xy=need_d,
                                       need_query_xy=need_q, need_p=want_p)
        gdata = torch.cat([gxy, gz[:, None]], 1) if need_d else None
        gp_out = gp.to(torch.float32).reshape(()) if want_p else None
        return gdata, gq if need_q else None, gp_out, None


def idw_knn(data, queries, p=2.0, k=16):
    """Autograd entry for the k-NN form; p may be a tensor to get dL/dp."""
    return KnnIDWFunction.apply(data, queries, p, k)


def sync_status(device=None, handle: Handle | None = None):
    """Synchronise the current stream and raise on a pending device error."""
    h = handle or get_handle(device)
    s = torch.cuda.current_stream(h.device)
    _lib.check(h.lib.idw_sync_status(h.ptr, ctypes.c_void_p(s.cuda_stream)), "idw_sync_status",
               h.ptr)


def set_option(name: str, value: int, handle: Handle | None = None):
    """Set a handle option (``_lib.OPTIONS``): autotune, sweep_variant,
    force_general_power, staging_layout, validate_inputs, local_query_order."""
    h = handle or get_handle()
    _lib.check(h.lib.idw_set_option(h.ptr, _lib.OPTIONS[name], int(value)), "idw_set_option")


def get_option(name: str, handle: Handle | None = None) -> int:
    """Read a handle option (also last_variant, tuned_classes)."""
    h = handle or get_handle()
    v = ctypes.c_int64()
    _lib.check(h.lib.idw_get_option(h.ptr, _lib.OPTIONS[name], ctypes.byref(v)), "idw_get_option")
    return v.value


def profile_enable(enable: bool = True, handle: Handle | None = None):
    """Record CUDA events around every all-pairs sweep launch of the handle."""
    h = handle or get_handle()
    _lib.check(h.lib.idw_profile_enable(h.ptr, int(bool(enable))), "idw_profile_enable")


def profile_read(handle: Handle | None = None):
    """(total sweep milliseconds, sweep launches) since the last read."""
    h = handle or get_handle()
    ms = ctypes.c_double()
    k = ctypes.c_int64()
    _lib.check(h.lib.idw_profile_read(h.ptr, ctypes.byref(ms), ctypes.byref(k)),
               "idw_profile_read", h.ptr)
    return ms.value, k.value


def selftest_bounded_wait(handle: Handle | None = None):
    """Launch the bounded-wait self-test (see include/idw.h); check with sync_status()."""
    h = handle or get_handle()
    s = torch.cuda.current_stream(h.device)
    _lib.check(h.lib.idw_selftest_bounded_wait(h.ptr, ctypes.c_void_p(s.cuda_stream)),
               "idw_selftest_bounded_wait", h.ptr)


def plan_forward(n: int, m: int, p: float = 2.0, precision="f32c", sm_count: int = 152,
                 ctas_per_sm: int = 0) -> dict:
    """Host-only launch plan of the forward pass (no GPU needed)."""
    lib = _lib.load()
    info = PlanInfo()
    _lib.check(lib.idw_plan_forward(sm_count, ctas_per_sm, int(n), int(m), float(p),
                                    _prec(precision), ctypes.byref(info)), "idw_plan_forward")
    return {name: getattr(info, name) for name, _ in PlanInfo._fields_}


def measure_pipe_rates(device: int = 0) -> dict:
    """Arithmetic-pipe issue rates in ops per SM per clock (see include/idw.h)."""
    lib = _lib.load()
    arr = (ctypes.c_double * 6)()
    _lib.check(lib.idw_measure_pipe_rates(int(device), arr), "idw_measure_pipe_rates")
    keys = ("ffma", "ffma2", "mufu_rcp", "mufu_lg2", "mufu_ex2", "dfma")
    return dict(zip(keys, list(arr)))


def measure_mufu_errors(device: int = 0) -> dict:
    """Worst-case accuracy of the MUFU rcp / lg2 / ex2 approximations, measured
    over every fp32 input of their ranges (see include/idw.h)."""
    lib = _lib.load()
    arr = (ctypes.c_double * 4)()
    _lib.check(lib.idw_measure_mufu_errors(int(device), arr), "idw_measure_mufu_errors")
    return {"rcp_rel": arr[0], "lg2_abs": arr[1], "ex2_rel": arr[2], "lg2_rel_outer": arr[3]}
