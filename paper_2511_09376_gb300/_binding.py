"""ctypes marshalling for libwoodelf.so (argument conversion only, no arithmetic).

Device tensors are passed by ``data_ptr()`` together with the current torch CUDA
stream; host inputs may be numpy arrays or CPU tensors (pinned memory makes the
library's copies asynchronous).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libwoodelf.so")

FP32, TF32X3, BF16X3, BF16X6 = 0, 1, 2, 3
_PRECISION = {"fp32": FP32, "tf32x3": TF32X3, "bf16x3": BF16X3, "bf16x6": BF16X6}
_METRIC = {"shapley": 0, "banzhaf": 1}
MEM_HOST, MEM_DEVICE = 0, 1

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"{_LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")
_lib = ctypes.CDLL(_LIB_PATH)

_c = ctypes
_vp = _c.c_void_p
_lib.wdf_last_error.restype = _c.c_char_p
_lib.wdf_version.restype = _c.c_char_p
for _name, _args in {
    "wdf_ctx_create": [_c.c_int32, _c.POINTER(_vp)],
    "wdf_load_ensemble": [_vp, _c.c_int32, _c.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _c.POINTER(_vp)],
    "wdf_ensemble_info": [_vp, _vp],
    "wdf_set_background": [_vp, _vp, _c.c_int64, _c.c_int64, _c.c_int, _c.c_int, _vp],
    "wdf_explain": [_vp, _vp, _c.c_int64, _c.c_int64, _c.c_int, _vp, _c.c_int64, _vp],
    "wdf_explain_interactions": [_vp, _vp, _c.c_int64, _c.c_int64, _vp, _c.c_int64, _vp],
    "wdf_background_counts": [_vp, _vp, _c.c_int64, _c.c_int64, _vp, _vp],
    "wdf_set_background_counts": [_vp, _vp, _c.c_int64, _c.c_int, _vp],
    "wdf_expected_value": [_vp, _c.POINTER(_c.c_double), _vp],
    "wdf_global_attribution": [_vp, _vp, _c.c_int64, _c.c_int64, _c.c_int32, _vp, _vp, _vp],
    "wdf_global_attribution_noalloc": [_c.c_int32, _vp, _c.c_int64, _c.c_int64, _c.c_int32, _vp, _vp, _vp],
    "wdf_debug_leaf_hist": [_vp, _vp, _c.c_int64],
    "wdf_batch_create": [_vp, _c.c_int32, _vp, _c.POINTER(_vp)],
    "wdf_batch_explain": [_vp, _c.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "wdf_batch_autotune": [_vp, _c.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _c.c_int32, _c.c_char_p, _vp],
    "wdf_batch_tile_rows": [_vp, _c.c_int32, _c.POINTER(_c.c_int32)],
    "wdf_debug_pair_table": [_vp, _c.c_int32, _vp, _c.c_int, _vp],
    "wdf_set_metric": [_vp, _c.c_int],
}.items():
    getattr(_lib, _name).argtypes = _args
    getattr(_lib, _name).restype = _c.c_int
_lib.wdf_background_counts_size.argtypes = [_vp]
_lib.wdf_background_counts_size.restype = _c.c_int64
_lib.wdf_launch_count.argtypes = []
_lib.wdf_launch_count.restype = _c.c_int64
_lib.wdf_ctx_destroy.argtypes = [_vp]
_lib.wdf_ctx_destroy.restype = None
_lib.wdf_ensemble_destroy.argtypes = [_vp]
_lib.wdf_ensemble_destroy.restype = None
_lib.wdf_batch_destroy.argtypes = [_vp]
_lib.wdf_batch_destroy.restype = None
_lib.wdf_explain_timing.argtypes = [_c.c_int32]
_lib.wdf_explain_timing_read.argtypes = [_c.POINTER(_c.c_double), _c.POINTER(_c.c_int64)]
_lib.wdf_debug_contract_wait_limit.argtypes = [_c.c_int32]
_lib.wdf_debug_contract_wait_limit.restype = None


class WdfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"wdf status {status}: {msg}")
        self.status = status


class _Info(_c.Structure):
    _fields_ = [("n_features", _c.c_int32), ("n_trees", _c.c_int32), ("depth", _c.c_int32),
                ("n_live_leaves", _c.c_int32), ("n_signatures", _c.c_int32), ("has_background", _c.c_int32),
                ("device_bytes", _c.c_int64)]


def _check(rc):
    if rc != 0:
        raise WdfError(rc, _lib.wdf_last_error().decode(errors="replace"))


def library_path() -> str:
    return _LIB_PATH


def launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(_lib.wdf_launch_count())


def explain_timing(enable: bool) -> None:
    """Bracket every later consumer-kernel launch of wdf_explain with CUDA events (True)
    or stop (False); either forgets the launches timed so far."""
    _check(_lib.wdf_explain_timing(1 if enable else 0))


def explain_timing_read():
    """(summed milliseconds, launches) of the consumer-kernel launches timed since the
    last read; waits for them."""
    ms, n = _c.c_double(0.0), _c.c_int64(0)
    _check(_lib.wdf_explain_timing_read(_c.byref(ms), _c.byref(n)))
    return float(ms.value), int(n.value)


def version() -> str:
    return _lib.wdf_version().decode()


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return _vp(torch.cuda.current_stream().cuda_stream)
        return _vp(0)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


class Context:
    def __init__(self, device: int = 0):
        h = _vp()
        _check(_lib.wdf_ctx_create(int(device), _c.byref(h)))
        self.handle = h
        self.device = int(device)

    def close(self):
        if self.handle:
            _lib.wdf_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    def close(self):
        if self.handle:
            _lib.wdf_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return ensemble_info(self)


def ctx_create(device: int = 0) -> Context:
    return Context(device)


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def load_ensemble(ctx: Context, ens) -> Ensemble:
    """ens: any object with n_features, tree_offset, feature, threshold, left, right, value."""
    off = _np(ens.tree_offset, np.int64)
    arrs = [_np(ens.feature, np.int32), _np(ens.threshold, np.float32), _np(ens.left, np.int32),
            _np(ens.right, np.int32), _np(ens.value, np.float32)]
    h = _vp()
    _check(_lib.wdf_load_ensemble(ctx.handle, int(ens.n_features), int(off.shape[0] - 1), off.ctypes.data,
                                  *[a.ctypes.data for a in arrs], _c.byref(h)))
    return Ensemble(ctx, h)


def ensemble_info(e: Ensemble) -> dict:
    info = _Info()
    _check(_lib.wdf_ensemble_info(e.handle, _c.byref(info)))
    return {k: getattr(info, k) for k, _ in _Info._fields_}


def _matrix(x):
    """(pointer, rows, leading dim, memkind, keepalive) of a row-major float32 matrix."""
    torch = _torch()
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float32 or x.dim() != 2 or (x.numel() > 0 and x.stride(1) != 1):
            raise ValueError("expected a 2-D float32 tensor with unit column stride")
        kind = MEM_DEVICE if x.is_cuda else MEM_HOST
        return x.data_ptr(), x.shape[0], max(x.stride(0), x.shape[1]), kind, x
    a = np.asarray(x)
    if a.dtype != np.float32 or a.ndim != 2 or a.strides[1] != 4 or a.strides[0] % 4:
        a = np.ascontiguousarray(a, dtype=np.float32)
    return a.ctypes.data, a.shape[0], a.strides[0] // 4, MEM_HOST, a


def set_background(e: Ensemble, B, precision="fp32", stream=None) -> None:
    p, m, ld, kind, keep = _matrix(B)
    prec = _PRECISION[precision] if isinstance(precision, str) else int(precision)
    _check(_lib.wdf_set_background(e.handle, _vp(p), int(m), int(ld), kind, prec, _stream_handle(stream)))
    del keep


def background_counts_size(e: Ensemble) -> int:
    return int(_lib.wdf_background_counts_size(e.handle))


def background_counts(e: Ensemble, B, counts=None, stream=None):
    """Joint pattern counts of the background rows B (a device tensor), ADDED into counts
    (a device uint32 tensor of background_counts_size elements; zeros when None)."""
    torch = _torch()
    p, m, ld, kind, keep = _matrix(B)
    if kind != MEM_DEVICE:
        raise ValueError("background shards take rows in device memory")
    size = int(_lib.wdf_background_counts_size(e.handle))
    if counts is None:
        counts = torch.zeros(size, dtype=torch.int32, device=B.device)
    if not (counts.is_cuda and counts.dtype in (torch.int32, torch.uint32) and counts.numel() == size
            and counts.is_contiguous()):
        raise ValueError(f"counts must be a contiguous CUDA int32/uint32 tensor of {size} elements")
    _check(_lib.wdf_background_counts(e.handle, _vp(p), int(m), int(ld), _vp(counts.data_ptr()),
                                      _stream_handle(stream)))
    del keep
    return counts


def set_background_counts(e: Ensemble, counts, m_total: int, precision="fp32", stream=None) -> None:
    """Finish the background from summed shard counts of m_total rows in total."""
    prec = _PRECISION[precision] if isinstance(precision, str) else int(precision)
    _check(_lib.wdf_set_background_counts(e.handle, _vp(counts.data_ptr()), int(m_total), prec,
                                          _stream_handle(stream)))


def explain(e: Ensemble, C, out=None, stream=None):
    """phi (n x F float32).  Device tensor in -> device tensor out (asynchronous on the
    stream); host array in -> host array out."""
    p, n, ld, kind, keep = _matrix(C)
    F = ensemble_info(e)["n_features"]
    torch = _torch()
    if out is None:
        if kind == MEM_DEVICE:
            out = torch.empty((n, F), dtype=torch.float32, device=C.device)
        elif isinstance(C, torch.Tensor):
            out = torch.empty((n, F), dtype=torch.float32, pin_memory=C.is_pinned())
        else:
            out = np.empty((n, F), dtype=np.float32)
    op, on, old, okind, okeep = _matrix(out)
    if okind != kind or on != n:
        raise ValueError("phi must live in the same memory kind as C and have n rows")
    _check(_lib.wdf_explain(e.handle, _vp(p), int(n), int(ld), kind, _vp(op), int(old), _stream_handle(stream)))
    del keep, okeep
    return out


def explain_interactions(e: Ensemble, C, out=None, stream=None):
    """Pairwise interaction values (n x F x F float32, symmetric, zero diagonal) of a
    device tensor of consumer rows, for the ensemble's metric; device tensor out."""
    p, n, ld, kind, keep = _matrix(C)
    if kind != MEM_DEVICE:
        raise ValueError("interaction values take consumer rows in device memory")
    F = ensemble_info(e)["n_features"]
    torch = _torch()
    if out is None:
        out = torch.empty((n, F, F), dtype=torch.float32, device=C.device)
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float32 and out.dim() == 3
            and tuple(out.shape) == (n, F, F) and out.stride(2) == 1 and out.stride(1) == F):
        raise ValueError("out must be a float32 CUDA tensor of shape (n, F, F), rows of F*F contiguous floats")
    ldo = out.stride(0) if n > 0 else F * F
    _check(_lib.wdf_explain_interactions(e.handle, _vp(p), int(n), int(ld), _vp(out.data_ptr()), int(ldo),
                                         _stream_handle(stream)))
    del keep
    return out


def expected_value(e: Ensemble, stream=None) -> float:
    v = _c.c_double(0.0)
    _check(_lib.wdf_expected_value(e.handle, _c.byref(v), _stream_handle(stream)))
    return v.value


def global_attribution(ctx: Context, phi, stream=None):
    """(mean |phi|, mean phi) per feature as FP64 device tensors."""
    torch = _torch()
    if not (isinstance(phi, torch.Tensor) and phi.is_cuda and phi.dtype == torch.float32 and phi.stride(1) == 1):
        raise ValueError("phi must be a float32 CUDA tensor with unit column stride")
    n, F = phi.shape
    ma = torch.empty(F, dtype=torch.float64, device=phi.device)
    mn = torch.empty(F, dtype=torch.float64, device=phi.device)
    _check(_lib.wdf_global_attribution(ctx.handle, _vp(phi.data_ptr()), int(n), int(phi.stride(0)), int(F),
                                       _vp(ma.data_ptr()), _vp(mn.data_ptr()), _stream_handle(stream)))
    return ma, mn


def global_attribution_noalloc(phi, stream=None):
    """global_attribution without device allocation (fixed 2 MiB scratch inside the
    library; see include/woodelf.h for its size limit and ordering rule)."""
    torch = _torch()
    if not (isinstance(phi, torch.Tensor) and phi.is_cuda and phi.dtype == torch.float32 and phi.stride(1) == 1):
        raise ValueError("phi must be a float32 CUDA tensor with unit column stride")
    n, F = phi.shape
    ma = torch.empty(F, dtype=torch.float64, device=phi.device)
    mn = torch.empty(F, dtype=torch.float64, device=phi.device)
    _check(_lib.wdf_global_attribution_noalloc(int(phi.device.index or 0), _vp(phi.data_ptr()), int(n),
                                               int(phi.stride(0)), int(F), _vp(ma.data_ptr()), _vp(mn.data_ptr()),
                                               _stream_handle(stream)))
    return ma, mn


def debug_leaf_hist(e: Ensemble) -> np.ndarray:
    info = ensemble_info(e)
    T, D = info["n_trees"], info["depth"]
    out = np.zeros((T, 1 << D, 1 << D), dtype=np.uint32)
    _check(_lib.wdf_debug_leaf_hist(e.handle, _vp(out.ctypes.data), int(out.size)))
    return out


def debug_pair_table(ctx: Context, first, metric="shapley") -> np.ndarray:
    f = np.ascontiguousarray(first, dtype=np.int32)
    D = int(f.shape[0])
    out = np.zeros((1 << D, D << D), dtype=np.float64)
    _check(_lib.wdf_debug_pair_table(ctx.handle, D, _vp(f.ctypes.data), _METRIC[metric], _vp(out.ctypes.data)))
    return out


def debug_contract_wait_limit(polls: int) -> None:
    """Test hook: poll limit of the first mbarrier wait of every CTA of later tensor-core
    contractions (0 restores the normal limit)."""
    _lib.wdf_debug_contract_wait_limit(int(polls))


def set_metric(e: Ensemble, metric="shapley") -> None:
    """'shapley' (default) or 'banzhaf'; the background must be set again afterwards."""
    _check(_lib.wdf_set_metric(e.handle, _METRIC[metric]))


class Batch:
    def __init__(self, ctx: Context, ensembles, handle):
        self.ctx = ctx
        self.ensembles = list(ensembles)  # kept alive with the batch
        self.handle = handle

    def close(self):
        if self.handle:
            _lib.wdf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_create(ctx: Context, ensembles) -> Batch:
    hs = (_vp * len(ensembles))(*[e.handle for e in ensembles])
    h = _vp()
    _check(_lib.wdf_batch_create(ctx.handle, len(ensembles), hs, _c.byref(h)))
    return Batch(ctx, ensembles, h)


def _batch_args(batch, requests, outs):
    """requests: list of (ensemble index, C device tensor); outs: phi tensors or None."""
    torch = _torch()
    k = len(requests)
    if outs is None:
        outs = []
        for i, C in requests:
            F = ensemble_info(batch.ensembles[i])["n_features"]
            outs.append(torch.empty((C.shape[0], F), dtype=torch.float32, device=C.device))
    for (i, C), o in zip(requests, outs):
        if not (C.is_cuda and o.is_cuda and C.dtype == torch.float32 and o.dtype == torch.float32
                and (C.numel() == 0 or C.stride(1) == 1) and (o.numel() == 0 or o.stride(1) == 1)):
            raise ValueError("batch requests take float32 CUDA tensors with unit column stride")
    idx = np.array([i for i, _ in requests], dtype=np.int32)
    cp = np.array([C.data_ptr() for _, C in requests], dtype=np.uint64)
    pp = np.array([o.data_ptr() for o in outs], dtype=np.uint64)
    n = np.array([C.shape[0] for _, C in requests], dtype=np.int64)
    ldc = np.array([max(C.stride(0), C.shape[1]) for _, C in requests], dtype=np.int64)
    ldp = np.array([max(o.stride(0), o.shape[1]) for o in outs], dtype=np.int64)
    arrs = (idx, cp, n, ldc, pp, ldp)
    return k, arrs, outs


def batch_explain(batch: Batch, requests, outs=None, stream=None):
    """One graph launch for all requests; returns the phi tensors (asynchronous)."""
    k, (idx, cp, n, ldc, pp, ldp), outs = _batch_args(batch, requests, outs)
    _check(_lib.wdf_batch_explain(batch.handle, k, _vp(idx.ctypes.data), _vp(cp.ctypes.data), _vp(n.ctypes.data),
                                  _vp(ldc.ctypes.data), _vp(pp.ctypes.data), _vp(ldp.ctypes.data),
                                  _stream_handle(stream)))
    return outs


def batch_autotune(batch: Batch, requests, outs=None, reps=3, cache_path=None, stream=None):
    k, (idx, cp, n, ldc, pp, ldp), outs = _batch_args(batch, requests, outs)
    _check(_lib.wdf_batch_autotune(batch.handle, k, _vp(idx.ctypes.data), _vp(cp.ctypes.data), _vp(n.ctypes.data),
                                   _vp(ldc.ctypes.data), _vp(pp.ctypes.data), _vp(ldp.ctypes.data), int(reps),
                                   cache_path.encode() if cache_path else None, _stream_handle(stream)))
    return outs


def batch_tile_rows(batch: Batch, depth: int) -> int:
    v = _c.c_int32(0)
    _check(_lib.wdf_batch_tile_rows(batch.handle, int(depth), _c.byref(v)))
    return int(v.value)


_lib.wdf_server_create.argtypes = [_vp, _c.c_int32, _vp, _c.c_int64, _c.c_int32, _c.c_int32, _c.POINTER(_vp)]
_lib.wdf_server_submit.argtypes = [_vp, _c.c_int32, _vp, _c.c_int64, _c.c_int64, _vp, _c.c_int64,
                                   _c.POINTER(_c.c_uint64)]
_lib.wdf_server_wait.argtypes = [_vp, _c.c_uint64, _c.c_int64]
_lib.wdf_server_poll.argtypes = [_vp, _c.c_uint64, _c.POINTER(_c.c_int32)]
_lib.wdf_server_request_ms.argtypes = [_vp, _c.c_uint64, _c.POINTER(_c.c_double)]
_lib.wdf_server_stats.argtypes = [_vp, _vp]
_lib.wdf_server_reset_stats.argtypes = [_vp]
for _f in ("wdf_server_create", "wdf_server_submit", "wdf_server_wait", "wdf_server_poll", "wdf_server_stats",
           "wdf_server_reset_stats", "wdf_server_request_ms"):
    getattr(_lib, _f).restype = _c.c_int
_lib.wdf_server_destroy.argtypes = [_vp]
_lib.wdf_server_destroy.restype = None


class _ServingStats(_c.Structure):
    _fields_ = [("submitted", _c.c_int64), ("completed", _c.c_int64), ("queued", _c.c_int64), ("waves", _c.c_int64),
                ("rows_completed", _c.c_int64), ("p50_ms", _c.c_double), ("p99_ms", _c.c_double),
                ("max_ms", _c.c_double), ("rows_per_s", _c.c_double), ("device_bytes_in_use", _c.c_int64),
                ("device_budget", _c.c_int64)]


class Server:
    def __init__(self, ctx, ensembles, handle):
        self.ctx = ctx
        self.ensembles = list(ensembles)
        self.handle = handle
        self._live = {}  # ticket -> (C, phi) kept alive until the request is done

    def close(self):
        if self.handle:
            _lib.wdf_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_create(ctx: Context, ensembles, device_budget_bytes: int, n_slots: int = 3, max_wave: int = 32) -> Server:
    hs = (_vp * len(ensembles))(*[e.handle for e in ensembles])
    h = _vp()
    _check(_lib.wdf_server_create(ctx.handle, len(ensembles), hs, int(device_budget_bytes), int(n_slots),
                                  int(max_wave), _c.byref(h)))
    return Server(ctx, ensembles, h)


def server_submit(server: Server, ensemble_index: int, C, phi=None):
    """Queue one request (host float32 rows, any row stride).  Returns (ticket, phi array
    filled when done); phi may be a row-strided float32 view."""
    C = np.asarray(C)
    if C.dtype != np.float32 or C.ndim != 2 or C.strides[1] != 4 or C.strides[0] % 4:
        C = np.ascontiguousarray(C, dtype=np.float32)
    F = ensemble_info(server.ensembles[ensemble_index])["n_features"]
    if phi is None:
        phi = np.empty((C.shape[0], F), dtype=np.float32)
    if phi.dtype != np.float32 or phi.ndim != 2 or phi.strides[1] != 4 or phi.strides[0] % 4:
        raise ValueError("phi must be a float32 matrix with unit column stride")
    t = _c.c_uint64(0)
    _check(_lib.wdf_server_submit(server.handle, int(ensemble_index), _vp(C.ctypes.data), int(C.shape[0]),
                                  int(max(C.strides[0] // 4, C.shape[1])), _vp(phi.ctypes.data),
                                  int(max(phi.strides[0] // 4, phi.shape[1])), _c.byref(t)))
    server._live[t.value] = (C, phi)
    return t.value, phi


def server_wait(server: Server, ticket: int, timeout_ms: int = 60_000) -> None:
    _check(_lib.wdf_server_wait(server.handle, _c.c_uint64(ticket), int(timeout_ms)))
    server._live.pop(ticket, None)


def server_poll(server: Server, ticket: int) -> bool:
    d = _c.c_int32(0)
    _check(_lib.wdf_server_poll(server.handle, _c.c_uint64(ticket), _c.byref(d)))
    if d.value:
        server._live.pop(ticket, None)
    return bool(d.value)


def server_request_ms(server: Server, ticket: int) -> float:
    """Latency (submit to completion, ms) of a completed request."""
    v = _c.c_double(0.0)
    _check(_lib.wdf_server_request_ms(server.handle, _c.c_uint64(ticket), _c.byref(v)))
    return v.value


def server_stats(server: Server) -> dict:
    st = _ServingStats()
    _check(_lib.wdf_server_stats(server.handle, _c.byref(st)))
    return {k: getattr(st, k) for k, _ in _ServingStats._fields_}


def server_reset_stats(server: Server) -> None:
    _check(_lib.wdf_server_reset_stats(server.handle))


_lib.wdf_set_covers.argtypes = [_vp, _vp]
_lib.wdf_set_covers.restype = _c.c_int
_lib.wdf_set_path_dependent.argtypes = [_vp, _c.c_int, _vp]
_lib.wdf_set_path_dependent.restype = _c.c_int


def set_covers(e: Ensemble, cover) -> None:
    """Node covers (one per input node, like the node arrays) for path-dependent values."""
    cv = np.ascontiguousarray(cover, dtype=np.float64)
    _check(_lib.wdf_set_covers(e.handle, _vp(cv.ctypes.data)))


def set_path_dependent(e: Ensemble, precision="fp32", stream=None) -> None:
    """Use the covers' path-dependent frequencies instead of a background."""
    prec = _PRECISION[precision] if isinstance(precision, str) else int(precision)
    _check(_lib.wdf_set_path_dependent(e.handle, prec, _stream_handle(stream)))
