"""Thin ctypes binding of libtor (C ABI in include/tor.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  If the library has not been built, every call raises TorError --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

TOR_OK, TOR_EINVAL, TOR_ENOTHERM, TOR_ENOTPD, TOR_ENOMEM, TOR_EAGAIN, TOR_ETIMEOUT, \
    TOR_ECANCELED, TOR_ECUDA, TOR_ETOOBIG = range(10)
STATUS_NAMES = ["TOR_OK", "TOR_EINVAL", "TOR_ENOTHERM", "TOR_ENOTPD", "TOR_ENOMEM", "TOR_EAGAIN",
                "TOR_ETIMEOUT", "TOR_ECANCELED", "TOR_ECUDA", "TOR_ETOOBIG"]
TOR_LAYOUT_BLOCK, TOR_LAYOUT_PAIRS = 0, 1
TOR_IN_DEVICE, TOR_NO_CHECK, TOR_GRAPHS, TOR_COMPLEX_PATH, TOR_EXTENDED = 1, 2, 4, 8, 16
TOR_SESSION_SIGMA, TOR_SESSION_O = 0, 1

# Every symbol include/tor.h declares (the ABI test checks the library exports them).
EXPORTS = ["tor_config_default", "tor_create", "tor_destroy", "tor_eval", "tor_eval_batch", "tor_submit",
           "tor_poll", "tor_poll_any", "tor_cancel", "tor_strerror", "tor_last_error", "tor_plan_prefix_depth",
           "tor_set_prefix_depth", "tor_eval_units", "tor_last_times", "tor_probe_fp64", "tor_check_recip",
           "tor_eval_noalloc", "tor_autotune", "tor_autotune_batch", "tor_plan_save", "tor_plan_load", "tor_serving_stats", "tor_memory",
           "tor_session_create", "tor_session_destroy", "tor_eval_marginal", "tor_submit_marginal",
           "tor_session_marginal_matrix", "tor_eval_seq", "tor_plan_leaves", "tor_eval_range",
           "tor_eval_range_batch", "tor_sample"]
TOR_NOALLOC_MAX_N = 16


class TorError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}{': ' + what if what else ''}")


class tor_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("mem_budget", ctypes.c_size_t),
                ("prefix_depth", ctypes.c_int), ("layout", ctypes.c_int), ("flags", ctypes.c_uint),
                ("timeout_s", ctypes.c_double)]


class tor_result(ctypes.Structure):
    _fields_ = [("hi", ctypes.c_double), ("lo", ctypes.c_double), ("abs_sum", ctypes.c_double),
                ("err_est", ctypes.c_double), ("n", ctypes.c_int), ("status", ctypes.c_int),
                ("path", ctypes.c_int), ("reserved", ctypes.c_int)]


@dataclass(slots=True)
class TorResult:
    hi: float
    lo: float
    abs_sum: float
    err_est: float
    n: int
    status: int
    path: int = 0  # bit 0: real (x, p) basis (else complex); bit 1: double-double factor

    @property
    def tor(self) -> float:
        return self.hi + self.lo

    @staticmethod
    def of(r: tor_result) -> "TorResult":
        return TorResult(r.hi, r.lo, r.abs_sum, r.err_est, r.n, r.status, r.path)


_LIB = None


def library_path() -> str:
    """The built library; the environment variable TOR_LIBRARY names another build to load."""
    return os.environ.get("TOR_LIBRARY") or _build.library_path()


def load_library():
    """Load the built CUDA library; raises TorError if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise TorError(TOR_ECUDA, f"libtor is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.POINTER
    lib.tor_config_default.argtypes = [P(tor_config)]
    lib.tor_config_default.restype = None
    lib.tor_create.argtypes = [P(tor_config), P(c_void_p)]
    lib.tor_destroy.argtypes = [c_void_p]
    lib.tor_destroy.restype = None
    lib.tor_eval.argtypes = [c_void_p, c_int, c_void_p, c_int, P(tor_result)]
    lib.tor_eval_batch.argtypes = [c_void_p, c_int, P(c_int), P(c_void_p), P(c_int), P(tor_result)]
    lib.tor_eval_seq.argtypes = [c_void_p, c_int, P(c_int), P(c_void_p), P(c_int), P(tor_result), P(c_double)]
    lib.tor_submit.argtypes = [c_void_p, c_int, c_void_p, c_int, P(ctypes.c_uint64)]
    lib.tor_poll.argtypes = [c_void_p, ctypes.c_uint64, P(tor_result), c_double]
    lib.tor_poll_any.argtypes = [c_void_p, P(ctypes.c_uint64), c_int, c_double, P(c_int), P(tor_result)]
    lib.tor_cancel.argtypes = [c_void_p]
    lib.tor_strerror.argtypes = [c_int]
    lib.tor_strerror.restype = ctypes.c_char_p
    lib.tor_last_error.argtypes = [c_void_p]
    lib.tor_last_error.restype = ctypes.c_char_p
    lib.tor_plan_prefix_depth.argtypes = [c_void_p, c_int]
    lib.tor_set_prefix_depth.argtypes = [c_void_p, c_int, c_int]
    lib.tor_eval_units.argtypes = [c_void_p, c_int, c_void_p, c_int, P(c_double), c_size_t, P(tor_result)]
    lib.tor_last_times.argtypes = [c_void_p, P(c_double)]
    lib.tor_probe_fp64.argtypes = [c_int, c_double, P(c_double), P(c_double)]
    lib.tor_check_recip.argtypes = [c_int, c_int, P(c_double), P(c_double)]
    lib.tor_eval_noalloc.argtypes = [c_int, c_int, c_void_p, c_int, c_int, c_void_p, c_void_p]
    lib.tor_autotune.argtypes = [c_void_p, c_int, c_int, c_double, P(c_int)]
    lib.tor_autotune_batch.argtypes = [c_void_p, c_int, P(c_int), P(c_void_p), P(c_int), c_double, P(c_int)]
    lib.tor_plan_save.argtypes = [c_void_p, ctypes.c_char_p]
    lib.tor_plan_load.argtypes = [c_void_p, ctypes.c_char_p]
    LL = ctypes.c_longlong
    lib.tor_serving_stats.argtypes = [c_void_p, P(LL), P(LL), P(LL)]
    lib.tor_memory.argtypes = [c_void_p, P(c_size_t), P(c_size_t)]
    lib.tor_session_create.argtypes = [c_void_p, c_int, c_void_p, c_int, c_int, P(c_void_p)]
    lib.tor_session_destroy.argtypes = [c_void_p]
    lib.tor_session_destroy.restype = None
    lib.tor_session_marginal_matrix.argtypes = [c_void_p, c_int, c_void_p, c_int]
    lib.tor_eval_marginal.argtypes = [c_void_p, c_void_p, c_int, c_int, P(c_int), P(tor_result)]
    lib.tor_submit_marginal.argtypes = [c_void_p, c_void_p, c_int, c_int, P(c_int), P(ctypes.c_uint64)]
    lib.tor_sample.argtypes = [c_void_p, c_void_p, c_int, c_int, P(c_double), c_void_p, P(c_double), P(c_double)]
    lib.tor_plan_leaves.argtypes = [c_void_p, c_int]
    lib.tor_plan_leaves.restype = LL
    lib.tor_eval_range.argtypes = [c_void_p, c_int, c_void_p, c_int, LL, LL, P(tor_result)]
    lib.tor_eval_range_batch.argtypes = [c_void_p, c_int, P(c_int), P(c_void_p), P(c_int), P(LL), P(LL),
                                         P(tor_result)]
    _LIB = lib
    return lib


def tor_strerror(status: int) -> str:
    return load_library().tor_strerror(int(status)).decode()


def _host_matrix(O):
    """complex128 C-contiguous host array -> (array, n, ld)."""
    a = np.ascontiguousarray(np.asarray(O, dtype=np.complex128))
    if a.ndim != 2 or a.shape[0] != a.shape[1] or a.shape[0] % 2:
        raise TorError(TOR_EINVAL, "O must be a square 2n x 2n matrix")
    return a, a.shape[0] // 2, max(a.shape[1], 1)


def _device_matrix(O):
    """torch.cdouble CUDA tensor with unit column stride -> (tensor, n, ld, pointer)."""
    if O.dim() != 2 or O.shape[0] != O.shape[1] or O.shape[0] % 2:
        raise TorError(TOR_EINVAL, "O must be a square 2n x 2n matrix")
    if not O.is_cuda or str(O.dtype) != "torch.complex128":
        raise TorError(TOR_EINVAL, "TOR_IN_DEVICE inputs are complex128 CUDA tensors")
    if O.stride(1) != 1:
        O = O.contiguous()
    return O, O.shape[0] // 2, max(O.stride(0), 1), O.data_ptr()


class Context:
    """A libtor context (tor_create / tor_destroy)."""

    def __init__(self, device: int = 0, stream=None, mem_budget: int = 0, prefix_depth: int = -1,
                 layout: int = TOR_LAYOUT_BLOCK, flags: int = 0, timeout_s: float = 0.0):
        lib = load_library()
        cfg = tor_config()
        lib.tor_config_default(ctypes.byref(cfg))
        cfg.device = device
        cfg.stream = ctypes.c_void_p(int(stream)) if stream is not None else None
        cfg.mem_budget = mem_budget
        cfg.prefix_depth = prefix_depth
        cfg.layout = layout
        cfg.flags = flags
        cfg.timeout_s = timeout_s
        h = ctypes.c_void_p()
        st = lib.tor_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != TOR_OK:
            raise TorError(st, "tor_create: " + lib.tor_last_error(None).decode())
        self._h = h
        self._lib = lib
        self.flags = flags
        self.device = device

    @property
    def handle(self):
        if self._h is None:
            raise TorError(TOR_EINVAL, "context is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.tor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def last_error(self) -> str:
        return self._lib.tor_last_error(self.handle).decode()

    def plan_prefix_depth(self, n: int) -> int:
        return int(self._lib.tor_plan_prefix_depth(self.handle, n))

    def set_prefix_depth(self, n: int, p: int):
        st = self._lib.tor_set_prefix_depth(self.handle, n, p)
        if st != TOR_OK:
            raise TorError(st, "tor_set_prefix_depth")

    def last_times(self):
        t = (ctypes.c_double * 4)()
        self._lib.tor_last_times(self.handle, t)
        return {"intake_ms": t[0], "units_ms": t[1], "reduce_ms": t[2], "total_ms": t[3]}

    def cancel(self):
        self._lib.tor_cancel(self.handle)

    def autotune(self, n_lo: int, n_hi: int, budget_s: float = 5.0):
        """Tune the prefix depth for n in [n_lo, n_hi]; returns {n: p}."""
        k = n_hi - n_lo + 1
        chosen = (ctypes.c_int * k)()
        st = self._lib.tor_autotune(self.handle, n_lo, n_hi, budget_s, chosen)
        if st != TOR_OK:
            raise TorError(st, self.last_error() or "tor_autotune")
        return {n_lo + i: chosen[i] for i in range(k)}

    def serving_stats(self):
        s, bt, q = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        self._lib.tor_serving_stats(self.handle, ctypes.byref(s), ctypes.byref(bt), ctypes.byref(q))
        return {"served": s.value, "batches": bt.value, "queued": q.value}

    def memory(self):
        """(device bytes the context holds, its budget; 0 = none)."""
        h, b = ctypes.c_size_t(), ctypes.c_size_t()
        self._lib.tor_memory(self.handle, ctypes.byref(h), ctypes.byref(b))
        return h.value, b.value

    def save_plan(self, path: str):
        st = self._lib.tor_plan_save(self.handle, os.fsencode(path))
        if st != TOR_OK:
            raise TorError(st, "tor_plan_save")

    def load_plan(self, path: str):
        st = self._lib.tor_plan_load(self.handle, os.fsencode(path))
        if st != TOR_OK:
            raise TorError(st, "tor_plan_load")


def tor_create(**kw) -> Context:
    return Context(**kw)


def tor_destroy(ctx: Context):
    ctx.close()


def _matrix_args(ctx: Context, O):
    if ctx.flags & TOR_IN_DEVICE:
        t, n, ld, ptr = _device_matrix(O)
        return t, n, ld, ptr
    a, n, ld = _host_matrix(O)
    return a, n, ld, a.ctypes.data


def tor_eval(ctx: Context, O, check: bool = True) -> TorResult:
    """Tor of one matrix (host numpy array, or torch CUDA tensor with TOR_IN_DEVICE)."""
    keep, n, ld, ptr = _matrix_args(ctx, O)
    res = tor_result()
    st = ctx._lib.tor_eval(ctx.handle, n, ctypes.c_void_p(ptr), ld, ctypes.byref(res))
    if check and st not in (TOR_OK,):
        raise TorError(st, ctx.last_error() or "tor_eval")
    del keep
    return TorResult.of(res)


# tor_result as a numpy record (the same 48 bytes)
RESULT_DTYPE = np.dtype([("hi", "<f8"), ("lo", "<f8"), ("abs_sum", "<f8"), ("err_est", "<f8"),
                         ("n", "<i4"), ("status", "<i4"), ("path", "<i4"), ("reserved", "<i4")])
_C128 = np.dtype(np.complex128)


def _batch_args(ctx: Context, mats):
    """Marshals a batch for the C ABI: (objects to keep alive, n[], ld[], pointers[]) as
    int32 / int32 / uint64 numpy arrays.  mats is a list of 2n x 2n matrices, or one
    stacked (count, 2n, 2n) array (CUDA tensor with TOR_IN_DEVICE) of equal sizes,
    whose pointers are arithmetic: no Python work per matrix."""
    dev = bool(ctx.flags & TOR_IN_DEVICE)
    stacked = (hasattr(mats, "dim") and mats.dim() == 3) if dev else (isinstance(mats, np.ndarray) and mats.ndim == 3)
    if stacked:
        if dev:
            if not mats.is_cuda or str(mats.dtype) != "torch.complex128":
                raise TorError(TOR_EINVAL, "TOR_IN_DEVICE inputs are complex128 CUDA tensors")
            t = mats if mats.stride(2) == 1 and mats.stride(1) == mats.shape[2] else mats.contiguous()
            count, m, m2 = t.shape
            base, step = t.data_ptr(), t.stride(0) * 16
            keep = t
        else:
            keep = np.ascontiguousarray(mats, dtype=np.complex128)
            count, m, m2 = keep.shape
            base, step = keep.ctypes.data, m * m2 * 16
        if m != m2 or m % 2:
            raise TorError(TOR_EINVAL, "O must be a stack of square 2n x 2n matrices")
        ptrs = np.uint64(base) + np.arange(count, dtype=np.uint64) * np.uint64(step)
        return keep, np.full(count, m // 2, np.int32), np.full(count, max(m, 1), np.int32), ptrs
    k = len(mats)
    try:  # a list of plain arrays / tensors: one pass per attribute, no per-matrix calls into the binding
        if dev:
            ok = all(O.dim() == 2 and O.is_cuda and str(O.dtype) == "torch.complex128" and O.stride(1) == 1
                     for O in mats)
        else:
            ok = all(type(O) is np.ndarray and O.ndim == 2 and O.dtype is _C128 and O.flags.c_contiguous
                     for O in mats)
    except AttributeError:
        ok = False
    if ok:
        r = np.fromiter((O.shape[0] for O in mats), np.int64, k)
        c = np.fromiter((O.shape[1] for O in mats), np.int64, k)
        if (r != c).any() or (r % 2 != 0).any():
            raise TorError(TOR_EINVAL, "O must be a square 2n x 2n matrix")
        if dev:
            ld = np.fromiter((O.stride(0) for O in mats), np.int64, k)
            ptrs = np.fromiter((O.data_ptr() for O in mats), np.uint64, k)
        else:
            ld = r
            ptrs = np.fromiter((O.ctypes.data for O in mats), np.uint64, k)
        return mats, (r // 2).astype(np.int32), np.maximum(ld, 1).astype(np.int32), ptrs
    args = [_matrix_args(ctx, O) for O in mats]
    return (args, np.array([a[1] for a in args], np.int32), np.array([a[2] for a in args], np.int32),
            np.array([a[3] for a in args], np.uint64))


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def tor_eval_batch_arrays(ctx: Context, mats, check: bool = True) -> np.ndarray:
    """Tor of several matrices in one launch (as tor_eval_batch); the results as one
    numpy record array of RESULT_DTYPE (fields hi, lo, abs_sum, err_est, n, status,
    path), without a Python object per matrix."""
    keep, ns, lds, ptrs = _batch_args(ctx, mats)
    k = len(ns)
    res = np.zeros(k, dtype=RESULT_DTYPE)
    if k == 0:
        return res
    st = ctx._lib.tor_eval_batch(ctx.handle, k, _ptr(ns, ctypes.c_int), _ptr(ptrs, ctypes.c_void_p),
                                 _ptr(lds, ctypes.c_int), _ptr(res, tor_result))
    if check and st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_eval_batch")
    del keep
    return res


def _results(res: np.ndarray):
    return [TorResult(hi, lo, a, e, n, st, path) for hi, lo, a, e, n, st, path, _ in res.tolist()]


def tor_eval_batch(ctx: Context, mats, check: bool = True):
    """Tor of several matrices of mixed sizes in one launch; returns a list of TorResult.
    mats: a list of matrices, or one stacked (count, 2n, 2n) array / CUDA tensor."""
    if len(mats) == 0:
        return []
    return _results(tor_eval_batch_arrays(ctx, mats, check))


def tor_eval_seq(ctx: Context, mats, check: bool = True):
    """The plain path looped in C: one tor_eval per matrix, no Python between
    the calls.  Returns (list of TorResult, array of per-matrix wall ms)."""
    if len(mats) == 0:
        return [], np.zeros(0)
    keep, ns, lds, ptrs = _batch_args(ctx, mats)
    k = len(ns)
    res = np.zeros(k, dtype=RESULT_DTYPE)
    ms = np.zeros(k, dtype=np.float64)
    st = ctx._lib.tor_eval_seq(ctx.handle, k, _ptr(ns, ctypes.c_int), _ptr(ptrs, ctypes.c_void_p),
                               _ptr(lds, ctypes.c_int), _ptr(res, tor_result), _ptr(ms, ctypes.c_double))
    if check and st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_eval_seq")
    del keep
    return _results(res), ms


def tor_autotune_batch(ctx: Context, mats, budget_s: float = 10.0):
    """Tune the prefix depths of the batch's sizes for the throughput of the whole
    batch (tor_autotune_batch); returns {n: p}.  The depths stay in ctx's plan."""
    if len(mats) == 0:
        return {}
    keep, ns, lds, ptrs = _batch_args(ctx, mats)
    k = len(ns)
    chosen = np.zeros(k, dtype=np.int32)
    st = ctx._lib.tor_autotune_batch(ctx.handle, k, _ptr(ns, ctypes.c_int), _ptr(ptrs, ctypes.c_void_p),
                                     _ptr(lds, ctypes.c_int), budget_s, _ptr(chosen, ctypes.c_int))
    if st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_autotune_batch")
    del keep
    return {int(n): int(p) for n, p in zip(ns, chosen)}


def tor_eval_units(ctx: Context, O):
    """tor_eval plus the per-unit partials: returns (TorResult, p, array of shape (2^p, 3))."""
    keep, n, ld, ptr = _matrix_args(ctx, O)
    p = ctx.plan_prefix_depth(n)
    parts = np.zeros((1 << p, 3), dtype=np.float64)
    res = tor_result()
    st = ctx._lib.tor_eval_units(ctx.handle, n, ctypes.c_void_p(ptr), ld,
                                 parts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), parts.size,
                                 ctypes.byref(res))
    if st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_eval_units")
    del keep
    return TorResult.of(res), p, parts


def tor_plan_leaves(ctx: Context, n: int) -> int:
    return int(ctx._lib.tor_plan_leaves(ctx.handle, n))


def tor_eval_range(ctx: Context, O, leaf_lo: int, leaf_count: int) -> TorResult:
    """Partial Tor over reduction leaves [leaf_lo, leaf_lo + leaf_count) (one shard)."""
    keep, n, ld, ptr = _matrix_args(ctx, O)
    res = tor_result()
    st = ctx._lib.tor_eval_range(ctx.handle, n, ctypes.c_void_p(ptr), ld, leaf_lo, leaf_count, ctypes.byref(res))
    if st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_eval_range")
    del keep
    return TorResult.of(res)


def tor_eval_range_batch(ctx: Context, mats, ranges, check: bool = True):
    """One launch over a leaf range of each matrix: ranges[i] = (leaf_lo, leaf_count),
    or None for the whole matrix.  Returns a list of TorResult."""
    if len(mats) != len(ranges):
        raise ValueError("one range per matrix")
    if len(mats) == 0:
        return []
    keep, ns, lds, ptrs = _batch_args(ctx, mats)
    k = len(ns)
    los = np.array([0 if r is None else int(r[0]) for r in ranges], dtype=np.int64)
    cnts = np.array([-1 if r is None else int(r[1]) for r in ranges], dtype=np.int64)
    res = np.zeros(k, dtype=RESULT_DTYPE)
    st = ctx._lib.tor_eval_range_batch(ctx.handle, k, _ptr(ns, ctypes.c_int), _ptr(ptrs, ctypes.c_void_p),
                                       _ptr(lds, ctypes.c_int), _ptr(los, ctypes.c_longlong),
                                       _ptr(cnts, ctypes.c_longlong), _ptr(res, tor_result))
    if check and st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_eval_range_batch")
    del keep
    return _results(res)


def tor_submit(ctx: Context, O) -> int:
    a, n, ld = _host_matrix(O)
    t = ctypes.c_uint64()
    st = ctx._lib.tor_submit(ctx.handle, n, ctypes.c_void_p(a.ctypes.data), ld, ctypes.byref(t))
    if st != TOR_OK:
        raise TorError(st, "tor_submit")
    return int(t.value)


def tor_poll(ctx: Context, ticket: int, timeout_s: float = -1.0):
    """Returns (status, TorResult or None); status TOR_EAGAIN means still pending."""
    res = tor_result()
    st = ctx._lib.tor_poll(ctx.handle, ticket, ctypes.byref(res), timeout_s)
    if st in (TOR_EAGAIN,) or (st == TOR_EINVAL and res.n == 0 and res.status == 0 and res.abs_sum == 0):
        return st, None
    return st, TorResult.of(res)


def tor_check_recip(x, device: int = 0):
    """(rcp64(x), 1.0/x, rsqrt64(x), rsqrt(x)) computed on the GPU, four float64 arrays."""
    lib = load_library()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    out = np.zeros((x.size, 4), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.tor_check_recip(device, x.size, x.ctypes.data_as(dp), out.ctypes.data_as(dp))
    if st != TOR_OK:
        raise TorError(st, "tor_check_recip")
    return out[:, 0], out[:, 1], out[:, 2], out[:, 3]


def tor_poll_any(ctx: Context, tickets, timeout_s: float = -1.0):
    """Waits for whichever of `tickets` completes first.  Returns (status,
    index into tickets, TorResult); (TOR_EAGAIN, -1, None) if none did in time."""
    k = len(tickets)
    arr = (ctypes.c_uint64 * max(k, 1))(*[int(t) for t in tickets])
    idx = ctypes.c_int(-1)
    res = tor_result()
    st = ctx._lib.tor_poll_any(ctx.handle, arr, k, timeout_s, ctypes.byref(idx), ctypes.byref(res))
    if st == TOR_EAGAIN or idx.value < 0:
        return st, -1, None
    return st, idx.value, TorResult.of(res)


def tor_probe_fp64(device: int = 0, seconds: float = 0.5):
    """(DFMA per second, FP64 TFLOP/s) from the library's saturating FMA kernel."""
    lib = load_library()
    d, t = ctypes.c_double(), ctypes.c_double()
    st = lib.tor_probe_fp64(device, seconds, ctypes.byref(d), ctypes.byref(t))
    if st != TOR_OK:
        raise TorError(st, "tor_probe_fp64")
    return d.value, t.value


class Session:
    """Resident chain-rule prefix matrices O^(j) of one Gaussian state (tor_session_create)."""

    def __init__(self, ctx: Context, M, kind: int = TOR_SESSION_SIGMA):
        a, n, ld = _host_matrix(M)
        h = ctypes.c_void_p()
        st = ctx._lib.tor_session_create(ctx.handle, n, ctypes.c_void_p(a.ctypes.data), ld, kind, ctypes.byref(h))
        if st != TOR_OK:
            raise TorError(st, ctx.last_error() or "tor_session_create")
        self._h, self.ctx, self.n = h, ctx, n

    def marginal_matrix(self, j: int) -> np.ndarray:
        """The resident O^(j) (2j x 2j complex128, the context's layout)."""
        out = np.zeros((2 * j, 2 * j), dtype=np.complex128)
        st = self.ctx._lib.tor_session_marginal_matrix(self._h, j, ctypes.c_void_p(out.ctypes.data), 2 * j)
        if st != TOR_OK:
            raise TorError(st, self.ctx.last_error() or "tor_session_marginal_matrix")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.ctx._lib.tor_session_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _modes_arg(modes):
    k = len(modes)
    return k, (ctypes.c_int * max(k, 1))(*[int(x) for x in modes])


def tor_eval_marginal(ctx: Context, session: Session, j: int, modes, check: bool = True) -> TorResult:
    """Tor(O^(j)_S), S = modes (each < j)."""
    k, arr = _modes_arg(modes)
    res = tor_result()
    st = ctx._lib.tor_eval_marginal(ctx.handle, session._h, j, k, arr, ctypes.byref(res))
    if check and st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_eval_marginal")
    return TorResult.of(res)


def tor_sample(ctx: Context, session: Session, uniforms):
    """Chain-rule threshold-detector samples (tor_sample).  uniforms: (count,
    n_modes) array in [0, 1).  Returns (patterns uint8 (count, n_modes),
    probability of each pattern, chain-rule consistency max_dev)."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    if u.ndim != 2:
        raise ValueError("uniforms must be (count, n_modes)")
    count, n_modes = u.shape
    pat = np.zeros((count, n_modes), dtype=np.uint8)
    prob = np.zeros(count, dtype=np.float64)
    dev = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    st = ctx._lib.tor_sample(ctx.handle, session._h, count, n_modes, u.ctypes.data_as(dp),
                             ctypes.c_void_p(pat.ctypes.data), prob.ctypes.data_as(dp), ctypes.byref(dev))
    if st != TOR_OK:
        raise TorError(st, ctx.last_error() or "tor_sample")
    return pat, prob, dev.value


def tor_submit_marginal(ctx: Context, session: Session, j: int, modes) -> int:
    k, arr = _modes_arg(modes)
    t = ctypes.c_uint64()
    st = ctx._lib.tor_submit_marginal(ctx.handle, session._h, j, k, arr, ctypes.byref(t))
    if st != TOR_OK:
        raise TorError(st, "tor_submit_marginal")
    return int(t.value)
