"""GB300 blocked Floyd-Warshall all-pairs shortest paths (arXiv 1811.01201).

Thin Python binding of the C ABI in ``include/apsp.h`` (``libapsp.so``). Every
step of the computation runs in the library's CUDA kernels; this module only
marshals torch tensors / numpy arrays into pointers and maps status codes to
exceptions. PyTorch is used for device memory and streams only.

There is no CPU fallback: if ``libapsp.so`` is missing or fails to load, every
entry point raises.
"""

from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np
import torch

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))

APSP_OK = 0
APSP_EINVAL = -1
APSP_ENOMEM = -2
APSP_ECUDA = -3
APSP_ETIMEOUT = -4
APSP_EBUSY = -5
APSP_ECANCELLED = -6
APSP_ENOTFOUND = -7

DTYPE_AUTO = 0
DTYPE_F32 = 1
DTYPE_U16X2 = 2

FLAG_TIME_PHASES = 1
FLAG_TEST_PANEL_TIMEOUT = 0x40000000  # testing only: phase-3 panel waits expire (results wrong by design)


class ApspError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


class apsp_options(ctypes.Structure):
    _fields_ = [("bs", ctypes.c_int), ("dtype", ctypes.c_int), ("validate", ctypes.c_int), ("flags", ctypes.c_int)]


class apsp_run_info(ctypes.Structure):
    _fields_ = [("bs_used", ctypes.c_int), ("dtype_used", ctypes.c_int), ("rounds", ctypes.c_int),
                ("n_pad", ctypes.c_int), ("launches", ctypes.c_int), ("phase_launches", ctypes.c_int * 3),
                ("phase_ms", ctypes.c_float * 3)]


class apsp_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("in_flight", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("graphs_per_s", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("hbm_in_use", ctypes.c_uint64), ("hbm_peak", ctypes.c_uint64)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libapsp.so (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libapsp.so not found at {_build.LIB}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(_build.LIB)
    vp, i32p, f32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)
    c_int, c_size = ctypes.c_int, ctypes.c_size_t
    L.apsp_default_bs.argtypes = [c_int]
    L.apsp_default_bs.restype = c_int
    L.apsp_status_str.argtypes = [c_int]
    L.apsp_status_str.restype = ctypes.c_char_p
    L.apsp_fw_workspace_size.argtypes = [c_int, ctypes.POINTER(apsp_options)]
    L.apsp_fw_workspace_size.restype = c_size
    L.apsp_fw_workspace_size_for.argtypes = [c_int, ctypes.POINTER(apsp_options), vp, vp]
    L.apsp_fw_workspace_size_for.restype = c_size
    L.apsp_fw.argtypes = [vp, vp, vp, c_int, vp]
    L.apsp_fw.restype = c_int
    L.apsp_fw_ex.argtypes = [vp, vp, vp, c_int, ctypes.POINTER(apsp_options), vp, c_size,
                             ctypes.POINTER(apsp_run_info), vp]
    L.apsp_fw_ex.restype = c_int
    L.apsp_fw_host.argtypes = [vp, vp, vp, c_int, ctypes.POINTER(apsp_options), ctypes.POINTER(apsp_run_info), vp]
    L.apsp_fw_host.restype = c_int
    L.apsp_path.argtypes = [i32p, c_int, c_int, c_int, i32p, c_int]
    L.apsp_path.restype = c_int
    L.apsp_paths.argtypes = [vp, c_int, vp, c_int, vp, c_int, vp, vp]
    L.apsp_paths.restype = c_int
    L.apsp_device_status.argtypes = [c_int]
    L.apsp_device_status.restype = c_int
    if hasattr(L, "apsp_fw_batched"):
        L.apsp_fw_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.POINTER(c_int), c_int, ctypes.POINTER(apsp_options),
                                      ctypes.POINTER(c_int), vp]
        L.apsp_fw_batched.restype = c_int
        L.apsp_batched_bs.argtypes = [c_int]
        L.apsp_batched_bs.restype = c_int
        L.apsp_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(c_int), c_int, ctypes.POINTER(apsp_options),
                                        ctypes.POINTER(vp), vp]
        L.apsp_batch_create.restype = c_int
        L.apsp_batch_autotune.argtypes = [vp, ctypes.POINTER(c_int), vp]
        L.apsp_batch_autotune.restype = c_int
        L.apsp_batch_launch.argtypes = [vp, vp]
        L.apsp_batch_launch.restype = c_int
        L.apsp_batch_destroy.argtypes = [vp]
        L.apsp_batch_destroy.restype = c_int
    if hasattr(L, "apsp_autotune_bs"):
        L.apsp_autotune_bs.argtypes = [c_int, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_float), vp]
        L.apsp_autotune_bs.restype = c_int
    if hasattr(L, "apsp_fw_noalloc"):
        L.apsp_fw_noalloc.argtypes = [vp, vp, vp, c_int, ctypes.POINTER(apsp_options),
                                      ctypes.POINTER(apsp_run_info), vp]
        L.apsp_fw_noalloc.restype = c_int
        L.apsp_noalloc_scratch_bytes.argtypes = []
        L.apsp_noalloc_scratch_bytes.restype = c_size
    if hasattr(L, "apsp_serve_create"):
        L.apsp_serve_create.argtypes = [ctypes.POINTER(vp), c_size, c_int]
        L.apsp_serve_create.restype = c_int
        L.apsp_serve_submit.argtypes = [vp, vp, c_int, ctypes.POINTER(ctypes.c_uint64)]
        L.apsp_serve_submit.restype = c_int
        L.apsp_serve_submit_ex.argtypes = [vp, vp, c_int, ctypes.POINTER(apsp_options),
                                           ctypes.POINTER(ctypes.c_uint64)]
        L.apsp_serve_submit_ex.restype = c_int
        L.apsp_serve_poll.argtypes = [vp, ctypes.c_uint64, vp, vp, ctypes.POINTER(c_int), c_int]
        L.apsp_serve_poll.restype = c_int
        L.apsp_serve_stats.argtypes = [vp, ctypes.POINTER(apsp_stats)]
        L.apsp_serve_stats.restype = c_int
        L.apsp_serve_destroy.argtypes = [vp]
        L.apsp_serve_destroy.restype = c_int
    _lib = L
    return L


def status_str(status: int) -> str:
    try:
        return load().apsp_status_str(int(status)).decode()
    except Exception:  # library not loadable: still give a readable message
        return {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error", -4: "timed out",
                -5: "busy / not ready", -6: "cancelled", -7: "not found"}.get(int(status), "unknown status")


def _check(status: int, what: str):
    if status != APSP_OK:
        raise ApspError(status, what)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev_ptr(t: torch.Tensor, dtype: torch.dtype, n: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n * n:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor with n*n elements")
    return t.data_ptr()


def _opts(bs: int = 0, dtype: int = DTYPE_AUTO, validate: bool = True, flags: int = 0) -> apsp_options:
    return apsp_options(int(bs), int(dtype), 1 if validate else 0, int(flags))


def apsp_default_bs(n: int) -> int:
    return int(load().apsp_default_bs(int(n)))


def apsp_batched_bs(n: int) -> int:
    return int(load().apsp_batched_bs(int(n)))


def apsp_autotune_bs(n: int, stream=None) -> tuple[int, list[float]]:
    """apsp_autotune_bs: fastest BS in {32, 64, 128} for order n on this GPU, and the three timings (ms)."""
    best = ctypes.c_int(0)
    ms = (ctypes.c_float * 3)()
    _check(load().apsp_autotune_bs(int(n), ctypes.byref(best), ms, _stream_ptr(stream)), "apsp_autotune_bs")
    return int(best.value), [float(x) for x in ms]


def apsp_fw_workspace_size(n: int, bs: int = 0, dtype: int = DTYPE_AUTO, validate: bool = True) -> int:
    o = _opts(bs, dtype, validate)
    return int(load().apsp_fw_workspace_size(int(n), ctypes.byref(o)))


def apsp_fw_workspace_size_for(n: int, D: int, P: int, bs: int = 0, dtype: int = DTYPE_AUTO,
                               validate: bool = True) -> int:
    """apsp_fw_workspace_size_for: workspace bytes for these D and P device addresses (a D or P
    that does not start on a 16-byte boundary needs a padded working copy)."""
    o = _opts(bs, dtype, validate)
    return int(load().apsp_fw_workspace_size_for(int(n), ctypes.byref(o), ctypes.c_void_p(int(D)),
                                                 ctypes.c_void_p(int(P))))


def apsp_fw(W: torch.Tensor, D: torch.Tensor, P: torch.Tensor, stream=None) -> None:
    """apsp_fw: device tensors W, D (float32, n x n) and P (int32, n x n)."""
    n = int(W.shape[0])
    _check(load().apsp_fw(_dev_ptr(W, torch.float32, n, "W"), _dev_ptr(D, torch.float32, n, "D"),
                          _dev_ptr(P, torch.int32, n, "P"), n, _stream_ptr(stream)), "apsp_fw")


def apsp_fw_ex(W: torch.Tensor, D: torch.Tensor, P: torch.Tensor, bs: int = 0, dtype: int = DTYPE_AUTO,
               validate: bool = True, workspace: torch.Tensor | None = None, stream=None,
               flags: int = 0) -> apsp_run_info:
    """apsp_fw_ex: options, optional workspace (uint8 CUDA tensor); returns the run info."""
    n = int(W.shape[0])
    o = _opts(bs, dtype, validate, flags)
    info = apsp_run_info()
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        if not workspace.is_cuda or not workspace.is_contiguous():
            raise ValueError("workspace must be a contiguous CUDA tensor")
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(load().apsp_fw_ex(_dev_ptr(W, torch.float32, n, "W"), _dev_ptr(D, torch.float32, n, "D"),
                             _dev_ptr(P, torch.int32, n, "P"), n, ctypes.byref(o), ws_ptr, ws_bytes,
                             ctypes.byref(info), _stream_ptr(stream)), "apsp_fw_ex")
    return info


def apsp_fw_noalloc(W: torch.Tensor, D: torch.Tensor, P: torch.Tensor, bs: int = 0, dtype: int = DTYPE_AUTO,
                    validate: bool = True, stream=None) -> apsp_run_info:
    """apsp_fw_noalloc: the solve of apsp_fw_ex without any device allocation, for callers that
    cannot allocate device memory at the call site. It works in a fixed device array inside the
    library (apsp_noalloc_scratch_bytes()); calls that overlap on the GPU share it and race."""
    n = int(W.shape[0])
    o = _opts(bs, dtype, validate)
    info = apsp_run_info()
    _check(load().apsp_fw_noalloc(_dev_ptr(W, torch.float32, n, "W"), _dev_ptr(D, torch.float32, n, "D"),
                                  _dev_ptr(P, torch.int32, n, "P"), n, ctypes.byref(o), ctypes.byref(info),
                                  _stream_ptr(stream)), "apsp_fw_noalloc")
    return info


def _host_ptr(a, dtype, n: int, name: str) -> int:
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != dtype or not a.is_contiguous() or a.numel() != n * n:
            raise ValueError(f"{name} must be a contiguous host {dtype} tensor with n*n elements")
        return a.data_ptr()
    raise ValueError(f"{name} must be a host torch tensor")


def apsp_fw_host(W: torch.Tensor, D: torch.Tensor, P: torch.Tensor, bs: int = 0, dtype: int = DTYPE_AUTO,
                 validate: bool = True, stream=None, flags: int = 0) -> apsp_run_info:
    """apsp_fw_host: HOST tensors (pinned memory for speed); synchronous."""
    n = int(W.shape[0])
    o = _opts(bs, dtype, validate, flags)
    info = apsp_run_info()
    _check(load().apsp_fw_host(_host_ptr(W, torch.float32, n, "W"), _host_ptr(D, torch.float32, n, "D"),
                               _host_ptr(P, torch.int32, n, "P"), n, ctypes.byref(o), ctypes.byref(info),
                               _stream_ptr(stream)), "apsp_fw_host")
    return info


def apsp_fw_batched(Ws: Sequence[torch.Tensor], Ds: Sequence[torch.Tensor], Ps: Sequence[torch.Tensor],
                    bs: int = 0, dtype: int = DTYPE_AUTO, validate: bool = True, stream=None) -> list[int]:
    """apsp_fw_batched: lists of device tensors (graph g: n_g x n_g). Returns bs_used per graph."""
    L = load()
    count = len(Ws)
    if not (len(Ds) == len(Ps) == count):
        raise ValueError("Ws, Ds, Ps must have the same length")
    vp = ctypes.c_void_p
    w_arr, d_arr, p_arr = (vp * count)(), (vp * count)(), (vp * count)()
    n_arr, bs_arr = (ctypes.c_int * count)(), (ctypes.c_int * count)()
    for g in range(count):
        n = int(Ws[g].shape[0])
        n_arr[g] = n
        w_arr[g] = _dev_ptr(Ws[g], torch.float32, n, f"W[{g}]")
        d_arr[g] = _dev_ptr(Ds[g], torch.float32, n, f"D[{g}]")
        p_arr[g] = _dev_ptr(Ps[g], torch.int32, n, f"P[{g}]")
    o = _opts(bs, dtype, validate)
    _check(L.apsp_fw_batched(w_arr, d_arr, p_arr, n_arr, count, ctypes.byref(o), bs_arr, _stream_ptr(stream)),
           "apsp_fw_batched")
    return list(bs_arr)


class Batch:
    """apsp_batch_*: a reusable batch; launch() is one queue reset + one kernel (graph-capturable)."""

    def __init__(self, Ws: Sequence[torch.Tensor], Ds: Sequence[torch.Tensor], Ps: Sequence[torch.Tensor],
                 validate: bool = True, stream=None):
        L = load()
        count = len(Ws)
        if not (len(Ds) == len(Ps) == count):
            raise ValueError("Ws, Ds, Ps must have the same length")
        vp = ctypes.c_void_p
        w_arr, d_arr, p_arr = (vp * count)(), (vp * count)(), (vp * count)()
        n_arr = (ctypes.c_int * count)()
        for g in range(count):
            n = int(Ws[g].shape[0])
            n_arr[g] = n
            w_arr[g] = _dev_ptr(Ws[g], torch.float32, n, f"W[{g}]")
            d_arr[g] = _dev_ptr(Ds[g], torch.float32, n, f"D[{g}]")
            p_arr[g] = _dev_ptr(Ps[g], torch.int32, n, f"P[{g}]")
        o = _opts(0, DTYPE_F32, validate)
        h = vp()
        _check(L.apsp_batch_create(w_arr, d_arr, p_arr, n_arr, count, ctypes.byref(o), ctypes.byref(h),
                                   _stream_ptr(stream)), "apsp_batch_create")
        self._h = h
        self._keep = (list(Ws), list(Ds), list(Ps))  # buffers must outlive launches

    def launch(self, stream=None) -> None:
        _check(load().apsp_batch_launch(self._h, _stream_ptr(stream)), "apsp_batch_launch")

    def autotune(self, stream=None) -> list[int]:
        """apsp_batch_autotune: time the per-graph size rule and each phase-3 tile height per size
        class (n <= 64, 128, 256, 512) and keep the fastest; returns per class the chosen height
        (0 = the size rule, -1 = no graphs in the class)."""
        rows = (ctypes.c_int * 4)()
        _check(load().apsp_batch_autotune(self._h, rows, _stream_ptr(stream)), "apsp_batch_autotune")
        return [int(x) for x in rows]

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().apsp_batch_destroy(self._h), "apsp_batch_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apsp_device_status(clear: bool = False) -> int:
    """apsp_device_status: APSP_ETIMEOUT if a phase-3 CTA's bounded wait expired on the current
    device since the last clear, else APSP_OK. Synchronise the streams that ran solves first."""
    return int(load().apsp_device_status(1 if clear else 0))


def apsp_path(P: np.ndarray | torch.Tensor, i: int, j: int, cap: int | None = None) -> list[int] | None:
    """apsp_path on a host copy of P: vertex list i..j (at most cap, default n), or None if malformed."""
    if isinstance(P, torch.Tensor):
        P = P.cpu().numpy()
    P = np.ascontiguousarray(P, dtype=np.int32)
    n = int(P.shape[0])
    cap = n if cap is None else int(cap)
    out = np.empty(max(cap, 1), dtype=np.int32)
    i32p = ctypes.POINTER(ctypes.c_int32)
    cnt = load().apsp_path(P.ctypes.data_as(i32p), n, int(i), int(j), out.ctypes.data_as(i32p), cap)
    return None if cnt < 0 else [int(v) for v in out[:cnt]]


def apsp_paths(P: torch.Tensor, pairs: torch.Tensor, cap: int = 64, out: torch.Tensor | None = None,
               lens: torch.Tensor | None = None, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    """apsp_paths: walk a device P for every (i, j) row of `pairs` (int32, shape (count, 2)) on the
    GPU. Returns (out, lens): out[t, :lens[t]] are the vertices of path t, lens[t] == -1 where the
    walk fails (as apsp_path). Asynchronous on `stream`."""
    n = int(P.shape[0])
    _dev_ptr(P, torch.int32, n, "P")
    if not isinstance(pairs, torch.Tensor) or not pairs.is_cuda or pairs.dtype != torch.int32 \
            or not pairs.is_contiguous() or pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must be a contiguous CUDA int32 tensor of shape (count, 2)")
    count = int(pairs.shape[0])
    if out is None:
        out = torch.empty((count, cap), dtype=torch.int32, device=P.device)
    if lens is None:
        lens = torch.empty((count,), dtype=torch.int32, device=P.device)
    if not out.is_cuda or out.dtype != torch.int32 or not out.is_contiguous() or out.numel() != count * cap:
        raise ValueError("out must be a contiguous CUDA int32 tensor with count*cap elements")
    if not lens.is_cuda or lens.dtype != torch.int32 or not lens.is_contiguous() or lens.numel() != count:
        raise ValueError("lens must be a contiguous CUDA int32 tensor with count elements")
    _check(load().apsp_paths(P.data_ptr(), n, pairs.data_ptr(), count, out.data_ptr(), int(cap), lens.data_ptr(),
                             _stream_ptr(stream)), "apsp_paths")
    return out, lens


class Server:
    """apsp_serve_*: continuous-batching APSP server on the current device."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64):
        L = load()
        h = ctypes.c_void_p()
        _check(L.apsp_serve_create(ctypes.byref(h), int(hbm_budget_bytes), int(max_slots)), "apsp_serve_create")
        self._h = h

    def submit(self, W: np.ndarray | torch.Tensor, bs: int | None = None, dtype: int | None = None,
               flags: int = 0) -> int:
        """apsp_serve_submit, or apsp_serve_submit_ex when bs, dtype or flags are given."""
        if isinstance(W, torch.Tensor):
            W = W.detach().cpu().numpy()
        W = np.ascontiguousarray(W, dtype=np.float32)
        jid = ctypes.c_uint64()
        if bs is None and dtype is None and not flags:
            _check(load().apsp_serve_submit(self._h, W.ctypes.data, int(W.shape[0]), ctypes.byref(jid)),
                   "apsp_serve_submit")
        else:
            o = _opts(bs or 0, DTYPE_AUTO if dtype is None else dtype, True, flags)
            _check(load().apsp_serve_submit_ex(self._h, W.ctypes.data, int(W.shape[0]), ctypes.byref(o),
                                               ctypes.byref(jid)), "apsp_serve_submit_ex")
        return int(jid.value)

    def poll(self, job_id: int, n: int, timeout_ms: int = -1, want_result: bool = True, out=None):
        """Returns (D, P, bs_used) as numpy arrays, or raises ApspError (EBUSY/ETIMEOUT while pending).
        out: optional (D, P) pair of C-contiguous numpy arrays (float32, int32) of n*n elements to
        receive the result, so that a caller polling many jobs reuses its buffers."""
        if want_result and out is not None:
            D, P = out
            if not (isinstance(D, np.ndarray) and isinstance(P, np.ndarray) and D.dtype == np.float32
                    and P.dtype == np.int32 and D.size == n * n and P.size == n * n
                    and D.flags.c_contiguous and P.flags.c_contiguous):
                raise ValueError("out must be C-contiguous float32 and int32 arrays of n*n elements")
        else:
            D = np.empty((n, n), np.float32) if want_result else None
            P = np.empty((n, n), np.int32) if want_result else None
        bs = ctypes.c_int(0)
        st = load().apsp_serve_poll(self._h, int(job_id), D.ctypes.data if D is not None else None,
                                    P.ctypes.data if P is not None else None, ctypes.byref(bs), int(timeout_ms))
        _check(st, "apsp_serve_poll")
        return D, P, int(bs.value)

    def try_poll(self, job_id: int, n: int, timeout_ms: int = 0, want_result: bool = True, out=None):
        try:
            return self.poll(job_id, n, timeout_ms, want_result, out)
        except ApspError as e:
            if e.status in (APSP_EBUSY, APSP_ETIMEOUT):
                return None
            raise

    def stats(self) -> apsp_stats:
        s = apsp_stats()
        _check(load().apsp_serve_stats(self._h, ctypes.byref(s)), "apsp_serve_stats")
        return s

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load().apsp_serve_destroy(self._h), "apsp_serve_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
