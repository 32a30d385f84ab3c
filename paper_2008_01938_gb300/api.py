"""PyTorch-facing wrappers of the C ABI (same names as the C entry points).

Marshalling only: tensors are checked for device, dtype and contiguity, then
their data pointers and the current CUDA stream are passed to the library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native
from .native import check


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, name, numel=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")


def _cost(cost) -> int:
    if cost in ("i32", "int32", native.DP_COST_I32):
        return native.DP_COST_I32
    if cost in ("i64", "int64", native.DP_COST_I64):
        return native.DP_COST_I64
    raise ValueError(f"unknown cost type {cost!r}")


def _op(op) -> int:
    if op in ("min", native.DP_OP_MIN):
        return native.DP_OP_MIN
    if op in ("add", "+", native.DP_OP_ADD_MOD32):
        return native.DP_OP_ADD_MOD32
    raise ValueError(f"unknown operator {op!r}")


def sync_status(stream=None, status=None) -> None:
    """Waits for the stream and raises DpError if the device reported one."""
    lib = native.load()
    check(lib.dp_sync_status(_stream_ptr(stream), _ptr(status)))


# ---------------------------------------------------------------------------
# MCM
# ---------------------------------------------------------------------------

def mcm_solve(p, cost="i32", m=None, s=None, status=None, stream=None):
    """Fills the MCM tables of the chain with dims ``p`` (CUDA int32, n+1).
    Returns (m, s): m int32 or int64 (n, n), s int16 (n, n).  Asynchronous on
    the current stream; call sync_status() to learn device-side errors."""
    torch = _torch()
    lib = native.load()
    ct = _cost(cost)
    _need(p, torch.int32, "p")
    n = p.numel() - 1
    mdt = torch.int32 if ct == native.DP_COST_I32 else torch.int64
    if m is None:
        m = torch.empty((n, n), dtype=mdt, device=p.device)
    if s is None:
        s = torch.empty((n, n), dtype=torch.int16, device=p.device)
    _need(m, mdt, "m", n * n)
    _need(s, torch.int16, "s", n * n)
    if status is not None:
        _need(status, torch.int32, "status", 1)
    check(lib.mcm_solve(_ptr(p), n, ct, _ptr(m), _ptr(s), _ptr(status), _stream_ptr(stream)))
    return m, s


def interval_dp_solve(p, w, cost="i32", m=None, s=None, status=None, stream=None):
    """Interval DP with a user weight: Eq. (2) with
    f(l, r) = l + r + p[i] p[k+1] p[j+1] + w[i][j].  ``p`` CUDA int32 (n+1),
    entries >= 0 (zeros drop the rank-1 term); ``w`` CUDA int32 (n, n), only
    entries with i < j read, each >= 0.  Int32 costs only (cost="i64" is
    refused by the library).  Returns (m, s) like mcm_solve."""
    torch = _torch()
    lib = native.load()
    ct = _cost(cost)
    _need(p, torch.int32, "p")
    n = p.numel() - 1
    mdt = torch.int32 if ct == native.DP_COST_I32 else torch.int64
    _need(w, mdt, "w", n * n)
    if m is None:
        m = torch.empty((n, n), dtype=mdt, device=p.device)
    if s is None:
        s = torch.empty((n, n), dtype=torch.int16, device=p.device)
    _need(m, mdt, "m", n * n)
    _need(s, torch.int16, "s", n * n)
    if status is not None:
        _need(status, torch.int32, "status", 1)
    check(lib.interval_dp_solve(_ptr(p), _ptr(w), n, ct, _ptr(m), _ptr(s), _ptr(status), _stream_ptr(stream)))
    return m, s


def mcm_solve_noalloc(p, m, s, status, stream=None):
    """mcm_solve for int32 costs through the entry point that allocates
    nothing: the caller passes every buffer (p int32 n+1, m int32 and s int16
    of n*n, status int32 holding 0), n <= 1024."""
    torch = _torch()
    lib = native.load()
    _need(p, torch.int32, "p")
    n = p.numel() - 1
    _need(m, torch.int32, "m", n * n)
    _need(s, torch.int16, "s", n * n)
    _need(status, torch.int32, "status", 1)
    check(lib.mcm_solve_noalloc(_ptr(p), n, _ptr(m), _ptr(s), _ptr(status), _stream_ptr(stream)))
    return m, s


def mcm_traceback(s, steps=None, status=None, stream=None):
    """Optimal parenthesisation from a split table (CUDA int16 n x n, as
    written by mcm_solve): int32 (n-1, 3) products (i, k, j) in post-order."""
    torch = _torch()
    lib = native.load()
    _need(s, torch.int16, "s")
    n = int(s.shape[0]) if s.dim() == 2 else int(round(s.numel() ** 0.5))
    if n * n != s.numel():
        raise ValueError("s must hold n*n entries")
    if steps is None:
        steps = torch.empty((max(n - 1, 0), 3), dtype=torch.int32, device=s.device)
    _need(steps, torch.int32, "steps", 3 * max(n - 1, 0))
    if status is not None:
        _need(status, torch.int32, "status", 1)
    check(lib.mcm_traceback(_ptr(s), n, _ptr(steps), _ptr(status), _stream_ptr(stream)))
    return steps


def mcm_solve_host(p, cost="i32", m=None, s=None, stream=None):
    """Host-buffer form: numpy arrays or torch CPU tensors in and out.

    When m and s are page-locked (torch ``pin_memory()``, cudaHostAlloc) the
    kernel writes the tables straight into them; other buffers are filled by
    a copy after the solve."""
    lib = native.load()
    ct = _cost(cost)
    p = np.ascontiguousarray(np.asarray(p, dtype=np.int32)) if not hasattr(p, "data_ptr") else p
    n = (p.size if isinstance(p, np.ndarray) else p.numel()) - 1
    mdt = np.int32 if ct == native.DP_COST_I32 else np.int64
    if m is None:
        m = np.empty((n, n), dtype=mdt)
    if s is None:
        s = np.empty((n, n), dtype=np.int16)

    def host_buf(x, dt, name, count):
        if isinstance(x, np.ndarray):
            ok = x.dtype == dt and x.flags.c_contiguous and x.size == count
        else:
            tdt = {np.int16: "int16", np.int32: "int32", np.int64: "int64"}[dt]
            ok = (x.device.type == "cpu" and x.is_contiguous() and x.numel() == count
                  and x.dtype == getattr(_torch(), tdt))
        if not ok:
            raise ValueError(f"{name} must be a contiguous host {np.dtype(dt).name} buffer of {count} entries")

    host_buf(p, np.int32, "p", n + 1)
    host_buf(m, mdt, "m", n * n)
    host_buf(s, np.int16, "s", n * n)

    def hp(x):
        return ctypes.c_void_p(x.ctypes.data) if isinstance(x, np.ndarray) else ctypes.c_void_p(x.data_ptr())

    check(lib.mcm_solve_host(hp(p), n, ct, hp(m), hp(s), _stream_ptr(stream)))
    return m, s


class McmPlan:
    """Batched MCM plan: diagonal-ordered work queue + device workspace for a
    fixed list of chain lengths (mcm_plan_create / mcm_solve_batched)."""

    def __init__(self, ns, cost="i64"):
        lib = native.load()
        self.cost = _cost(cost)
        arr = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
        self.ns = arr
        h = ctypes.c_void_p()
        check(lib.mcm_plan_create(int(arr.size), ctypes.c_void_p(arr.ctypes.data), self.cost, ctypes.byref(h)))
        self._h = h

    @property
    def ntasks(self) -> int:
        return int(native.load().dp_mcm_plan_tasks(self._h))

    def solve(self, p_all, p_off, tab_off, m_all, s_all, status=None, stream=None):
        torch = _torch()
        lib = native.load()
        _need(p_all, torch.int32, "p_all")
        _need(p_off, torch.int64, "p_off", self.ns.size)
        _need(tab_off, torch.int64, "tab_off", self.ns.size)
        _need(m_all, torch.int32 if self.cost == native.DP_COST_I32 else torch.int64, "m_all")
        _need(s_all, torch.int16, "s_all")
        check(lib.mcm_solve_batched(self._h, _ptr(p_all), _ptr(p_off), _ptr(tab_off), _ptr(m_all), _ptr(s_all),
                                    _ptr(status), _stream_ptr(stream)))

    def autotune(self, p_all, p_off, tab_off, m_all, s_all, status=None, stream=None):
        """mcm_plan_autotune: time the candidate configurations on these
        buffers, keep the fastest (the tables hold the solution afterwards)."""
        check(native.load().mcm_plan_autotune(self._h, _ptr(p_all), _ptr(p_off), _ptr(tab_off), _ptr(m_all),
                                              _ptr(s_all), _ptr(status), _stream_ptr(stream)))
        return self.config()

    def config(self):
        """(levels per bulk task, resident blocks per SM; 0 = occupancy limit)"""
        lpp, bps = ctypes.c_int32(), ctypes.c_int32()
        check(native.load().mcm_plan_config(self._h, ctypes.byref(lpp), ctypes.byref(bps)))
        return int(lpp.value), int(bps.value)

    def destroy(self):
        if getattr(self, "_h", None):
            native.load().mcm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# S-DP
# ---------------------------------------------------------------------------

def sdp_solve(st, offsets, op="min", n=None, status=None, stream=None):
    """Fills the S-DP table ``st`` (CUDA int32 tensor holding uint32 bit
    patterns; st[0 .. a_1-1] preset) in place for the given offsets."""
    torch = _torch()
    lib = native.load()
    _need(st, torch.int32, "st")
    a = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    n = st.numel() if n is None else int(n)
    check(lib.sdp_solve(_ptr(st), n, ctypes.c_void_p(a.ctypes.data), int(a.size), _op(op), _ptr(status),
                        _stream_ptr(stream)))
    return st


def sdp_solve_host(st, offsets, op="min", stream=None):
    """Host form: ``st`` holds the n table words (preset in front) and is
    filled in place.  It is a contiguous numpy uint32 array or a contiguous
    torch CPU tensor of 32-bit integers; a page-locked one (``pin_memory()``)
    is written by the kernel directly when the window fits on chip."""
    lib = native.load()
    if isinstance(st, np.ndarray):
        if st.dtype != np.uint32 or not st.flags.c_contiguous:
            raise TypeError("st must be a contiguous numpy uint32 array")
        ptr, n = st.ctypes.data, int(st.size)
    else:
        torch = _torch()
        dts = [torch.int32] + ([torch.uint32] if hasattr(torch, "uint32") else [])
        if st.device.type != "cpu" or not st.is_contiguous() or st.dtype not in dts:
            raise TypeError("st must be a contiguous CPU tensor of 32-bit integers")
        ptr, n = st.data_ptr(), int(st.numel())
    a = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    check(lib.sdp_solve_host(ctypes.c_void_p(ptr), n, ctypes.c_void_p(a.ctypes.data),
                             int(a.size), _op(op), _stream_ptr(stream)))
    return st


class SdpPlan:
    """Batched S-DP plan (one thread block per instance, one launch)."""

    def __init__(self, ns, offsets_list, op="min"):
        lib = native.load()
        self.ns = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
        ks = np.ascontiguousarray(np.asarray([len(o) for o in offsets_list], dtype=np.int32))
        allo = np.ascontiguousarray(np.concatenate([np.asarray(o, dtype=np.int32) for o in offsets_list])
                                    if len(offsets_list) else np.zeros(1, np.int32))
        h = ctypes.c_void_p()
        check(lib.sdp_plan_create(int(self.ns.size), ctypes.c_void_p(self.ns.ctypes.data),
                                  ctypes.c_void_p(ks.ctypes.data), ctypes.c_void_p(allo.ctypes.data), _op(op),
                                  ctypes.byref(h)))
        self._h = h

    def solve(self, st_all, st_off, status=None, stream=None):
        torch = _torch()
        lib = native.load()
        _need(st_all, torch.int32, "st_all")
        _need(st_off, torch.int64, "st_off", self.ns.size)
        check(lib.sdp_solve_batched(self._h, _ptr(st_all), _ptr(st_off), _ptr(status), _stream_ptr(stream)))

    def destroy(self):
        if getattr(self, "_h", None):
            native.load().sdp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------

class _CudaArray:
    """__cuda_array_interface__ over a raw device pointer (for torch.as_tensor)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def _device_view(ptr, shape, typestr):
    torch = _torch()
    if not ptr:
        raise ValueError("result holds no device table")
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")

class Server:
    """Continuous-batching request server (serve_create / serve_submit /
    serve_poll / serve_release / serve_destroy)."""

    def __init__(self, hbm_cap_bytes=150 << 30, max_inflight=4096, num_streams=4, max_batch=64, device=0):
        lib = native.load()
        cfg = native.ServeConfig(hbm_cap_bytes, max_inflight, num_streams, max_batch, device)
        h = ctypes.c_void_p()
        check(lib.serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def now(self) -> float:
        return float(native.load().serve_now(self._h))

    def submit_mcm(self, dims, cost="i64"):
        d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
        req = native.Request(native.DP_REQ_MCM, _cost(cost), int(d.size) - 1, ctypes.c_void_p(d.ctypes.data),
                             None, 0, 0, None)
        return self._submit(req)

    def submit_sdp(self, n, offsets, preset, op="min"):
        a = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        pr = np.ascontiguousarray(np.asarray(preset, dtype=np.uint32))
        req = native.Request(native.DP_REQ_SDP, 0, int(n), None, ctypes.c_void_p(a.ctypes.data), int(a.size),
                             _op(op), ctypes.c_void_p(pr.ctypes.data))
        return self._submit(req)

    def _submit(self, req):
        t = ctypes.c_uint64()
        code = native.load().serve_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if code == native.DP_EBUSY:
            return None
        check(code)
        return int(t.value)

    def poll(self, ticket):
        res = native.Result()
        code = native.load().serve_poll(self._h, ticket, ctypes.byref(res))
        if code == native.DP_EPENDING:
            return None
        check(code)
        return res

    def release(self, ticket, stream=None):
        """Returns a finished request's tables to the server.  Reads of the
        views from tables() that are still enqueued on ``stream`` (default:
        torch's current stream) finish before the memory can be reused;
        reads on another stream must be synchronised first."""
        check(native.load().serve_release_stream(self._h, ticket, _stream_ptr(stream)))

    @staticmethod
    def tables(res, cost="i64"):
        """Zero-copy torch views of a finished request's server-owned device
        tables, valid until release: (m, s) for MCM (``cost`` as submitted),
        ST (int32 holding uint32) for S-DP."""
        n = int(res.n)
        if res.kind == native.DP_REQ_MCM:
            dt = "<i8" if _cost(cost) == native.DP_COST_I64 else "<i4"
            return _device_view(res.m_dev, (n, n), dt), _device_view(res.s_dev, (n, n), "<i2")
        return _device_view(res.st_dev, (n,), "<i4")

    def close(self):
        if getattr(self, "_h", None):
            check(native.load().serve_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
