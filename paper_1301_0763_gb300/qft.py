"""Python binding of the GB300 improved-QFT library (C ABI in include/qft_gb300.h).

Argument marshalling only: every step of every transform runs in the CUDA
kernels of ``_qft_gb300.so``.  PyTorch provides device memory and streams.
If the library is missing this module raises -- there is no CPU fallback.

Transforms (the improved QFT of Pasquini, arXiv 1301.0763, Sec. 5):
  fft(x)        X(k) = sum_n x(n) e^{-2 pi i n k/N}       (eq qft_0A), complex
  ifft(X)       x = swap(DFT(swap X))/N                    (1/N scaled inverse)
  rfft(x)       real [.., N] -> complex [.., N/2+1]        (rdft of Sec. 4.2)
  irfft(Y, n)   complex [.., N/2+1] -> real [.., N]        (1/N scaled)
All four are differentiable (torch.autograd.Function); their backward passes
call the library's adjoint kernels and store nothing but the plan.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_qft_gb300.so")

KIND_C2C, KIND_R2C, KIND_DCT0, KIND_DST0 = 0, 1, 2, 3
DTYPE_F32, DTYPE_F16, DTYPE_BF16, DTYPE_I16 = 0, 1, 2, 3
OP_FORWARD, OP_INVERSE, OP_FORWARD_ADJOINT, OP_INVERSE_ADJOINT = 0, 1, 2, 3
PLAN_AUTOTUNE = 1
PLAN_FP32_PLAIN = 2
PLAN_IN_PLACE = 4
SCHEDULE_KEYS = ("threads", "L1", "LS", "LL", "LB", "LF", "staging", "node_log2", "node_threads", "chunk_rows")

_lib = None
_lock = threading.Lock()


class QFTError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


def load_library(path: str | None = None):
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or os.environ.get("QFT_GB300_LIB", LIB_PATH)
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -m paper_1301_0763_gb300.build` "
                "(nvcc, sm_103a). There is no CPU fallback.")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        lib.qft_plan_create.argtypes = [ctypes.POINTER(vp), i64, i64, ci, ci, ctypes.c_uint]
        lib.qft_plan_create_ragged.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                                               i64, ci, ci, ctypes.c_uint]
        lib.qft_execute.argtypes = [vp, ci, vp, vp, vp]
        lib.qft_execute_fixed.argtypes = [vp, vp, vp, vp, vp]
        for f in (lib.qft_execute_forward, lib.qft_execute_inverse, lib.qft_execute_backward):
            f.argtypes = [vp, vp, vp, vp]
        lib.qft_plan_destroy.argtypes = [vp]
        lib.qft_plan_sync_status.argtypes = [vp]
        lib.qft_plan_last_cuda_error.argtypes = [vp]
        lib.qft_plan_info.argtypes = [vp] + [ctypes.POINTER(ci)] * 4
        lib.qft_filter_create.argtypes = [ctypes.POINTER(vp), i64, i64, i64, ctypes.c_uint]
        lib.qft_filter_forward.argtypes = [vp, vp, vp, vp, vp]
        lib.qft_filter_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.qft_execute_static_scratch.argtypes = [i64, i64, ci, vp, vp, vp]
        lib.qft_static_scratch_sync_status.argtypes = [vp]
        lib.qft_plan_set_wait_limit.argtypes = [vp, i64]
        lib.qft_plan_comp_classes.argtypes = [vp]
        lib.qft_plan_scratch_bytes.argtypes = [vp, ctypes.POINTER(i64)]
        lib.qft_plan_withhold_next_copy.argtypes = [vp]
        lib.qft_plan_schedule.argtypes = [vp, ctypes.POINTER(ci)]
        lib.qft_plan_set_schedule.argtypes = [vp, ctypes.POINTER(ci)]
        lib.qft_plan_time_launches.argtypes = [vp, ci]
        lib.qft_plan_launch_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ci)]
        lib.qft_status_string.argtypes = [ci]
        lib.qft_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load_library().qft_status_string(int(status)).decode()


def _check(rc: int, what: str):
    if rc != 0:
        raise QFTError(rc, what)


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Plan:
    """A plan of `batch` transforms of length `n` (see qft_plan_create)."""

    def __init__(self, n: int, batch: int, kind: int = KIND_C2C, dtype: int = DTYPE_F32, device=None,
                 autotune: bool = False, plain: bool = False, in_place: bool = False):
        self.lib = load_library()
        self.n, self.batch, self.kind, self.dtype = int(n), int(batch), int(kind), int(dtype)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.handle = ctypes.c_void_p()
        flags = ((PLAN_AUTOTUNE if autotune else 0) | (PLAN_FP32_PLAIN if plain else 0) |
                 (PLAN_IN_PLACE if in_place else 0))
        with torch.cuda.device(self.device):
            _check(self.lib.qft_plan_create(ctypes.byref(self.handle), self.n, self.batch, self.kind,
                                            self.dtype, flags), "qft_plan_create")

    def scratch_bytes(self) -> int:
        """Device scratch the plan holds (qft_plan_scratch_bytes)."""
        b = ctypes.c_int64()
        _check(self.lib.qft_plan_scratch_bytes(self.handle, ctypes.byref(b)), "qft_plan_scratch_bytes")
        return int(b.value)

    def comp_classes(self) -> int:
        """Classes per side evaluated on compensated FP32 pairs (qft_plan_comp_classes)."""
        rc = int(self.lib.qft_plan_comp_classes(self.handle))
        if rc < 0:
            raise QFTError(rc, "qft_plan_comp_classes")
        return rc

    def time_launches(self, enable: bool = True):
        _check(self.lib.qft_plan_time_launches(self.handle, 1 if enable else 0), "qft_plan_time_launches")

    def launch_times(self) -> dict:
        """{kernel kind: (summed ms, launches)} of the executes since timing was enabled."""
        ms = (ctypes.c_float * 4)()
        n = (ctypes.c_int * 4)()
        _check(self.lib.qft_plan_launch_times(self.handle, ms, n), "qft_plan_launch_times")
        names = ("k_rows", "k_large_global", "k_large_node", "k_large_slice")
        return {names[k]: (float(ms[k]), int(n[k])) for k in range(4) if n[k]}

    def schedule(self) -> dict:
        """The plan's schedule (see qft_plan_schedule)."""
        v = (ctypes.c_int * 10)()
        _check(self.lib.qft_plan_schedule(self.handle, v), "qft_plan_schedule")
        return dict(zip(SCHEDULE_KEYS, list(v)))

    def set_schedule(self, **kw):
        """Change some schedule values (keys of schedule()); the result is unchanged."""
        cur = self.schedule()
        cur.update(kw)
        v = (ctypes.c_int * 10)(*[int(cur[k]) for k in SCHEDULE_KEYS])
        _check(self.lib.qft_plan_set_schedule(self.handle, v), "qft_plan_set_schedule")

    def execute(self, op: int, inp: torch.Tensor, out: torch.Tensor, stream=None):
        with torch.cuda.device(self.device):
            _check(self.lib.qft_execute(self.handle, int(op), ctypes.c_void_p(inp.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_handle(stream))),
                   "qft_execute")
        return out

    def execute_fixed(self, inp: torch.Tensor, out: torch.Tensor, exps: torch.Tensor, stream=None):
        """Fixed-point forward (QFT_DTYPE_I16 plans, qft_execute_fixed)."""
        with torch.cuda.device(self.device):
            _check(self.lib.qft_execute_fixed(self.handle, ctypes.c_void_p(inp.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(exps.data_ptr()),
                                              ctypes.c_void_p(_stream_handle(stream))), "qft_execute_fixed")
        return out, exps

    def info(self):
        t, c, s, l = (ctypes.c_int() for _ in range(4))
        _check(self.lib.qft_plan_info(self.handle, ctypes.byref(t), ctypes.byref(c), ctypes.byref(s),
                                      ctypes.byref(l)), "qft_plan_info")
        return {"threads": t.value, "ctas": c.value, "smem": s.value, "launches": l.value}

    def sync_status(self) -> int:
        return int(self.lib.qft_plan_sync_status(self.handle))

    def set_wait_limit(self, ns: int):
        """Limit of the kernels' bounded waits for staged copies (0: the default 2 s)."""
        _check(self.lib.qft_plan_set_wait_limit(self.handle, int(ns)), "qft_plan_set_wait_limit")

    def withhold_next_copy(self):
        """Test of the timeout path: the next execute withholds each CTA's first
        staged copy, so its bounded wait runs out (see qft_plan_withhold_next_copy)."""
        _check(self.lib.qft_plan_withhold_next_copy(self.handle), "qft_plan_withhold_next_copy")

    def destroy(self):
        if self.handle and self.handle.value:
            self.lib.qft_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class RaggedPlan(Plan):
    """Many C2C transforms of uneven power-of-two lengths in one packed buffer
    (see qft_plan_create_ragged): row i occupies complex elements
    [offsets[i], offsets[i+1]) and has length 2^log2n[i].  One execute is one
    CUDA-graph launch of every length class."""

    def __init__(self, offsets, log2n, device=None, autotune: bool = False, plain: bool = False,
                 in_place: bool = False):
        import numpy as np
        self.lib = load_library()
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        lg = np.ascontiguousarray(np.asarray(log2n, dtype=np.int32))
        self.count = int(lg.shape[0])
        self.total = int(off[-1]) if off.size else 0
        self.n, self.batch, self.kind, self.dtype = 0, self.count, KIND_C2C, DTYPE_F32
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.qft_plan_create_ragged(
                ctypes.byref(self.handle), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                lg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.count, KIND_C2C, DTYPE_F32,
                (PLAN_AUTOTUNE if autotune else 0) | (PLAN_FP32_PLAIN if plain else 0) |
                (PLAN_IN_PLACE if in_place else 0)),
                "qft_plan_create_ragged")


class FilterPlan(Plan):
    """Plan of the spectral-filter layer y = irfft(W (.) rfft(x)) for x [B, C, N]."""

    def __init__(self, n: int, batch: int, channels: int, device=None):
        self.lib = load_library()
        self.n, self.batch, self.channels = int(n), int(batch), int(channels)
        self.kind, self.dtype = -1, DTYPE_F32
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.qft_filter_create(ctypes.byref(self.handle), self.n, self.batch, self.channels, 0),
                   "qft_filter_create")

    def forward(self, x: torch.Tensor, W: torch.Tensor, y: torch.Tensor, stream=None):
        with torch.cuda.device(self.device):
            _check(self.lib.qft_filter_forward(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(_stream_handle(stream))),
                   "qft_filter_forward")
        return y

    def backward(self, x, W, gy, gx, gW, stream=None):
        with torch.cuda.device(self.device):
            _check(self.lib.qft_filter_backward(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                                ctypes.c_void_p(gy.data_ptr()), ctypes.c_void_p(gx.data_ptr()),
                                                ctypes.c_void_p(gW.data_ptr()), ctypes.c_void_p(_stream_handle(stream))),
                   "qft_filter_backward")


_filter_plans: dict = {}


def _filter_plan(x: torch.Tensor) -> FilterPlan:
    B, C, N = x.shape
    key = (N, B, C, x.device.index)
    p = _filter_plans.get(key)
    if p is None:
        p = FilterPlan(N, B, C, x.device)
        _filter_plans[key] = p
    return p


class _SpectralFilter(torch.autograd.Function):
    """y = irfft(W (.) rfft(x)); backward recomputes rfft(x) (nothing saved but x, W)."""

    @staticmethod
    def forward(ctx, x, W):
        _need_cuda(x)
        x = x.contiguous()
        W = W.contiguous()
        assert x.dtype == torch.float32 and W.dtype == torch.complex64 and x.dim() == 3
        assert W.shape == (x.shape[1], x.shape[2] // 2 + 1)
        y = torch.empty_like(x)
        _filter_plan(x).forward(x, W, y)
        ctx.save_for_backward(x, W)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, W = ctx.saved_tensors
        gy = gy.contiguous()
        gx = torch.empty_like(x)
        gW = torch.empty_like(W)
        _filter_plan(x).backward(x, W, gy, gx, gW)
        return gx, gW


def spectral_filter(x: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    """Spectral-filter layer y = irfft(W (.) rfft(x)) over the last dim of x [B, C, N]."""
    return _SpectralFilter.apply(x, W)


_plans: dict = {}


_autotune = False


def set_autotune(enable: bool):
    """Make the plans that fft / ifft / rfft / irfft create from now on autotuned
    (QFT_PLAN_AUTOTUNE); plans already cached keep their schedule."""
    global _autotune
    _autotune = bool(enable)


def get_plan(n: int, batch: int, kind: int, dtype: int, device: torch.device) -> Plan:
    key = (n, batch, kind, dtype, device.index, _autotune)
    p = _plans.get(key)
    if p is None:
        p = Plan(n, batch, kind, dtype, device, autotune=_autotune and dtype != DTYPE_I16)
        _plans[key] = p
    return p


def _rows(x: torch.Tensor, last: int):
    return x.numel() // last if last else 0


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype in (torch.complex64, torch.float32):
        return DTYPE_F32
    if t.dtype == torch.complex32:
        return DTYPE_F16
    raise TypeError(f"unsupported dtype {t.dtype}")


def _need_cuda(x: torch.Tensor):
    if not x.is_cuda:
        raise ValueError("the improved-QFT library runs on CUDA tensors only (no CPU fallback)")


def _c2c(x: torch.Tensor, op: int) -> torch.Tensor:
    _need_cuda(x)
    x = x.contiguous()
    n = x.shape[-1]
    out = torch.empty_like(x)
    get_plan(n, _rows(x, n), KIND_C2C, _dtype_code(x), x.device).execute(op, x, out)
    return out


def fft_bf16(x: torch.Tensor, op: int = OP_FORWARD) -> torch.Tensor:
    """C2C on bf16 storage: x is a real tensor [..., N, 2] of dtype bfloat16 (re, im)."""
    _need_cuda(x)
    assert x.dtype == torch.bfloat16 and x.shape[-1] == 2
    x = x.contiguous()
    n = x.shape[-2]
    out = torch.empty_like(x)
    get_plan(n, x.numel() // (2 * n), KIND_C2C, DTYPE_BF16, x.device).execute(op, x, out)
    return out


def fft_fixed(z: torch.Tensor):
    """Fixed-point forward DFT (the improved QFT in int32 block floating
    point, qft_execute_fixed): z is an int16 tensor [..., N, 2] of Q15 (re, im)
    samples (value q 2^-15), 2 <= N <= 2^14.  Returns (mantissas int32
    [..., N, 2], exponents int32 [...]); X(k) = mantissa(k) * 2^exponent."""
    _need_cuda(z)
    if z.dtype != torch.int16 or z.dim() < 2 or z.shape[-1] != 2:
        raise TypeError("fft_fixed expects an int16 tensor [..., N, 2]")
    z = z.contiguous()
    n = z.shape[-2]
    out = torch.empty(z.shape, dtype=torch.int32, device=z.device)
    exps = torch.empty(z.shape[:-2], dtype=torch.int32, device=z.device)
    get_plan(n, z.numel() // (2 * n), KIND_C2C, DTYPE_I16, z.device).execute_fixed(z, out, exps)
    return out, exps


def _real_fwd(x: torch.Tensor, op: int) -> torch.Tensor:
    _need_cuda(x)
    x = x.contiguous()
    assert x.dtype == torch.float32
    n = x.shape[-1]
    out = torch.empty(x.shape[:-1] + (n // 2 + 1,), dtype=torch.complex64, device=x.device)
    get_plan(n, _rows(x, n), KIND_R2C, DTYPE_F32, x.device).execute(op, x, out)
    return out


def _real_inv(Y: torch.Tensor, n: int, op: int) -> torch.Tensor:
    _need_cuda(Y)
    Y = Y.contiguous()
    assert Y.dtype == torch.complex64 and Y.shape[-1] == n // 2 + 1
    out = torch.empty(Y.shape[:-1] + (n,), dtype=torch.float32, device=Y.device)
    get_plan(n, _rows(Y, n // 2 + 1), KIND_R2C, DTYPE_F32, Y.device).execute(op, Y, out)
    return out


class _FFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x):
        return _c2c(x, OP_FORWARD)

    @staticmethod
    def backward(ctx, g):
        return _c2c(g, OP_FORWARD_ADJOINT)


class _IFFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X):
        return _c2c(X, OP_INVERSE)

    @staticmethod
    def backward(ctx, g):
        return _c2c(g, OP_INVERSE_ADJOINT)


class _RFFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x):
        ctx.n = x.shape[-1]
        return _real_fwd(x, OP_FORWARD)

    @staticmethod
    def backward(ctx, g):
        return _real_inv(g, ctx.n, OP_FORWARD_ADJOINT)


class _IRFFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, n):
        return _real_inv(Y, n, OP_INVERSE)

    @staticmethod
    def backward(ctx, g):
        return _real_fwd(g, OP_INVERSE_ADJOINT), None


def dct0(c: torch.Tensor) -> torch.Tensor:
    """DCT-0 of periodization N = 2 (c.shape[-1] - 1) of each row (eq qft_0B):
    C(k) = sum_{n=0}^{N/2} c(n) cos(2 pi n k / N), k in [0, N/2]."""
    _need_cuda(c)
    c = c.contiguous()
    assert c.dtype == torch.float32
    N = 2 * (c.shape[-1] - 1)
    rows = _rows(c, c.shape[-1])
    out = torch.empty_like(c)
    get_plan(N, rows, KIND_DCT0, DTYPE_F32, c.device).execute(OP_FORWARD, c, out)
    return out


def dst0(d: torch.Tensor) -> torch.Tensor:
    """DST-0 of periodization N = 2 (d.shape[-1] + 1) of each row (eq qft_0C):
    d holds d(1..N/2-1); S(k) = sum_{n=1}^{N/2-1} d(n) sin(2 pi n k / N), k in [1, N/2-1]."""
    _need_cuda(d)
    d = d.contiguous()
    assert d.dtype == torch.float32
    N = 2 * (d.shape[-1] + 1)
    rows = _rows(d, d.shape[-1])
    out = torch.empty_like(d)
    get_plan(N, rows, KIND_DST0, DTYPE_F32, d.device).execute(OP_FORWARD, d, out)
    return out


_host_streams: dict = {}


def _host_state(dev: torch.device, cells: int) -> dict:
    """The streams, device buffer pairs and events fft_host keeps per device
    (reused by every call; grown, after the streams drain, when a call needs
    larger chunks)."""
    st = _host_streams.get(dev.index)
    if st is None:
        st = {"streams": tuple(torch.cuda.Stream(device=dev) for _ in range(3)), "cells": 0, "next": 0}
        _host_streams[dev.index] = st
    if st["cells"] < cells:
        for s_ in st["streams"]:
            s_.synchronize()
        nbuf = 3
        st["din"] = [torch.empty(cells, dtype=torch.complex64, device=dev) for _ in range(nbuf)]
        st["dout"] = [torch.empty(cells, dtype=torch.complex64, device=dev) for _ in range(nbuf)]
        st["ev_read"] = [torch.cuda.Event() for _ in range(nbuf)]
        st["ev_sent"] = [torch.cuda.Event() for _ in range(nbuf)]
        for e in st["ev_read"] + st["ev_sent"]:
            e.record(st["streams"][0])
        st["cells"] = cells
        st["next"] = 0
    return st


def fft_host(x, out=None, chunk_bytes: int = 512 << 20, device=None):
    """Forward DFT of complex64 rows [..., N] held in pinned host memory, written
    to pinned host memory (``out``, allocated if None).  ``x`` may also be a
    list of such tensors (each with its own N; ``out`` then a list or None):
    one pipeline runs through all of them.  The rows move in chunks of about
    ``chunk_bytes`` through three device buffer pairs: the copy of chunk i+1 to
    the device, the transform of chunk i and the copy of chunk i-1 back run on
    three streams and overlap, and a buffer is refilled as soon as the transform
    that read it is done.  The buffers, streams and events persist per device
    across calls.  Returns ``out`` once the current stream has been ordered
    after the last copy (synchronise before reading it on the host)."""
    xs = list(x) if isinstance(x, (list, tuple)) else [x]
    if out is None:
        outs = [None] * len(xs)
    else:
        outs = list(out) if isinstance(out, (list, tuple)) else [out]
    if len(outs) != len(xs):
        raise ValueError("fft_host: one output per input")
    for i, t in enumerate(xs):
        if t.is_cuda or not t.is_pinned():
            raise ValueError("fft_host takes pinned host tensors")
        if t.dtype != torch.complex64:
            raise TypeError("fft_host takes complex64 tensors")
        if not t.is_contiguous():
            raise ValueError("fft_host takes contiguous tensors")
        if outs[i] is None:
            outs[i] = torch.empty(t.shape, dtype=t.dtype).pin_memory()
        elif outs[i].shape != t.shape or outs[i].dtype != t.dtype or outs[i].is_cuda:
            raise ValueError("fft_host: out must be a host tensor of the input's shape and dtype")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    # the chunks of every input, in order: (input rows, output rows, N)
    work = []
    for t, o in zip(xs, outs):
        N = t.shape[-1]
        rows = t.numel() // N if N else 0
        if rows == 0:
            continue
        xv, ov = t.view(rows, N), o.view(rows, N)
        chunk = max(1, min(rows, chunk_bytes // (8 * N)))
        for r0 in range(0, rows, chunk):
            n = min(chunk, rows - r0)
            work.append((xv[r0:r0 + n], ov[r0:r0 + n], N))
    if not work:
        return outs if isinstance(x, (list, tuple)) else outs[0]
    st = _host_state(dev, max(a.numel() for a, _, _ in work))
    s_in, s_cmp, s_out = st["streams"]
    din, dout, ev_read, ev_sent = st["din"], st["dout"], st["ev_read"], st["ev_sent"]
    nbuf = len(din)
    cur = torch.cuda.current_stream(dev)
    s_in.wait_stream(cur)
    for i, (a, o, N) in enumerate(work):
        b = st["next"]
        st["next"] = (b + 1) % nbuf
        n = a.shape[0]
        di = din[b][: n * N].view(n, N)
        do = dout[b][: n * N].view(n, N)
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_read[b])             # the transform that last read din[b] is done
            di.copy_(a, non_blocking=True)
            e_in = torch.cuda.Event()
            e_in.record(s_in)
        s_cmp.wait_event(e_in)
        s_cmp.wait_event(ev_sent[b])                # the copy that last read dout[b] is done
        get_plan(N, n, KIND_C2C, DTYPE_F32, dev).execute(OP_FORWARD, di, do, s_cmp)
        ev_read[b].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_read[b])
            o.copy_(do, non_blocking=True)
            ev_sent[b].record(s_out)
    cur.wait_stream(s_out)
    return outs if isinstance(x, (list, tuple)) else outs[0]


def fft(x: torch.Tensor) -> torch.Tensor:
    """Forward DFT along the last dim (complex64 or complex32 storage)."""
    return _FFT.apply(x)


def ifft(X: torch.Tensor) -> torch.Tensor:
    """Inverse DFT along the last dim, 1/N scaled."""
    return _IFFT.apply(X)


def rfft(x: torch.Tensor) -> torch.Tensor:
    """Real-input DFT along the last dim: [..., N] float32 -> [..., N/2+1] complex64."""
    return _RFFT.apply(x)


def irfft(Y: torch.Tensor, n: int) -> torch.Tensor:
    """Inverse of rfft: [..., N/2+1] complex64 -> [..., n] float32 (1/n scaled)."""
    return _IRFFT.apply(Y, n)
