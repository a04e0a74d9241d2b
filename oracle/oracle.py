"""ctypes front end of the FP64 improved-QFT oracle (``qft_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``.  The GPU library never
imports it.

Every function here marshals numpy arrays into the C oracle, which follows the
eight recursive functions of Sec. 5 of the paper in FP64 (see the C file's
header for the readings of the paper it takes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_qft_oracle.so")
_LIB32_PATH = os.path.join(_HERE, "_qft_oracle_f32.so")
_LIB32C_PATH = os.path.join(_HERE, "_qft_oracle_f32c.so")
_SRC_FX = os.path.join(_HERE, "qft_oracle_fx.c")
_LIBFX_PATH = os.path.join(_HERE, "_qft_oracle_fx.so")
FLAGS32 = ("-DORACLE_REAL=float", "-ffp-contract=off")
FLAGS32C = ("-DORACLE_REAL=float", "-DORACLE_COMPENSATED", "-ffp-contract=off")
_lock = threading.Lock()
_lib = None
_lib32 = None
_lib32c = None
_libfx = None


def build(force: bool = False, out: str | None = None, extra_flags=(), src: str | None = None) -> str:
    """Compile qft_oracle.c (or `src`) into a shared library (gcc, OpenMP if available)."""
    out = out or _LIB_PATH
    src = src or _SRC
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", src, "-o", out, "-lm", *extra_flags]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return out


def _declare(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    L = ctypes.c_long
    lib.oracle_cdft.argtypes = [L, L, dp, dp, ctypes.c_int]
    lib.oracle_icdft.argtypes = [L, L, dp, dp, ctypes.c_int]
    lib.oracle_rdft.argtypes = [L, L, dp, dp, ctypes.c_int]
    lib.oracle_irdft.argtypes = [L, L, dp, dp, ctypes.c_int]
    lib.oracle_rdft_adjoint.argtypes = [L, L, dp, dp, ctypes.c_int]
    lib.oracle_dct0.argtypes = [L, dp, dp]
    lib.oracle_dst0.argtypes = [L, dp, dp]
    lib.oracle_function.argtypes = [ctypes.c_int, L, dp, dp]
    lib.oracle_counts.argtypes = [ctypes.c_int, L, ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_longlong)]
    lib.oracle_constants_used.argtypes = [L, ctypes.POINTER(ctypes.c_ubyte),
                                          ctypes.POINTER(ctypes.c_int)]
    lib.oracle_constants_used.restype = L
    lib.oracle_secant_table.argtypes = [L, dp]
    lib.oracle_brute_dft.argtypes = [L, dp, dp]
    lib.oracle_cdft_cla.argtypes = [L, L, dp, dp, ctypes.c_int]
    lib.oracle_function_cla.argtypes = [ctypes.c_int, L, dp, dp]
    lib.oracle_counts_cla.argtypes = [ctypes.c_int, L, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_longlong)]
    lib.oracle_constants_used_cla.argtypes = [L, ctypes.POINTER(ctypes.c_ubyte), ctypes.POINTER(ctypes.c_int)]
    lib.oracle_constants_used_cla.restype = L
    lib.oracle_fft_ld.argtypes = [L, dp, dp]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_is_float.restype = ctypes.c_int
    lib.oracle_is_compensated.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


def _load32(comp: bool = True):
    """The same oracle source built with every arithmetic value in FP32
    (-DORACLE_REAL=float): the recursion of Sec. 5 evaluated in single
    precision, operation by operation, with constants rounded once to FP32.
    comp=True (the default) adds -DORACLE_COMPENSATED: the class trees of the
    largest periodizations (N >= 2^16 only) run on compensated pairs, as the
    library does by default; comp=False is the plain FP32 evaluation."""
    global _lib32, _lib32c
    with _lock:
        if comp:
            if _lib32c is None:
                _lib32c = _declare(ctypes.CDLL(build(out=_LIB32C_PATH, extra_flags=FLAGS32C)))
            return _lib32c
        if _lib32 is None:
            _lib32 = _declare(ctypes.CDLL(build(out=_LIB32_PATH, extra_flags=FLAGS32)))
        return _lib32


def build_fx(force: bool = False) -> str:
    """Compile the fixed-point oracle (qft_oracle_fx.c) into its own library."""
    return build(force=force, out=_LIBFX_PATH, src=_SRC_FX)


def _load_fx():
    global _libfx
    with _lock:
        if _libfx is None:
            lib = ctypes.CDLL(build_fx())
            i16 = ctypes.POINTER(ctypes.c_int16)
            i32 = ctypes.POINTER(ctypes.c_int32)
            L = ctypes.c_long
            lib.oracle_cdft_fx.argtypes = [L, L, i16, i32, i32, ctypes.c_int]
            lib.oracle_fx_const.argtypes = [L, L, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
            lib.oracle_fx_rs.argtypes = [ctypes.c_int64, ctypes.c_int]
            lib.oracle_fx_rs.restype = ctypes.c_int64
            _libfx = lib
        return _libfx


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    return x


def _check(rc):
    if rc != 0:
        raise ValueError("oracle rejected the arguments")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def cdft(z, threads: int = 0, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """Forward DFT (eq qft_0A) of each row of z [..., N] by the improved QFT.
    fp32=True evaluates the same recursion in single precision."""
    z = _c128(z)
    N = z.shape[-1]
    batch = z.size // N if N else 0
    out = np.empty_like(z)
    lib = _load32(comp) if fp32 else _load()
    _check(lib.oracle_cdft(N, batch, _dp(z.view(np.float64)), _dp(out.view(np.float64)), threads))
    return out


def icdft(X, threads: int = 0, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """Inverse DFT, 1/N scaled: swap(cdft(swap(X)))/N."""
    X = _c128(X)
    N = X.shape[-1]
    out = np.empty_like(X)
    lib = _load32(comp) if fp32 else _load()
    _check(lib.oracle_icdft(N, X.size // N, _dp(X.view(np.float64)), _dp(out.view(np.float64)), threads))
    return out


def rdft(x, threads: int = 0, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """Forward real DFT [..., N] -> [..., N/2+1] (rdft_cla of Sec. 4.2)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    N = x.shape[-1]
    out = np.empty(x.shape[:-1] + (N // 2 + 1,), dtype=np.complex128)
    lib = _load32(comp) if fp32 else _load()
    _check(lib.oracle_rdft(N, x.size // N, _dp(x), _dp(out.view(np.float64)), threads))
    return out


def irdft(Y, N: int, threads: int = 0, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """Inverse real DFT [..., N/2+1] -> [..., N] (1/N scaled) through DCT-0/DST-0."""
    Y = _c128(Y)
    assert Y.shape[-1] == N // 2 + 1
    out = np.empty(Y.shape[:-1] + (N,), dtype=np.float64)
    lib = _load32(comp) if fp32 else _load()
    _check(lib.oracle_irdft(N, Y.size // (N // 2 + 1), _dp(Y.view(np.float64)), _dp(out), threads))
    return out


def rdft_adjoint(G, N: int, threads: int = 0, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """Adjoint of ``rdft`` for the real inner product on (Re, Im) pairs."""
    G = _c128(G)
    out = np.empty(G.shape[:-1] + (N,), dtype=np.float64)
    lib = _load32(comp) if fp32 else _load()
    _check(lib.oracle_rdft_adjoint(N, G.size // (N // 2 + 1), _dp(G.view(np.float64)), _dp(out), threads))
    return out


def cdft_adjoint(g, threads: int = 0, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """Adjoint of the forward CDFT: F^H g = conj(F conj(g))."""
    return np.conj(cdft(np.conj(_c128(g)), threads, fp32=fp32, comp=comp))


def irdft_adjoint(g, threads: int = 0, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """Adjoint of ``irdft`` (1/N scaled C2R): (w_k/N) rdft(g), w = 1 at k=0,N/2, 2 elsewhere;
    the imaginary parts at k = 0 and N/2 do not reach the output, so their gradient is 0.
    With fp32=True the spectrum and the (power-of-two) weights are applied in FP32."""
    g = np.asarray(g, dtype=np.float64)
    N = g.shape[-1]
    Y = rdft(g, threads, fp32=fp32, comp=comp)
    w = np.full(N // 2 + 1, 2.0 / N)
    w[0] = w[-1] = 1.0 / N
    Y = Y * w
    Y[..., 0] = Y[..., 0].real
    Y[..., -1] = Y[..., -1].real
    return Y


def dct0(c, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """DCT-0 of periodization N = 2 (len - 1) of each row of c [..., N/2+1]
    (eq qft_0B, the dct recursion of Sec. 5); fp32=True evaluates it in FP32."""
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
    N = 2 * (c.shape[-1] - 1)
    out = np.empty_like(c)
    lib = _load32(comp) if fp32 else _load()
    rows_in, rows_out = c.reshape(-1, N // 2 + 1), out.reshape(-1, N // 2 + 1)
    for i in range(rows_in.shape[0]):
        _check(lib.oracle_dct0(N, _dp(rows_in[i]), _dp(rows_out[i])))
    return out


def dst0(d, N: int, fp32: bool = False, comp: bool = True) -> np.ndarray:
    """DST-0 of periodization N (eq qft_0C, the dst recursion of Sec. 5) of each
    row of d [..., N/2+1] indexed by n (the ends n = 0, N/2 are ignored; the
    output is 0 there); fp32=True evaluates it in FP32."""
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float64))
    assert d.shape[-1] == N // 2 + 1
    out = np.empty_like(d)
    lib = _load32(comp) if fp32 else _load()
    rows_in, rows_out = d.reshape(-1, N // 2 + 1), out.reshape(-1, N // 2 + 1)
    for i in range(rows_in.shape[0]):
        _check(lib.oracle_dst0(N, _dp(rows_in[i]), _dp(rows_out[i])))
    return out


FUNCTIONS = {"dct": 0, "dct_ot": 1, "dct_oo": 2, "dst": 3, "dst_ot": 4, "dst_oo": 5}


def function(name: str, N: int, s) -> np.ndarray:
    """Run one recursive function of Sec. 5 on a signal indexed by n (len N/2+1)."""
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    assert s.shape == (N // 2 + 1,)
    out = np.zeros_like(s)
    _check(_load().oracle_function(FUNCTIONS[name], N, _dp(s), _dp(out)))
    return out


KINDS = {"cdft": 0, "rdft": 1, "dct0": 2, "dst0": 3}


def counts(kind: str, N: int):
    """(adds, muls) the oracle performs for one transform of size N."""
    a = ctypes.c_longlong()
    m = ctypes.c_longlong()
    _check(_load().oracle_counts(KINDS[kind], N, ctypes.byref(a), ctypes.byref(m)))
    return int(a.value), int(m.value)


def constants_used(N: int):
    """(used[m] for m in [0, N/4], cos(pi/4) used?) for one CDFT of size N."""
    used = np.zeros(N // 4 + 1, dtype=np.uint8)
    c = ctypes.c_int()
    cnt = _load().oracle_constants_used(N, used.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), ctypes.byref(c))
    if cnt < 0:
        raise ValueError("bad N")
    return used, bool(c.value)


def secant_table(N: int) -> np.ndarray:
    out = np.zeros(N // 4 + 1)
    _check(_load().oracle_secant_table(N, _dp(out)))
    return out


def brute_dft(z) -> np.ndarray:
    """O(N^2) DFT of one row straight from eq qft_0A, long-double accumulation."""
    z = _c128(z)
    assert z.ndim == 1
    out = np.empty_like(z)
    _check(_load().oracle_brute_dft(z.shape[0], _dp(z.view(np.float64)), _dp(out.view(np.float64))))
    return out


# --------------------------------------------------------- classical QFT (Sec. 4)
def cdft_cla(z, threads: int = 0, fp32: bool = False) -> np.ndarray:
    """Forward DFT of each row by the classical QFT of Sec. 4 (cdft_cla ->
    rdft_cla -> dct_cla / dct_to_cla / dst_cla / dst_to_cla), the paper's
    comparison algorithm; fp32=True evaluates it in single precision."""
    z = _c128(z)
    N = z.shape[-1]
    out = np.empty_like(z)
    lib = _load32(False) if fp32 else _load()
    _check(lib.oracle_cdft_cla(N, z.size // N if N else 0, _dp(z.view(np.float64)), _dp(out.view(np.float64)),
                               threads))
    return out


FUNCTIONS_CLA = {"dct_cla": 0, "dct_to_cla": 1, "dst_cla": 2, "dst_to_cla": 3}


def function_cla(name: str, N: int, s) -> np.ndarray:
    """Run one classical function of Sec. 4 on a signal indexed by n (len N/2+1)."""
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    assert s.shape == (N // 2 + 1,)
    out = np.zeros_like(s)
    _check(_load().oracle_function_cla(FUNCTIONS_CLA[name], N, _dp(s), _dp(out)))
    return out


def counts_cla(kind: str, N: int):
    """(adds, muls) the classical QFT performs for one CDFT ('cdft') or RDFT ('rdft')."""
    a = ctypes.c_longlong()
    m = ctypes.c_longlong()
    _check(_load().oracle_counts_cla({"cdft": 0, "rdft": 1}[kind], N, ctypes.byref(a), ctypes.byref(m)))
    return int(a.value), int(m.value)


def constants_used_cla(N: int):
    """(used[m] for m in [0, N/4], cos(pi/4) used?) for one classical CDFT of size N."""
    used = np.zeros(N // 4 + 1, dtype=np.uint8)
    c = ctypes.c_int()
    cnt = _load().oracle_constants_used_cla(N, used.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                            ctypes.byref(c))
    if cnt < 0:
        raise ValueError("bad N")
    return used, bool(c.value)


def fft_ld(z) -> np.ndarray:
    """Reference DFT of one row computed in long double (radix-2, exact-angle
    twiddles), for error measurements; not either QFT algorithm."""
    z = _c128(z)
    assert z.ndim == 1
    out = np.empty_like(z)
    _check(_load().oracle_fft_ld(z.shape[0], _dp(z.view(np.float64)), _dp(out.view(np.float64))))
    return out


# ------------------------------------------------------- fixed-point variant
def cdft_fx(z, threads: int = 0):
    """Fixed-point forward DFT of each row (block floating point, see
    qft_oracle_fx.c): z int16 [..., N, 2] (Q15 re, im) -> (mantissas int32
    [..., N, 2], exponents int32 [...]); the value of X(k) is m(k) 2^E."""
    z = np.ascontiguousarray(np.asarray(z, dtype=np.int16))
    assert z.ndim >= 2 and z.shape[-1] == 2
    N = z.shape[-2]
    batch = z.size // (2 * N) if N else 0
    X = np.empty(z.shape, dtype=np.int32)
    E = np.empty(z.shape[:-2], dtype=np.int32)
    _check(_load_fx().oracle_cdft_fx(N, batch, z.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)),
                                     X.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     E.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), threads))
    return X, E


def fx_value(X, E) -> np.ndarray:
    """complex128 values m 2^E of fixed-point outputs (exact for |m| < 2^53)."""
    X = np.asarray(X)
    E = np.asarray(E)
    return np.ldexp(X[..., 0].astype(np.float64), E[..., None]) + 1j * np.ldexp(
        X[..., 1].astype(np.float64), E[..., None])


def fx_const(N: int, n: int):
    """(c, x): the fixed-point secant 1/(2 cos(2 pi n/N)) = c 2^x, c in [2^30, 2^31)."""
    c = ctypes.c_int64()
    x = ctypes.c_int()
    _check(_load_fx().oracle_fx_const(N, n, ctypes.byref(c), ctypes.byref(x)))
    return int(c.value), int(x.value)


def fx_rs(v: int, s: int) -> int:
    """The oracle's rounding shift v 2^-s (half up; s <= 0 exact)."""
    return int(_load_fx().oracle_fx_rs(v, s))


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))


# ------------------------------------------------------------ spectral filter
def filter_forward(x, W, fp32: bool = False) -> np.ndarray:
    """y = irfft(W (.) rfft(x)) for x [B, C, N] (real) and W [C, N/2+1] (complex),
    by the oracle's rdft / real inverse.  With fp32=True the transforms run in
    FP32 and the product is re = wr*xr - wi*xi, im = wr*xi + wi*xr with every
    operation rounded to FP32 separately."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[-1]
    X = rdft(x.reshape(-1, N), fp32=fp32).reshape(x.shape[:-1] + (N // 2 + 1,))
    if fp32:
        f = np.float32
        Xr, Xi = X.real.astype(f), X.imag.astype(f)
        Wr, Wi = np.asarray(W).real.astype(f), np.asarray(W).imag.astype(f)
        Yr = (Wr * Xr).astype(f) - (Wi * Xi).astype(f)
        Yi = (Wr * Xi).astype(f) + (Wi * Xr).astype(f)
        Y = Yr.astype(np.float64) + 1j * Yi.astype(np.float64)
    else:
        Y = np.asarray(W, dtype=np.complex128) * X
    return irdft(Y.reshape(-1, N // 2 + 1), N, fp32=fp32).reshape(x.shape)


def filter_backward(x, W, gy):
    """(gx, gW) of the filter layer for the upstream gradient gy (FP64):
    gx = rfft^H(conj(W) (.) irfft^H(gy)), gW = sum_b irfft^H(gy_b) (.) conj(rfft(x_b))."""
    x = np.asarray(x, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    B, C, N = x.shape
    H = N // 2 + 1
    G = irdft_adjoint(gy.reshape(-1, N)).reshape(B, C, H)
    X = rdft(x.reshape(-1, N)).reshape(B, C, H)
    gW = (G * np.conj(X)).sum(axis=0)
    gX = np.conj(np.asarray(W, dtype=np.complex128))[None] * G
    gx = rdft_adjoint(gX.reshape(-1, H), N).reshape(B, C, N)
    return gx, gW
