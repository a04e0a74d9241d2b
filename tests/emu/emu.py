"""Builds and loads the host emulation of the row engine (tests only)."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SRC = os.path.join(HERE, "qft_emu.cpp")
DEPS = [os.path.join(ROOT, "paper_1301_0763_gb300", "csrc", f)
        for f in ("qft_engine.cuh", "qft_io.cuh", "qft_planner.h", "qft_plan.h", "qft_consts.h")]
LIB = os.path.join(HERE, "_qft_emu.so")
_lib = None
SRC_FX = os.path.join(HERE, "qft_fx_emu.cpp")
DEP_FX = os.path.join(ROOT, "paper_1301_0763_gb300", "csrc", "qft_fixed.cuh")
LIB_FX = os.path.join(HERE, "_qft_fx_emu.so")
_lib_fx = None


def load_fx():
    """The host emulation of the fixed-point kernel (qft_fx_emu.cpp)."""
    global _lib_fx
    if _lib_fx is not None:
        return _lib_fx
    newest = max(os.path.getmtime(p) for p in (SRC_FX, DEP_FX))
    if not os.path.exists(LIB_FX) or os.path.getmtime(LIB_FX) < newest:
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", SRC_FX, "-o", LIB_FX], check=True)
    lib = ctypes.CDLL(LIB_FX)
    lib.emu_cdft_fx.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    _lib_fx = lib
    return lib


def cdft_fx(z):
    """z int16 [..., N, 2] -> (int32 mantissas [..., N, 2], int32 exponents [...])."""
    z = np.ascontiguousarray(z, dtype=np.int16)
    N = z.shape[-2]
    X = np.empty(z.shape, dtype=np.int32)
    E = np.empty(z.shape[:-2], dtype=np.int32)
    rc = load_fx().emu_cdft_fx(N, z.size // (2 * N), z.ctypes.data, X.ctypes.data, E.ctypes.data)
    if rc != 0:
        raise ValueError(f"fixed-point emulation failed (rc={rc})")
    return X, E


def load():
    global _lib
    if _lib is not None:
        return _lib
    newest = max(os.path.getmtime(p) for p in [SRC] + DEPS)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", LIB],
                       check=True)
    lib = ctypes.CDLL(LIB)
    fp = ctypes.POINTER(ctypes.c_float)
    ip = ctypes.POINTER(ctypes.c_int)
    up = ctypes.POINTER(ctypes.c_uint16)
    lib.emu_c2c.argtypes = [ctypes.c_int, ctypes.c_int64, fp, fp, ctypes.c_int, ip, ctypes.c_int]
    lib.emu_c2c_half.argtypes = [ctypes.c_int, ctypes.c_int64, up, up, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.emu_r2c.argtypes = [ctypes.c_int, ctypes.c_int64, fp, fp, ctypes.c_int, ctypes.c_int]
    lib.emu_plan_info.argtypes = [ctypes.c_int, ip, ip, ip, ip]
    lib.emu_c2c_large.argtypes = [ctypes.c_int, ctypes.c_int64, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int]
    lib.emu_r2c_large.argtypes = [ctypes.c_int, ctypes.c_int64, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.emu_ip_perm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    _lib = lib
    return lib


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def c2c(z, op=0, tune=None, nthr=0):
    z = np.ascontiguousarray(z, dtype=np.complex64)
    N = z.shape[-1]
    out = np.empty_like(z)
    t = None
    if tune is not None:
        t = (ctypes.c_int * 5)(*tune)
    rc = load().emu_c2c(N, z.size // N, _fp(z.view(np.float32)), _fp(out.view(np.float32)), op,
                        ctypes.cast(t, ctypes.POINTER(ctypes.c_int)) if t is not None else None, nthr)
    if rc != 0:
        raise ValueError(f"emulation rejected N={N} tune={tune} (rc={rc})")
    return out


def c2c_half(z16, dtype, op=0, nthr=0):
    """z16: uint16 array [..., N, 2] holding fp16 (dtype=1) or bf16 (dtype=2) pairs."""
    z16 = np.ascontiguousarray(z16, dtype=np.uint16)
    N = z16.shape[-2]
    out = np.empty_like(z16)
    up = ctypes.POINTER(ctypes.c_uint16)
    rc = load().emu_c2c_half(N, z16.size // (2 * N), z16.ctypes.data_as(up), out.ctypes.data_as(up), dtype, op, nthr)
    if rc != 0:
        raise ValueError("emulation rejected")
    return out


def r2c(x, op, N, nthr=0):
    """op 0: real [B,N] -> complex [B,N/2+1]; 1: complex -> real (1/N); 2: complex -> real (adjoint);
    3: real -> complex (adjoint of the real inverse)."""
    if op in (0, 3):
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty(x.shape[:-1] + (N // 2 + 1,), dtype=np.complex64)
        rows = x.size // N
        rc = load().emu_r2c(N, rows, _fp(x), _fp(out.view(np.float32)), op, nthr)
    else:
        x = np.ascontiguousarray(x, dtype=np.complex64)
        out = np.empty(x.shape[:-1] + (N,), dtype=np.float32)
        rows = x.size // (N // 2 + 1)
        rc = load().emu_r2c(N, rows, _fp(x.view(np.float32)), _fp(out), op, nthr)
    if rc != 0:
        raise ValueError("emulation rejected")
    return out


def plan_info(N, tune=None):
    t = (ctypes.c_int * 5)(*tune) if tune is not None else None
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = load().emu_plan_info(N, ctypes.cast(t, ctypes.POINTER(ctypes.c_int)) if t is not None else None,
                              ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return rc, a.value, b.value, c.value


def c2c_large(z, op=0, plain=False, node_log2=None, inplace=False):
    """The large-row launch sequence on the host; plain=True runs every class
    tree in plain FP32 instead of the library's compensated classes (node
    groups of 2^node_log2 cells, the library's default 2^12); inplace=True runs
    the one-scratch schedule (in-place SLICE levels)."""
    z = np.ascontiguousarray(z, dtype=np.complex64)
    N = z.shape[-1]
    if node_log2 is None:
        node_log2 = 12
    out = np.empty_like(z)
    rc = load().emu_c2c_large(N, z.size // N, _fp(z.view(np.float32)), _fp(out.view(np.float32)), op,
                              1 if plain else 0, node_log2, 1 if inplace else 0)
    if rc != 0:
        raise ValueError("emulation rejected")
    return out


def r2c_large(x, op, N, plain=False, inplace=False):
    if op in (0, 3):
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty(x.shape[:-1] + (N // 2 + 1,), dtype=np.complex64)
        rc = load().emu_r2c_large(N, x.size // N, _fp(x), _fp(out.view(np.float32)), op, 1 if plain else 0,
                                  1 if inplace else 0)
    else:
        x = np.ascontiguousarray(x, dtype=np.complex64)
        out = np.empty(x.shape[:-1] + (N,), dtype=np.float32)
        rc = load().emu_r2c_large(N, x.size // (N // 2 + 1), _fp(x.view(np.float32)), _fp(out), op,
                                  1 if plain else 0, 1 if inplace else 0)
    if rc != 0:
        raise ValueError("emulation rejected")
    return out


def r2r(x, N, dst, nthr=0):
    """DCT-0 (dst=False, rows of N/2+1) or DST-0 (dst=True, rows of N/2-1)."""
    lib = load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    out = np.empty_like(x)
    lib.emu_r2r.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    rows = x.size // x.shape[-1]
    rc = lib.emu_r2r(N, rows, x.ctypes.data, out.ctypes.data, 1 if dst else 0, nthr)
    if rc != 0:
        raise ValueError(f"emulation rejected N={N} (rc={rc})")
    return out
