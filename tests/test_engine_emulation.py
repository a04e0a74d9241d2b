"""The kernel's engine source, compiled for the host, against the oracle (no GPU).

The row engine (qft_engine.cuh / qft_io.cuh) is the code the sm_103a kernels
run.  Built for the host with QFT_HOST_EMULATION and driven phase by phase like
one CTA, it must reproduce the improved-QFT recursion evaluated in FP32 by the
oracle bit for bit: every task performs exactly the additions and multiplies
of Sec. 5 on exactly the same operands, so any index mistake shows up as a
mismatch.  It is also checked against the FP64 oracle within the FP32 error
level of the method.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_0763_gb300 import inputs
from tests.emu import emu

LOGS = list(range(2, 15))


def bits_equal(a, b):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def rel_l2_rows(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("lg", LOGS)
def test_c2c_forward_bit_exact(lg):
    N = 1 << lg
    z = inputs.normal_complex(3, N, seed=1)
    X = emu.c2c(z)
    ref32 = orc.cdft(z, fp32=True).astype(np.complex64)
    assert bits_equal(X, ref32)
    ref64 = orc.cdft(z)
    assert rel_l2_rows(X.astype(np.complex128), ref64).max() < 4e-8 * np.sqrt(N) + 1e-7


@pytest.mark.parametrize("lg", [2, 3, 6, 10, 13])
@pytest.mark.parametrize("op", [1, 2, 3])
def test_c2c_other_ops_bit_exact(lg, op):
    N = 1 << lg
    z = inputs.uniform_complex(2, N, seed=3)
    out = emu.c2c(z, op=op)
    if op == 1:
        ref = orc.icdft(z, fp32=True)
    elif op == 2:
        ref = orc.cdft_adjoint(z, fp32=True)
    else:
        ref = orc.cdft(z, fp32=True) / N
    assert bits_equal(out, ref.astype(np.complex64))


@pytest.mark.parametrize("tune", [(3, 4, 3, 4, 3), (4, 2, 2, 2, 2), (2, 3, 4, 3, 1), (4, 4, 1, 1, 0),
                                  (0, 1, 1, 4, 3), (4, 4, 3, 4, 3), (3, 3, 3, 3, 2)])
@pytest.mark.parametrize("lg", [5, 9, 12])
def test_schedules_do_not_change_the_result(tune, lg):
    """Any tile/stage schedule of the planner yields the same bits."""
    N = 1 << lg
    rc, _, _, max_slice = emu.plan_info(N, tune)
    if rc != 0 or max_slice > (512 if lg >= 14 else 256):
        pytest.skip("schedule not valid for this N with 256 threads")
    z = inputs.normal_complex(1, N, seed=5)
    assert bits_equal(emu.c2c(z, tune=tune), emu.c2c(z))


@pytest.mark.parametrize("lg", [2, 3, 5, 8, 12])
@pytest.mark.parametrize("rows", [1, 2, 5])
def test_real_forward_and_inverse_bit_exact(lg, rows):
    N = 1 << lg
    x = inputs.normal_real(rows, N, seed=7)
    X = emu.r2c(x, 0, N)
    assert bits_equal(X, orc.rdft(x, fp32=True).astype(np.complex64))
    Y = X.copy()
    Y[:, 0] += 0.25j          # imaginary parts at 0 and N/2 are ignored by the inverse
    Y[:, -1] -= 0.5j
    xr = emu.r2c(Y, 1, N)
    assert bits_equal(xr, orc.irdft(Y, N, fp32=True).astype(np.float32))
    assert np.abs(xr - x).max() < 1e-5 * np.sqrt(N)


@pytest.mark.parametrize("lg", [2, 4, 9, 12])
def test_real_adjoints_bit_exact(lg):
    N = 1 << lg
    g = inputs.normal_complex(3, N // 2 + 1, seed=8)
    gx = emu.r2c(g, 2, N)
    assert bits_equal(gx, orc.rdft_adjoint(g, N, fp32=True).astype(np.float32))
    u = inputs.normal_real(3, N, seed=9)
    gy = emu.r2c(u, 3, N)
    ref = orc.irdft_adjoint(u, fp32=True).astype(np.complex64)
    assert bits_equal(gy, ref)


def _bf16_round(x32):
    """Round float32 -> bfloat16 (nearest even), returned as uint16 bits."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def _bf16_to_f32(b):
    return (b.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("lg", [4, 10, 13])
@pytest.mark.parametrize("dtype", [1, 2])
def test_half_storage_bit_exact(lg, dtype):
    N = 1 << lg
    z = inputs.uniform_complex(2, N, seed=10).view(np.float32).reshape(2, N, 2)
    if dtype == 1:
        zin = z.astype(np.float16)
        bits = zin.view(np.uint16)
        zf = zin.astype(np.float32)
    else:
        bits = _bf16_round(z)
        zf = _bf16_to_f32(bits)
    out = emu.c2c_half(bits, dtype)
    zc = zf[..., 0].astype(np.float64) + 1j * zf[..., 1]
    ref = orc.cdft(zc, fp32=True).astype(np.complex64)
    ref2 = ref.view(np.float32).reshape(2, N, 2)
    ref_bits = ref2.astype(np.float16).view(np.uint16) if dtype == 1 else _bf16_round(ref2)
    assert np.array_equal(out, ref_bits)


# ------------------------------------------------------------------ large rows
@pytest.mark.parametrize("lg", [15, 16, 17, 18, 20])
def test_large_path_forward_bit_exact(lg):
    """Rows longer than one CTA (global phases + shared-memory node groups +
    ping-pong slices) reproduce the FP32 recursion bit for bit -- with the
    library's compensated classes (from N = 2^16) and in plain FP32."""
    N = 1 << lg
    z = inputs.normal_complex(1, N, seed=20 + lg)
    assert bits_equal(emu.c2c_large(z), orc.cdft(z, fp32=True).astype(np.complex64))
    assert bits_equal(emu.c2c_large(z, plain=True), orc.cdft(z, fp32=True, comp=False).astype(np.complex64))


@pytest.mark.parametrize("lg", [16, 18])
@pytest.mark.parametrize("node_log2", [10, 11])
def test_large_path_node_sizes(lg, node_log2):
    """Node groups of 2^10 and 2^11 cells (the default is 2^12): same bits."""
    N = 1 << lg
    z = inputs.normal_complex(1, N, seed=40 + lg)
    assert bits_equal(emu.c2c_large(z, node_log2=node_log2), orc.cdft(z, fp32=True).astype(np.complex64))


@pytest.mark.parametrize("lg", [7, 8, 10, 12])
@pytest.mark.parametrize("J", [1, 2])
def test_large_path_compensated_classes_small_n(lg, J):
    """The compensated class trees at small N (the class count forced on both
    sides), where every launch of the large-row path is exercised in seconds."""
    import ctypes
    N = 1 << lg
    z = inputs.normal_complex(2, N, seed=60 + lg).astype(np.complex64)
    L = emu.load()
    fp = ctypes.POINTER(ctypes.c_float)
    out = np.empty_like(z)
    assert L.emu_c2c_large(N, 2, z.view(np.float32).ctypes.data_as(fp), out.view(np.float32).ctypes.data_as(fp),
                           0, -J, 12, 0) == 0
    lib = orc._load32(True)
    lib.oracle_set_comp_classes.argtypes = [ctypes.c_int]
    lib.oracle_set_comp_classes(J)
    try:
        ref = orc.cdft(z, fp32=True).astype(np.complex64)
    finally:
        lib.oracle_set_comp_classes(-1)
    assert bits_equal(out, ref)
    assert not bits_equal(ref, orc.cdft(z, fp32=True, comp=False).astype(np.complex64))


@pytest.mark.parametrize("op", [1, 2, 3])
@pytest.mark.parametrize("lg", [15, 16])
def test_large_path_other_ops(op, lg):
    N = 1 << lg
    z = inputs.uniform_complex(2, N, seed=op)
    ref = {1: lambda: orc.icdft(z, fp32=True), 2: lambda: orc.cdft_adjoint(z, fp32=True),
           3: lambda: orc.cdft(z, fp32=True) / N}[op]()
    assert bits_equal(emu.c2c_large(z, op), ref.astype(np.complex64))


def test_large_path_real():
    N = 1 << 16
    x = inputs.normal_real(3, N, seed=4)
    X = emu.r2c_large(x, 0, N)
    assert bits_equal(X, orc.rdft(x, fp32=True).astype(np.complex64))
    assert bits_equal(emu.r2c_large(X, 1, N), orc.irdft(X, N, fp32=True).astype(np.float32))
    assert bits_equal(emu.r2c_large(X, 2, N), orc.rdft_adjoint(X, N, fp32=True).astype(np.float32))
    assert bits_equal(emu.r2c_large(x, 3, N), orc.irdft_adjoint(x, fp32=True).astype(np.complex64))
    assert bits_equal(emu.r2c_large(x, 0, N, plain=True), orc.rdft(x, fp32=True, comp=False).astype(np.complex64))


# ------------------------------------------- large rows, one scratch copy
def _brev(x, n):
    return int(format(x, f"0{n}b")[::-1], 2) if n else 0


@pytest.mark.parametrize("sb", [1, 3, 6])
@pytest.mark.parametrize("L", [1, 2, 3])
def test_in_place_order_composes(sb, L):
    """The in-place order (ip_perm) against its derivation, written out here
    by brute force: a level of L backward levels over 2^L descendants of 2^sb
    cells, each already in the order of dp in-place levels, writes output u of
    chunk i over descendant bitrev_L(u)'s cell i.  The node's output k = i 2^L
    + u must then sit where ip_perm(k, dp + L, sb + L) says, for every dp; and
    ip_perm(., d, s) is a permutation of 2^s cells."""
    lib = emu.load()
    for dp in range(0, sb + 1):
        S = 1 << sb
        pos = {}
        for i in range(S):
            for u in range(1 << L):
                pos[i * (1 << L) + u] = (_brev(u, L) << sb) + lib.emu_ip_perm(i, dp, sb)
        assert sorted(pos.values()) == list(range(S << L))
        for k, p in pos.items():
            assert lib.emu_ip_perm(k, dp + L, sb + L) == p, (dp, k)
    assert lib.emu_ip_perm(5, 0, 4) == 5
    assert lib.emu_ip_perm(1, 4, 4) == 8 and lib.emu_ip_perm(2, 4, 4) == 4


@pytest.mark.parametrize("lg,node_log2", [(15, 12), (15, 5), (16, 8), (17, 6), (18, 12), (18, 9)])
def test_large_path_in_place_bit_exact(lg, node_log2):
    """The one-scratch schedule (Sec. 6.1): the SLICE levels above the node
    depth write over the cells they read, the class outputs stay in the order
    that leaves, the final combine reads them through it, and neighbour cells
    cross block edges through halo copies (blocks emulated odd ones first, so
    at every edge one block has written before the other reads).  Same bits
    as the oracle; smaller nodes give several in-place phases a class."""
    N = 1 << lg
    z = inputs.normal_complex(1, N, seed=80 + lg)
    ref = orc.cdft(z, fp32=True).astype(np.complex64)
    assert bits_equal(emu.c2c_large(z, node_log2=node_log2, inplace=True), ref)
    assert bits_equal(emu.c2c_large(z, plain=True, node_log2=node_log2, inplace=True),
                      orc.cdft(z, fp32=True, comp=False).astype(np.complex64))


@pytest.mark.parametrize("lg", [8, 10, 12])
@pytest.mark.parametrize("J", [1, 2])
def test_large_path_in_place_compensated_small_n(lg, J):
    """Compensated classes on the in-place schedule at small N, nodes of 2^4
    cells (up to eight in-place phases a class)."""
    import ctypes
    N = 1 << lg
    z = inputs.normal_complex(2, N, seed=90 + lg).astype(np.complex64)
    L = emu.load()
    fp = ctypes.POINTER(ctypes.c_float)
    out = np.empty_like(z)
    assert L.emu_c2c_large(N, 2, z.view(np.float32).ctypes.data_as(fp), out.view(np.float32).ctypes.data_as(fp),
                           0, -J, 4, 1) == 0
    lib = orc._load32(True)
    lib.oracle_set_comp_classes.argtypes = [ctypes.c_int]
    lib.oracle_set_comp_classes(J)
    try:
        ref = orc.cdft(z, fp32=True).astype(np.complex64)
    finally:
        lib.oracle_set_comp_classes(-1)
    assert bits_equal(out, ref)


@pytest.mark.parametrize("op", [1, 2, 3])
def test_large_path_in_place_other_ops_and_real(op):
    N = 1 << 16
    z = inputs.uniform_complex(2, N, seed=95 + op)
    ref = {1: lambda: orc.icdft(z, fp32=True), 2: lambda: orc.cdft_adjoint(z, fp32=True),
           3: lambda: orc.cdft(z, fp32=True) / N}[op]()
    assert bits_equal(emu.c2c_large(z, op, node_log2=9, inplace=True), ref.astype(np.complex64))
    x = inputs.normal_real(2, N, seed=98)
    X = orc.rdft(x, fp32=True).astype(np.complex64)
    if op == 1:
        assert bits_equal(emu.r2c_large(x, 0, N, inplace=True), X)
        assert bits_equal(emu.r2c_large(X, 1, N, inplace=True), orc.irdft(X, N, fp32=True).astype(np.float32))


@pytest.mark.parametrize("lg", [2, 3, 4, 6, 9, 12, 14])
@pytest.mark.parametrize("rows", [1, 3])
def test_dct0_dst0_bit_exact(lg, rows):
    """Standalone DCT-0 / DST-0 of periodization N (eqs qft_0B, qft_0C): the
    bits of the dct / dst recursions of the oracle evaluated in FP32."""
    N = 1 << lg
    g = inputs.rng(400 + lg)
    c = g.standard_normal((rows, N // 2 + 1)).astype(np.float32)
    C = emu.r2r(c, N, dst=False)
    assert bits_equal(C, orc.dct0(c, fp32=True).astype(np.float32))
    d = g.standard_normal((rows, N // 2 - 1)).astype(np.float32)
    S = emu.r2r(d, N, dst=True)
    dfull = np.zeros((rows, N // 2 + 1))
    dfull[:, 1:-1] = d
    assert bits_equal(S, orc.dst0(dfull, N, fp32=True)[:, 1:-1].astype(np.float32))
