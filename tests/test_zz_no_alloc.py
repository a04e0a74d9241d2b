"""qft_execute_static_scratch: the large-row C2C FP32 transform on the
library's static device scratch, with no plan and no allocation.

Who needs it: code that cannot call cudaMalloc where it wants a transform --
another allocator already holds the device's free memory, or a tight loop
cannot afford the device-wide synchronisation of cudaMalloc / cudaFree.

Checked on two calls in a row against the plan-based entry point
(qft_execute), bit for bit: both run the same FP32 operations of the
recursion of Sec. 5 on the same operands.  Rows outnumber what the static
scratch holds at once, so they run in several chunks.  One call is also
compared bit for bit with the oracle evaluated in FP32, at 2^15 and 2^20.
The device's free memory is unchanged across the second call, the static
status word reads QFT_OK afterwards, and an in-place call (in == out) gives
the same bits.  The file name makes pytest collect it last; it also passes
when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1301_0763_gb300 import inputs

QFT_OP_FORWARD = 0
QFT_OP_INVERSE = 1
QFT_OP_FORWARD_ADJOINT = 2
QFT_OP_INVERSE_ADJOINT = 3
QFT_ERR_INVALID_N = -1
QFT_ERR_INVALID_BATCH = -2
QFT_ERR_INVALID_ARG = -9


def _lib():
    from paper_1301_0763_gb300 import build
    build.build()
    from paper_1301_0763_gb300 import qft
    return qft, qft.load_library()


def _bits_equal(a, b):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def _oracle32(op, z):
    N = z.shape[-1]
    ref = {QFT_OP_FORWARD: lambda: orc.cdft(z, fp32=True),
           QFT_OP_INVERSE: lambda: orc.icdft(z, fp32=True),
           QFT_OP_FORWARD_ADJOINT: lambda: orc.cdft_adjoint(z, fp32=True),
           QFT_OP_INVERSE_ADJOINT: lambda: orc.cdft(z, fp32=True) / N}[op]()
    return ref.astype(np.complex64)


def test_static_scratch_rejects_sizes_beyond_its_limit():
    """Host-side checks, before any device work: n outside [2^15, 2^20] or not a
    power of two, negative batch, unknown op."""
    _, lib = _lib()
    p = ctypes.c_void_p(8)
    for n in (1 << 21, 1 << 24, 1 << 14, 3 << 15):
        assert lib.qft_execute_static_scratch(n, 1, QFT_OP_FORWARD, p, p, None) == QFT_ERR_INVALID_N
    assert lib.qft_execute_static_scratch(1 << 16, -1, QFT_OP_FORWARD, p, p, None) == QFT_ERR_INVALID_BATCH
    assert lib.qft_execute_static_scratch(1 << 16, 1, 7, p, p, None) == QFT_ERR_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("r,batch,op,oracle_rows", [
    (15, 130, QFT_OP_FORWARD, (0, 129)),
    (20, 4, QFT_OP_FORWARD, (3,)),
    (17, 9, QFT_OP_INVERSE, ()),
    (16, 5, QFT_OP_FORWARD_ADJOINT, ()),
    (18, 4, QFT_OP_INVERSE_ADJOINT, ()),
])
def test_static_scratch_matches_plan_two_calls(r, batch, op, oracle_rows):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qft, lib = _lib()
    N = 1 << r
    z1 = inputs.uniform_complex(batch, N, seed=31)
    z2 = inputs.normal_complex(batch, N, seed=32)
    x1 = torch.from_numpy(z1).cuda()
    x2 = torch.from_numpy(z2).cuda()
    y1 = torch.empty_like(x1)
    y2 = torch.empty_like(x2)
    stream = torch.cuda.current_stream()
    st = ctypes.c_void_p(stream.cuda_stream)
    torch.cuda.synchronize()
    rc = lib.qft_execute_static_scratch(N, batch, op, ctypes.c_void_p(x1.data_ptr()),
                                        ctypes.c_void_p(y1.data_ptr()), st)
    assert rc == 0, qft.QFTError(rc, "qft_execute_static_scratch")
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    rc = lib.qft_execute_static_scratch(N, batch, op, ctypes.c_void_p(x2.data_ptr()),
                                        ctypes.c_void_p(y2.data_ptr()), st)
    assert rc == 0, qft.QFTError(rc, "qft_execute_static_scratch")
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    # any scratch allocation would take at least one row's copies (>= 0.5 MiB)
    assert free_before - free_after < (1 << 19)
    assert lib.qft_static_scratch_sync_status(st) == 0

    plan = qft.Plan(N, batch)
    for x, y in ((x1, y1), (x2, y2)):
        ref = torch.empty_like(x)
        plan.execute(op, x, ref)
        torch.cuda.synchronize()
        assert _bits_equal(y.cpu().numpy(), ref.cpu().numpy())
    plan.destroy()
    if oracle_rows:
        rows = list(oracle_rows)
        assert _bits_equal(y1.cpu().numpy()[rows], _oracle32(op, z1[rows]))


@pytest.mark.gpu
def test_static_scratch_in_place():
    """in == out: the same bits as the out-of-place call."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qft, lib = _lib()
    N, batch = 1 << 16, 7
    x = torch.from_numpy(inputs.normal_complex(batch, N, seed=33)).cuda()
    y = torch.empty_like(x)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.qft_execute_static_scratch(N, batch, QFT_OP_FORWARD, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr()), st) == 0
    assert lib.qft_execute_static_scratch(N, batch, QFT_OP_FORWARD, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(x.data_ptr()), st) == 0
    assert lib.qft_static_scratch_sync_status(st) == 0
    assert torch.equal(x.view(torch.int32), y.view(torch.int32))
