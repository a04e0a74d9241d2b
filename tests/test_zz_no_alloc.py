"""qft_execute_static_scratch: the large-row C2C FP32 transform on the
library's static device scratch, with no plan and no allocation.

Checked against the plan-based entry point (qft_execute) on two calls in a row,
with more rows than the static scratch holds at once (so the rows run in
several chunks), and with the device's free memory unchanged across the second
call.  The file name makes pytest collect it last; it also passes alone.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1301_0763_gb300 import inputs

QFT_OP_FORWARD = 0
QFT_OP_INVERSE = 1
QFT_ERR_INVALID_N = -1
QFT_ERR_INVALID_BATCH = -2


def tol(N):
    return max(1e-5, 6e-8 * np.sqrt(N))


def _lib():
    from paper_1301_0763_gb300 import build
    build.build()
    from paper_1301_0763_gb300 import qft
    return qft, qft.load_library()


def test_static_scratch_rejects_sizes_beyond_its_limit():
    """Host-side checks, before any device work: n outside [2^15, 2^20] or not a
    power of two, negative batch."""
    _, lib = _lib()
    p = ctypes.c_void_p(8)
    for n in (1 << 21, 1 << 24, 1 << 14, 3 << 15):
        assert lib.qft_execute_static_scratch(n, 1, QFT_OP_FORWARD, p, p, None) == QFT_ERR_INVALID_N
    assert lib.qft_execute_static_scratch(1 << 16, -1, QFT_OP_FORWARD, p, p, None) == QFT_ERR_INVALID_BATCH


@pytest.mark.gpu
@pytest.mark.parametrize("r,batch,op", [(15, 130, QFT_OP_FORWARD), (20, 4, QFT_OP_FORWARD), (17, 9, QFT_OP_INVERSE)])
def test_static_scratch_matches_plan_two_calls(r, batch, op):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qft, lib = _lib()
    N = 1 << r
    x1 = torch.from_numpy(inputs.uniform_complex(batch, N, seed=31)).to(torch.complex64).cuda()
    x2 = torch.from_numpy(inputs.uniform_complex(batch, N, seed=32)).to(torch.complex64).cuda()
    y1 = torch.empty_like(x1)
    y2 = torch.empty_like(x2)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
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

    plan = qft.Plan(N, batch)
    for x, y in ((x1, y1), (x2, y2)):
        ref = torch.empty_like(x)
        plan.execute(op, x, ref)
        torch.cuda.synchronize()
        a = y.cpu().numpy()
        b = ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() <= tol(N) * np.abs(b).max()
    plan.destroy()
