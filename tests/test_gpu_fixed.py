"""GPU parity of the fixed-point variant (qft_execute_fixed, kernel k_fixed)
against the fixed-point oracle: integer work, so every mantissa and every row
exponent must be equal.  Calls go through the C ABI."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1301_0763_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1301_0763_gb300 import build
    build.build()
    from paper_1301_0763_gb300 import qft
    qft.load_library()
    torch.cuda.set_device(0)
    return qft


def _cases(N, seed, rows=4):
    cs = [inputs.q15_complex(rows, N, seed=seed),
          np.zeros((1, N, 2), np.int16),
          np.full((1, N, 2), -32768, np.int16),
          np.full((1, N, 2), 32767, np.int16)]
    for n0 in sorted({0, N // 2, N // 4, 1, N - 1}):
        z = np.zeros((1, N, 2), np.int16)
        z[0, n0, 0] = -32768
        z[0, n0, 1] = 1
        cs.append(z)
    for step in (2, 4, 8):
        z = inputs.q15_complex(2, N, seed=seed + step)
        z[:, np.arange(N) % step != 0, :] = 0
        cs.append(z)
    z = inputs.q15_complex(2, N, seed=seed + 20)
    z[..., 1] = 0
    cs.append(z)
    cs.append((inputs.q15_complex(2, N, seed=seed + 30) >> 12).astype(np.int16))
    return np.concatenate(cs)


def _gpu_fx(q, z):
    X, E = q.fft_fixed(torch.from_numpy(np.ascontiguousarray(z)).cuda())
    torch.cuda.synchronize()
    return X.cpu().numpy(), E.cpu().numpy()


@pytest.mark.parametrize("lg", range(1, 15))
def test_fixed_bit_exact(q, lg):
    N = 1 << lg
    z = _cases(N, 900 + lg)
    X, E = _gpu_fx(q, z)
    Xo, Eo = orc.cdft_fx(z)
    assert np.array_equal(E, Eo)
    assert np.array_equal(X, Xo)


@pytest.mark.parametrize("lg,rows", [(4, 5000), (10, 1200), (12, 400), (13, 320), (14, 200)])
def test_fixed_many_rows_per_cta(q, lg, rows):
    """More rows than resident CTAs: every CTA loops over rows (shared memory reused)."""
    N = 1 << lg
    z = inputs.q15_complex(rows, N, seed=950 + lg)
    X, E = _gpu_fx(q, z)
    Xo, Eo = orc.cdft_fx(z)
    assert np.array_equal(E, Eo) and np.array_equal(X, Xo)


@pytest.mark.parametrize("lg", [10, 13])
def test_fixed_full_batch_sampled(q, lg):
    """2^26 samples (256 MiB in, 512 MiB out); 64 seeded rows against the oracle."""
    N = 1 << lg
    rows = (1 << 26) // N
    z = torch.randint(-32768, 32768, (rows, N, 2), dtype=torch.int32, generator=torch.Generator().manual_seed(lg))
    z = z.to(torch.int16)
    X, E = q.fft_fixed(z.cuda())
    torch.cuda.synchronize()
    pick = np.sort(np.random.default_rng(lg).choice(rows, 64, replace=False))
    Xo, Eo = orc.cdft_fx(z[pick].numpy())
    assert np.array_equal(E.cpu().numpy()[pick], Eo)
    assert np.array_equal(X[torch.from_numpy(pick).cuda()].cpu().numpy(), Xo)


def test_fixed_deterministic_and_accurate(q):
    N = 4096
    z = inputs.q15_complex(64, N, seed=970)
    X1, E1 = _gpu_fx(q, z)
    X2, E2 = _gpu_fx(q, z)
    assert np.array_equal(X1, X2) and np.array_equal(E1, E2)
    zf = (z[..., 0] + 1j * z[..., 1]) / 2.0 ** 15
    ref = np.fft.fft(zf.astype(np.complex128), axis=-1)
    err = np.linalg.norm(orc.fx_value(X1, E1) - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert err.max() < 1e-6


def test_fixed_abi_errors(q):
    lib = q.load_library()
    h = ctypes.c_void_p()
    assert lib.qft_plan_create(ctypes.byref(h), 1 << 15, 4, q.KIND_C2C, q.DTYPE_I16, 0) == -1   # INVALID_N
    assert lib.qft_plan_create(ctypes.byref(h), 1 << 10, 4, q.KIND_R2C, q.DTYPE_I16, 0) == -3   # DTYPE
    assert lib.qft_plan_create(ctypes.byref(h), 1 << 10, 4, q.KIND_C2C, q.DTYPE_I16, 1) == -9   # flags
    p = q.Plan(1024, 4, q.KIND_C2C, q.DTYPE_I16)
    z = torch.zeros((4, 1024, 2), dtype=torch.int16, device="cuda")
    X = torch.empty((4, 1024, 2), dtype=torch.int32, device="cuda")
    E = torch.empty(4, dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    assert lib.qft_execute(p.handle, 0, vp(z.data_ptr()), vp(X.data_ptr()), None) == -3        # use _fixed
    assert lib.qft_execute_fixed(p.handle, vp(z.data_ptr()), vp(X.data_ptr() + 4), vp(E.data_ptr()), None) == -4
    assert lib.qft_execute_fixed(p.handle, vp(z.data_ptr()), vp(X.data_ptr()), None, None) == -5
    assert lib.qft_execute_fixed(p.handle, vp(X.data_ptr()), vp(X.data_ptr()), vp(E.data_ptr()), None) == -10
    assert lib.qft_execute_fixed(p.handle, vp(z.data_ptr()), vp(X.data_ptr()), vp(E.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert not X.any() and not E.any()
    f = q.Plan(1024, 4)
    assert lib.qft_execute_fixed(f.handle, vp(z.data_ptr()), vp(X.data_ptr()), vp(E.data_ptr()), None) == -3
    empty = q.Plan(1024, 0, q.KIND_C2C, q.DTYPE_I16)
    assert lib.qft_execute_fixed(empty.handle, None, None, None, None) == 0
    for pl in (p, f, empty):
        pl.destroy()
