"""Pins of the fixed-point oracle (oracle/qft_oracle_fx.c): the improved QFT of
Sec. 5 on int16 input with int32 block-floating-point arithmetic (the scaling
rule is this project's reading; the paper names fixed point as its target
application, Sec. 1 and 7, but gives no rule).

Each pin is independent of the oracle's own code:
 * N = 2 and N = 4 use no constant, so every value is exact: the result
   equals the integer DFT;
 * impulses at n = 0, N/2, N/4 pass through adds only (every secant product
   block is zero), so the result is exact: q, q(-1)^k, q(-i)^k;
 * real input gives an exactly Hermitian spectrum (the CDFT combine of
   Sec. 4.1 and one shared output exponent);
 * block floating point is scale invariant: 2z gives the same mantissas with
   the exponent one larger; outputs are normalized to 29 bits;
 * the result equals the long-double DFT within the bound the FP32 path
   meets, and is closer to it than the plain FP32 evaluation of the same
   recursion;
 * the secant constants are within half a unit of the 31-bit mantissa of the
   exact secant (mpmath, 200 bits); the rounding rule is half up.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_0763_gb300 import inputs

Q = 2.0 ** 15


def _dft_int(z):
    """Exact integer DFT for N <= 4 (twiddles are 1, -i, -1, i)."""
    N = z.shape[-2]
    zc = z[..., 0].astype(np.int64) + 1j * z[..., 1].astype(np.int64)
    W = {0: 1, 1: -1j, 2: -1, 3: 1j}
    step = 4 // N if N <= 4 else None
    out = np.zeros(zc.shape, dtype=np.complex128)
    for k in range(N):
        for n in range(N):
            out[..., k] += zc[..., n] * W[(n * k * step) % 4]
    return out


@pytest.mark.parametrize("N", [2, 4])
def test_small_sizes_are_exact(N):
    z = inputs.q15_complex(64, N, seed=700 + N)
    X, E = orc.cdft_fx(z)
    assert np.array_equal(orc.fx_value(X, E) * Q, _dft_int(z))


@pytest.mark.parametrize("lg", range(1, 15))
def test_impulses_are_exact(lg):
    N = 1 << lg
    P = [1, -1j, -1, 1j]
    cases = [(0, lambda k: 1), (N // 2, lambda k: (-1) ** k)]
    if N >= 4:
        cases.append((N // 4, lambda k: P[k % 4]))
    for n0, f in cases:
        for q in (12345, -32768, 1):
            z = np.zeros((1, N, 2), np.int16)
            z[0, n0, 0] = q
            X, E = orc.cdft_fx(z)
            ref = np.array([q * f(k) for k in range(N)])
            assert np.array_equal(orc.fx_value(X, E)[0] * Q, ref), (N, n0, q)


@pytest.mark.parametrize("lg", range(1, 15))
def test_real_input_hermitian_and_zero_rows(lg):
    N = 1 << lg
    z = inputs.q15_complex(4, N, seed=710 + lg)
    z[..., 1] = 0
    X, E = orc.cdft_fx(z)
    k = np.arange(1, N)
    assert np.array_equal(X[:, k, 0], X[:, N - k, 0])
    assert np.array_equal(X[:, k, 1], -X[:, N - k, 1])
    assert np.all(X[:, 0, 1] == 0)
    Xz, Ez = orc.cdft_fx(np.zeros((2, N, 2), np.int16))
    assert not Xz.any() and np.all(Ez == 0)


@pytest.mark.parametrize("lg", range(1, 15))
def test_scale_invariance_and_normalization(lg):
    N = 1 << lg
    z = inputs.q15_complex(4, N, seed=720 + lg) // 2
    X1, E1 = orc.cdft_fx(z)
    X2, E2 = orc.cdft_fx(z * 2)
    assert np.array_equal(X1, X2) and np.array_equal(E2, E1 + 1)
    top = np.abs(X1.astype(np.int64)).max(axis=(1, 2))
    assert np.all((top >= 2 ** 28) & (top <= 2 ** 29))


def _rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("lg", range(3, 15))
def test_close_to_exact_dft_and_better_than_fp32(lg):
    N = 1 << lg
    h = 16 if lg <= 10 else 4
    z = inputs.q15_complex(h, N, seed=730 + lg)
    X, E = orc.cdft_fx(z)
    zf = (z[..., 0] + 1j * z[..., 1]) / Q
    exact = np.array([orc.fft_ld(r) for r in zf])
    err = _rel(orc.fx_value(X, E), exact)
    assert np.max(err) < 6e-8 * np.sqrt(N), (N, np.max(err))
    err32 = _rel(orc.cdft(zf, fp32=True, comp=False), exact)
    assert np.mean(err) < np.mean(err32), (N, np.mean(err), np.mean(err32))


@pytest.mark.parametrize("lg", range(3, 7))
def test_small_sizes_against_brute_force(lg):
    N = 1 << lg
    z = inputs.q15_complex(8, N, seed=740 + lg)
    X, E = orc.cdft_fx(z)
    v = orc.fx_value(X, E)
    for r in range(8):
        ref = orc.brute_dft((z[r, :, 0] + 1j * z[r, :, 1]) / Q)
        assert np.linalg.norm(v[r] - ref) / np.linalg.norm(ref) < 1e-9 * N


@pytest.mark.parametrize("N", [8, 16, 64, 1024, 8192])
def test_secant_constants(N):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    for n in sorted({1, 3, N // 8 - 1 if N >= 16 else 1, N // 8 + 1 if N >= 16 else 1, N // 4 - 1}):
        if n % 2 == 0 or n >= N // 4:
            continue
        c, x = orc.fx_const(N, n)
        assert 2 ** 30 <= c < 2 ** 31
        sec = mpmath.mpf(1) / (2 * mpmath.cos(2 * mpmath.pi * n / N))
        assert abs(mpmath.mpf(c) * mpmath.mpf(2) ** x - sec) <= mpmath.mpf(2) ** (x - 1)


def test_rounding_rule():
    """floor(v / 2^s + 1/2); s <= 0 multiplies exactly."""
    cases = [(5, 1, 3), (-5, 1, -2), (7, 2, 2), (-6, 2, -1), (-7, 2, -2), (9, 0, 9), (3, -2, 12),
             (-(2 ** 30), 1, -(2 ** 29)), (2 ** 60, 70, 0), (-(2 ** 60), 62, 0)]
    for v, s, want in cases:
        assert orc.fx_rs(v, s) == want, (v, s)


@pytest.mark.parametrize("lg,step", [(6, 2), (8, 4), (10, 2), (12, 8)])
def test_zero_blocks_do_not_cost_precision(lg, step):
    """Input supported on multiples of `step` makes the classes of smaller
    2-adic valuation zero blocks (exponent EZERO); the accuracy stays within
    the dense-input bound."""
    N = 1 << lg
    z = inputs.q15_complex(8, N, seed=750 + lg)
    z[:, np.arange(N) % step != 0, :] = 0
    X, E = orc.cdft_fx(z)
    zf = (z[..., 0] + 1j * z[..., 1]) / Q
    exact = np.array([orc.fft_ld(r) for r in zf])
    assert np.max(_rel(orc.fx_value(X, E), exact)) < 6e-8 * np.sqrt(N)
