"""Host emulation of the fixed-point kernel (qft_fixed.cuh built for the CPU,
steps run as the kernel runs them) against the fixed-point oracle: every
mantissa and exponent equal, for N = 2 .. 2^14 and the edge cases (zeros,
full scale, impulses, sparse and real input, tiny values).  The emulation also
checks the block structure the kernel's warp reduction relies on."""
import os
import sys

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_0763_gb300 import inputs

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "emu"))
import emu  # noqa: E402


def _cases(N, seed):
    cs = [inputs.q15_complex(4, N, seed=seed),
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


@pytest.mark.parametrize("lg", range(1, 15))
def test_fixed_emulation_bit_exact(lg):
    N = 1 << lg
    z = _cases(N, 800 + lg)
    X, E = emu.cdft_fx(z)
    Xo, Eo = orc.cdft_fx(z)
    assert np.array_equal(E, Eo)
    assert np.array_equal(X, Xo)
