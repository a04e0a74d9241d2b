"""GPU parity of the one-scratch (in-place) schedule of the large-row path
(QFT_PLAN_IN_PLACE, Sec. 6.1): the backward levels above the node depth
overwrite the cells they read, so a plan keeps one scratch copy of the class
data instead of two.  The arithmetic is unchanged, so every result must equal
the FP32 evaluation of the recursion (the oracle) bit for bit, as without the
flag.  Calls go through the C ABI (qft_execute via ctypes)."""
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


def bits_equal(a, b):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def run(q, n, rows, op, x, kind=0, dtype=0, out_shape=None, out_dtype=torch.complex64, plain=False, **sched):
    p = q.Plan(n, rows, kind, dtype, in_place=True, plain=plain)
    if sched:
        p.set_schedule(**sched)
    xin = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = torch.empty(out_shape or (rows, n), dtype=out_dtype, device="cuda")
    p.execute(op, xin, out)
    torch.cuda.synchronize()
    assert p.sync_status() == 0
    res = out.cpu().numpy()
    p.destroy()
    return res


@pytest.mark.parametrize("lg", [15, 16, 17, 18, 20])
def test_in_place_forward_bit_exact(q, lg):
    N = 1 << lg
    z = inputs.normal_complex(3, N, seed=300 + lg)
    X = run(q, N, 3, q.OP_FORWARD, z)
    assert bits_equal(X, orc.cdft(z, fp32=True).astype(np.complex64))


def test_in_place_plain_fp32(q):
    N = 1 << 18
    z = inputs.normal_complex(2, N, seed=318)
    X = run(q, N, 2, q.OP_FORWARD, z, plain=True)
    assert bits_equal(X, orc.cdft(z, fp32=True, comp=False).astype(np.complex64))


@pytest.mark.parametrize("lg,node_log2", [(16, 8), (18, 9), (18, 10)])
def test_in_place_small_nodes(q, lg, node_log2):
    """Smaller node groups leave more backward levels to the in-place SLICE
    phases (several phases a class, each over the order the one below left;
    many block edges inside one node, whose neighbour cells go through the
    halo copy)."""
    N = 1 << lg
    z = inputs.normal_complex(2, N, seed=330 + node_log2)
    X = run(q, N, 2, q.OP_FORWARD, z, node_log2=node_log2)
    assert bits_equal(X, orc.cdft(z, fp32=True).astype(np.complex64))


@pytest.mark.parametrize("op", [1, 2, 3])
def test_in_place_other_ops(q, op):
    N = 1 << 17
    z = inputs.uniform_complex(2, N, seed=340 + op)
    out = run(q, N, 2, op, z)
    ref32 = {1: lambda: orc.icdft(z, fp32=True), 2: lambda: orc.cdft_adjoint(z, fp32=True),
             3: lambda: orc.cdft(z, fp32=True) / N}[op]()
    assert bits_equal(out, ref32.astype(np.complex64))


def test_in_place_real(q):
    N = 1 << 18
    H = N // 2 + 1
    x = inputs.normal_real(3, N, seed=350)
    X = run(q, N, 3, q.OP_FORWARD, x, kind=q.KIND_R2C, out_shape=(3, H))
    assert bits_equal(X, orc.rdft(x, fp32=True).astype(np.complex64))
    xr = run(q, N, 3, q.OP_INVERSE, X, kind=q.KIND_R2C, out_shape=(3, N), out_dtype=torch.float32)
    assert bits_equal(xr, orc.irdft(X, N, fp32=True).astype(np.float32))


def test_in_place_n2_24_one_scratch_copy(q):
    """One N = 2^24 transform and its adjoint with one scratch copy: the plan
    holds about half the scratch of the two-copy plan."""
    N = 1 << 24
    z = inputs.normal_complex(1, N, seed=360)
    p2 = q.Plan(N, 1)
    p1 = q.Plan(N, 1, in_place=True)
    two, one = p2.scratch_bytes(), p1.scratch_bytes()
    p2.destroy()
    # one copy of the class data (2 (N/2 + 1) cells, padded by 1/16) and of
    # its lo parts fewer, plus halo copies of 8 cells per block edge (h, lo)
    cells = 2 * ((N // 2 + N // 32 + 2) & ~1) * 8 * 2
    halo = 2 * (N // 512 + 2) * 8 * 8
    assert two - one == cells - halo and one < 0.55 * two
    xin = torch.from_numpy(z).cuda()
    out = torch.empty_like(xin)
    p1.execute(q.OP_FORWARD, xin, out)
    torch.cuda.synchronize()
    assert bits_equal(out.cpu().numpy(), orc.cdft(z, fp32=True).astype(np.complex64))
    p1.execute(q.OP_FORWARD_ADJOINT, xin, out)
    torch.cuda.synchronize()
    assert bits_equal(out.cpu().numpy(), orc.cdft_adjoint(z, fp32=True).astype(np.complex64))
    assert p1.sync_status() == 0
    p1.destroy()


def _bf16_round(x):
    """float32 -> bfloat16 bits, round to nearest even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


@pytest.mark.parametrize("half", ["f16", "bf16"])
def test_in_place_half_storage(q, half):
    """FP16 / BF16 rows of 2^16 on the in-place schedule: the stored result is
    the FP32 oracle of the rounded input, rounded to the storage type."""
    N, rows = 1 << 16, 3
    z = inputs.uniform_complex(rows, N, seed=370).view(np.float32).reshape(rows, N, 2)
    if half == "f16":
        zin = z.astype(np.float16)
        zf = zin.astype(np.float32)
        t = torch.from_numpy(zin).cuda().view(torch.complex32).reshape(rows, N)
        p = q.Plan(N, rows, q.KIND_C2C, q.DTYPE_F16, in_place=True)
    else:
        bits = _bf16_round(z)
        zf = (bits.astype(np.uint32) << 16).view(np.float32)
        t = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
        p = q.Plan(N, rows, q.KIND_C2C, q.DTYPE_BF16, in_place=True)
    out = torch.empty_like(t)
    p.execute(q.OP_FORWARD, t, out)
    torch.cuda.synchronize()
    ob = out.cpu().view(torch.int16).numpy().view(np.uint16).reshape(rows, N, 2)
    ref = orc.cdft(zf[..., 0].astype(np.float64) + 1j * zf[..., 1], fp32=True)
    ref = ref.astype(np.complex64).view(np.float32).reshape(rows, N, 2)
    assert np.array_equal(ob, ref.astype(np.float16).view(np.uint16) if half == "f16" else _bf16_round(ref))
    p.destroy()


def test_in_place_many_rows_sampled(q):
    """256 rows of 2^20 (2^28 elements, the batched workload's largest size) on
    the in-place schedule; sampled rows against the oracle."""
    N = 1 << 20
    rows = 256
    z = torch.randn(rows, N, dtype=torch.complex64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(380))
    p = q.Plan(N, rows, in_place=True)
    X = torch.empty_like(z)
    p.execute(q.OP_FORWARD, z, X)
    torch.cuda.synchronize()
    assert p.sync_status() == 0
    idx = np.array([0, 1, 77, 254, 255])
    zs = z[idx].cpu().numpy()
    assert bits_equal(X[idx].cpu().numpy(), orc.cdft(zs, fp32=True).astype(np.complex64))
    p.destroy()
    del z, X
    torch.cuda.empty_cache()


def test_in_place_ragged(q):
    """A ragged plan with the flag: every length class on its own schedule."""
    lgs = np.array([16, 4, 15, 10, 16, 17], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(1 << lgs.astype(np.int64))])
    z = inputs.normal_complex(1, int(off[-1]), seed=390)[0]
    p = q.RaggedPlan(off, lgs, in_place=True)
    xin = torch.from_numpy(z).cuda()
    out = torch.empty_like(xin)
    p.execute(q.OP_FORWARD, xin, out)
    torch.cuda.synchronize()
    X = out.cpu().numpy()
    for i, lg in enumerate(lgs):
        seg = slice(int(off[i]), int(off[i + 1]))
        assert bits_equal(X[seg], orc.cdft(z[None, seg], fp32=True).astype(np.complex64)[0]), lg
    p.destroy()


def test_in_place_autotuned_and_scratch_accounting(q):
    """An autotuned in-place plan keeps the in-place schedule under every
    candidate (same bits); scratch_bytes of a ragged plan is the sum of its
    length classes'."""
    N = 1 << 18
    z = inputs.normal_complex(4, N, seed=400)
    p = q.Plan(N, 4, in_place=True, autotune=True)
    xin = torch.from_numpy(z).cuda()
    out = torch.empty_like(xin)
    p.execute(q.OP_FORWARD, xin, out)
    torch.cuda.synchronize()
    assert bits_equal(out.cpu().numpy(), orc.cdft(z, fp32=True).astype(np.complex64))
    assert p.sync_status() == 0
    one = p.scratch_bytes()
    p.destroy()
    p2 = q.Plan(N, 4)
    assert one < 0.6 * p2.scratch_bytes()
    p2.destroy()
    small = q.Plan(1 << 12, 4, in_place=True)
    assert small.scratch_bytes() == 0
    small.destroy()
    lgs = np.array([16, 12, 17], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(1 << lgs.astype(np.int64))])
    rp = q.RaggedPlan(off, lgs, in_place=True)
    parts = [q.Plan(1 << 16, 1, in_place=True), q.Plan(1 << 17, 1, in_place=True)]
    assert rp.scratch_bytes() == sum(pp.scratch_bytes() for pp in parts)
    for pp in parts + [rp]:
        pp.destroy()
