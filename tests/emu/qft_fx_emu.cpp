// Host emulation of the fixed-point kernel (test infrastructure only).
//
// Compiles the library's qft_fixed.cuh for the host and runs one row the way
// k_fixed does: every step computes all its items, takes the block maxima,
// then stores all of them.  It also checks the properties the kernel's
// warp-level reduction relies on: every item of a block reports the same
// block size, and blocks of 32 items or more start on a multiple of 32 and
// hold only working items.  The test-suite compares the result bit for bit
// with the fixed-point oracle.  The product never loads this.
#define QFT_HOST_EMULATION 1
#include "../../paper_1301_0763_gb300/csrc/qft_fixed.cuh"
#include <stdint.h>
#include <vector>

using namespace qfx;

namespace {

// block maxima of k1 / k2 over aligned runs of `seg` items; returns false if
// the block structure breaks the kernel's assumptions
bool reduce(const std::vector<Item>& it, std::vector<int>& m1, std::vector<int>& m2) {
  const int n = (int)it.size();
  std::vector<int> b1(n, 0), b2(n, 0);
  for (int w = 0; w < n; ++w) {
    const int sg = it[w].seg;
    if (!sg) continue;
    if (sg & (sg - 1)) return false;
    const int b = w & ~(sg - 1);
    if (b + sg > n) return false;
    for (int v = b; v < b + sg; ++v)
      if (it[v].seg != sg) return false;   // same block size everywhere in the block
    b1[b] = imax(b1[b], it[w].k1);
    b2[b] = imax(b2[b], it[w].k2);
  }
  m1.assign(n, 0);
  m2.assign(n, 0);
  for (int w = 0; w < n; ++w) {
    const int sg = it[w].seg;
    if (!sg) continue;
    m1[w] = b1[w & ~(sg - 1)];
    m2[w] = b2[w & ~(sg - 1)];
  }
  return true;
}

int row(int r, const uint32_t* z, Cell* out, int* E, const std::vector<Sec>& sec) {
  const int N = 1 << r, H = N / 2;
  if (N == 2) { row_n2(z, out, E); return 0; }
  std::vector<Cell> V0(H + 2), V1(H + 2);
  std::vector<int16_t> X0(N, 0x5555), X1(N, 0x5555);   // garbage: every read must follow a write
  std::vector<int> ch(32, 0x5555);
  Row R;
  R.V0 = V0.data(); R.V1 = V1.data(); R.X0 = X0.data(); R.X1 = X1.data(); R.ch = ch.data();
  R.sec = sec.data(); R.r = r; R.N = N;
  std::vector<int> m1, m2;
  {
    std::vector<Item> it(N);
    fold_base(R, z);
    for (int w = 0; w < N; ++w) fold_compute(R, z, w, it[w]);
    if (!reduce(it, m1, m2)) return -2;
    for (int w = 0; w < N; ++w) if (it[w].seg) fold_write(R, w, it[w], m1[w]);
  }
  for (int dep = 0; dep <= r - 3; ++dep) {
    std::vector<Item> it(H);
    for (int w = 0; w < H; ++w) fwd_compute(R, dep, w, it[w]);
    if (!reduce(it, m1, m2)) return -3;
    for (int w = 0; w < H; ++w) if (it[w].seg) fwd_write(R, dep, w, it[w], m1[w], m2[w]);
  }
  for (int h = 1; h <= r - 1; ++h) {
    std::vector<Item> it(N);
    for (int w = 0; w < N; ++w) bwd_compute(R, h, w, it[w]);
    if (!reduce(it, m1, m2)) return -4;
    for (int w = 0; w < N; ++w) if (it[w].seg) bwd_write(R, h, w, it[w], m1[w]);
  }
  {
    std::vector<Item> it(H);
    for (int w = 0; w < H; ++w) fin_compute(R, w, it[w]);
    if (!reduce(it, m1, m2)) return -5;
    for (int w = 0; w < H; ++w) fin_write(R, w, m1[w], out, E);
  }
  return 0;
}

}  // namespace

extern "C" int emu_cdft_fx(int N, int64_t batch, const uint32_t* z, int32_t* out, int32_t* E) {
  int r = 0;
  while ((1 << r) < N) ++r;
  if (N < 2 || (1 << r) != N || r > kMaxLog2) return -1;
  std::vector<Sec> sec(N >= 8 ? N / 4 - 1 : 1);
  if (N >= 8) fill_consts(N, sec.data());
  for (int64_t b = 0; b < batch; ++b) {
    int e = 0;
    const int rc = row(r, z + b * N, reinterpret_cast<Cell*>(out) + b * N, &e, sec);
    if (rc) return rc;
    E[b] = e;
  }
  return 0;
}
