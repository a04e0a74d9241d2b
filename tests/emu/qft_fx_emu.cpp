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

// One step's keys -> block maxima over aligned runs of `seg` items; false if
// the block structure breaks the kernel's assumptions.
bool reduce(const std::vector<int>& seg, const std::vector<int>& k1, const std::vector<int>& k2,
            std::vector<int>& m1, std::vector<int>& m2) {
  const int n = (int)seg.size();
  std::vector<int> b1(n, 0), b2(n, 0);
  for (int w = 0; w < n; ++w) {
    const int sg = seg[w];
    if (!sg) continue;
    if (sg & (sg - 1)) return false;
    const int b = w & ~(sg - 1);
    if (b + sg > n) return false;
    for (int v = b; v < b + sg; ++v)
      if (seg[v] != sg) return false;   // same block size everywhere in the block
    b1[b] = imax(b1[b], k1[w]);
    b2[b] = imax(b2[b], k2[w]);
  }
  m1.assign(n, 0);
  m2.assign(n, 0);
  for (int w = 0; w < n; ++w) {
    if (!seg[w]) continue;
    m1[w] = b1[w & ~(seg[w] - 1)];
    m2[w] = b2[w & ~(seg[w] - 1)];
  }
  return true;
}

// the kernel's two phases of a step: evaluate every item, reduce, store every item
template <class EV, class ST>
bool step(int items, EV ev, ST st) {
  std::vector<Val> v(items);
  std::vector<int> sg(items), k1(items), k2(items), m1, m2;
  for (int w = 0; w < items; ++w) {
    ev(w, v[w]);
    sg[w] = v[w].seg;
    k1[w] = v[w].k1;
    k2[w] = v[w].k2;
  }
  if (!reduce(sg, k1, k2, m1, m2)) return false;
  for (int w = 0; w < items; ++w)
    if (sg[w]) st(w, v[w], m1[w], m2[w]);
  return true;
}

int row(int r, const uint32_t* z, Cell* out, int* E, const std::vector<Sec>& sec) {
  const int N = 1 << r, H = N / 2;
  if (N == 2) { row_n2(z, out, E); return 0; }
  // the row's shared-memory image; garbage everywhere, so that a read before a write shows
  std::vector<unsigned char> mem(row_bytes(N), 0x55);
  const Row R = make_row(mem.data(), r, sec.data());
  uint32_t* zs = staged(R);
  for (int n = 0; n < N; ++n) zs[n] = z[n];
  fold_base(R, zs);
  if (!step(H, [&](int w, Val& v) { fold_eval(R, zs, w, v); },
            [&](int w, const Val& v, int m1, int) { fold_store(R, w, v, m1); }))
    return -2;
  for (int dep = 0; dep <= r - 3; ++dep)
    if (!step(N / 4, [&](int w, Val& v) { fwd_eval(R, dep, w, v); },
              [&](int w, const Val& v, int m1, int m2) { fwd_store(R, dep, w, v, m1, m2); }))
      return -3;
  for (int h = 1; h <= r - 1; ++h)
    if (!step(H, [&](int w, Val& v) { bwd_eval(R, h, w, v); },
              [&](int w, const Val& v, int m1, int) { bwd_store(R, h, w, v, m1); }))
      return -4;
  if (!step(H, [&](int w, Val& v) { fin_eval(R, w, v); },
            [&](int w, const Val& v, int m1, int) { fin_store(R, w, v, m1, out, E); }))
    return -5;
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
