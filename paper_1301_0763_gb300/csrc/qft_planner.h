// qft_planner.h -- builds the phase/segment schedule (QftRowPlan) of the row
// engine for one transform length N = 2^r.  Host code only.
//
// Tuning knobs (the "tile/stage schedule" of a plan):
//   L1  mirror levels done while loading the row (register tile 2^L1 per side)
//   LS  levels per in-place DIF phase
//   LL  forward levels left for the LEAF phase (which then does the same
//       number of backward levels in registers)
//   LB  backward levels per SLICE phase
//   LF  class-combine levels per FINAL task (tile 2^(LF+1) outputs)
#pragma once
#include <string.h>
#include "qft_plan.h"

struct QftTune {
  int L1, LS, LL, LB, LF;
};

// The library's schedule: register tiles of 8 cells per side in F1 and SLICE,
// 16 in DIF, 8 in LEAF, 16 output bins per FINAL task; 256 threads per CTA
// (512 for N = 2^14, whose top SLICE phase has 512 tasks per node).
static inline QftTune qft_default_tune(int r) {
  QftTune t;
  t.L1 = 3; t.LS = 4; t.LL = 3; t.LB = 3; t.LF = 3;
  (void)r;
  return t;
}

static inline int qft_default_threads(int r) { return r >= 14 ? 512 : 256; }

namespace qft_planner_detail {
struct Builder {
  QftRowPlan* P;
  int cur_begin;
  bool open;
  void begin(int is_slice) {
    P->phase_seg0[P->nphase] = P->nseg;
    P->phase_is_slice[P->nphase] = is_slice;
    P->phase_ntasks[P->nphase] = 0;
    cur_begin = 0;
    open = true;
  }
  bool add(int type, int side, int cls, int L, int D, int count) {
    if (P->nseg >= QFT_MAX_SEGS || count <= 0) return count <= 0;
    QftSeg& s = P->segs[P->nseg++];
    memset(&s, 0, sizeof s);
    s.type = (uint8_t)type; s.side = (uint8_t)side; s.cls = (uint8_t)cls;
    s.L = (uint8_t)L; s.D = (uint8_t)D;
    s.begin = cur_begin; s.count = count;
    cur_begin += count;
    return true;
  }
  // returns false if the phase is empty (and drops it)
  bool end() {
    open = false;
    if (P->nseg == P->phase_seg0[P->nphase]) return false;
    P->phase_ntasks[P->nphase] = cur_begin;
    P->nphase++;
    P->phase_seg0[P->nphase] = P->nseg;
    return true;
  }
};
}  // namespace qft_planner_detail

// Returns 0 on success, -1 for an unsupported r or tuning.
static inline int qft_build_row_plan(int r, QftTune t, QftRowPlan* P) {
  using qft_planner_detail::Builder;
  memset(P, 0, sizeof *P);
  if (r < 2 || r > 24) return -1;
  if (t.L1 < 0 || t.L1 > 4 || t.LS < 1 || t.LS > 4 || t.LL < 1 || t.LL > 4 || t.LB < 1 || t.LB > 4 ||
      t.LF < 0 || t.LF > 3)
    return -1;
  int LF = t.LF;
  if (LF > r - 2) LF = r - 2;
  P->r = r; P->L1 = t.L1; P->LF = LF;
  const int ncls = r - 1;          // DCT classes 0..r-2 (DST: 0..r-3)
  int depth[32];
  bool big[32];
  for (int j = 0; j < ncls; ++j) {
    const int b = r - 2 - j;
    big[j] = b > t.L1;
    depth[j] = big[j] ? t.L1 : 0;
  }
  Builder B;
  B.P = P;
  // ---- F1
  B.begin(0);
  for (int j = 0; j < ncls; ++j)
    if (big[j] && !B.add(QFT_SEG_F1_BIG, 0, j, t.L1, 0, 1 << (r - 2 - j - t.L1))) return -1;
  for (int j = 0; j < ncls; ++j)
    if (!big[j] && !B.add(QFT_SEG_F1_SMALL, 0, j, r - 2 - j, 0, 1)) return -1;
  if (!B.add(QFT_SEG_F1_BASE, 0, 0, 0, 0, 1)) return -1;
  B.end();
  // ---- DIF phases
  for (;;) {
    int Ls[32];
    bool any = false;
    for (int j = 0; j < ncls; ++j) {
      Ls[j] = 0;
      if (!big[j]) continue;
      const int rem = (r - 2 - j) - depth[j];
      int L = rem - t.LL;
      if (L > t.LS) L = t.LS;
      if (L > 0) { Ls[j] = L; any = true; }
    }
    if (!any) break;
    B.begin(0);
    for (int side = 0; side < 2; ++side)
      for (int j = 0; j < ncls; ++j)
        if (Ls[j] > 0 && !B.add(QFT_SEG_DIF, side, j, Ls[j], depth[j], 1 << (r - 2 - j - Ls[j]))) return -1;
    B.end();
    for (int j = 0; j < ncls; ++j) depth[j] += Ls[j];
  }
  // ---- LEAF
  B.begin(0);
  for (int side = 0; side < 2; ++side)
    for (int j = 0; j < ncls; ++j)
      if (big[j]) {
        const int L = (r - 2 - j) - depth[j];
        if (L < 1 || L > 4) return -1;
        if (!B.add(QFT_SEG_LEAF, side, j, L, depth[j], 1 << depth[j])) return -1;
      }
  B.end();
  // ---- SLICE phases (segments sorted by decreasing node task count S)
  for (;;) {
    int Ls[32];
    bool any = false;
    for (int j = 0; j < ncls; ++j) {
      Ls[j] = 0;
      if (!big[j] || depth[j] == 0) continue;
      // the remainder first, so that the top phase always spans LB levels and
      // the number of tasks sharing one node there is 2^(b_j - LB)
      Ls[j] = depth[j] % t.LB;
      if (Ls[j] == 0) Ls[j] = t.LB;
      any = true;
    }
    if (!any) break;
    B.begin(1);
    // S_j = 2^(b_j - depth_j); emit in decreasing S
    for (int sb = 30; sb >= 0; --sb)
      for (int side = 0; side < 2; ++side)
        for (int j = 0; j < ncls; ++j)
          if (Ls[j] > 0 && (r - 2 - j) - depth[j] == sb) {
            if (!B.add(QFT_SEG_SLICE, side, j, Ls[j], depth[j], 1 << (r - 2 - j - Ls[j]))) return -1;
            if ((1 << sb) > P->max_slice_nodes) P->max_slice_nodes = 1 << sb;
          }
    B.end();
    for (int j = 0; j < ncls; ++j) depth[j] -= Ls[j];
  }
  // ---- FINAL
  B.begin(0);
  const int W = 1 << (r - LF - 1);
  if (W >= 2 && !B.add(QFT_SEG_FIN_REG, 0, 0, LF, 0, W - 1)) return -1;
  if (!B.add(QFT_SEG_FIN_SPEC, 0, 0, LF, 0, (1 << LF) + 1)) return -1;
  B.end();
  return 0;
}
