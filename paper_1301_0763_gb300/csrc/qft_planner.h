// qft_planner.h -- builds the phase/segment schedule (QftRowPlan) of the row
// engine for one transform length N = 2^r.  Host code only.
//
// Tuning knobs (the "tile/stage schedule" of a plan):
//   L1  mirror levels done while loading the row (register tile 2^L1 per side)
//   LS  levels per in-place DIF phase
//   LL  forward levels left for the LEAF phase (which then does the same
//       number of backward levels in registers); 0 = chosen per class so that
//       the remaining backward levels are a multiple of LB
//   LB  backward levels per SLICE phase
//   LF  class-combine levels per FINAL task (tile 2^(LF+1) outputs)
#pragma once
#include <string.h>
#include "qft_plan.h"

struct QftTune {
  int L1, LS, LL, LB, LF;
};

// The library's schedule: register tiles of 8 cells per side in F1 and SLICE,
// 16 in DIF (8 from N = 2^13 on, where the autotuner prefers them), 8 in LEAF,
// 16 output bins per FINAL task; 256 threads per CTA (512 for N = 2^14, whose
// top SLICE phase has 512 tasks per node).
static inline QftTune qft_default_tune(int r) {
  QftTune t;
  t.L1 = 3; t.LS = r >= 13 ? 3 : 4; t.LL = 0; t.LB = 3; t.LF = 3;
  return t;
}

static inline int qft_default_threads(int r) { return r >= 14 ? 512 : 256; }

// Forward levels left to a LEAF task: the given LL, or (LL = 0) the value in
// [2, 4] that leaves a multiple of LB backward levels to the SLICE phases
// above it (`total` = levels from the leaf's top node up to where the SLICE
// phases stop), capped by `cap` (the forward levels still to do).
static inline int qft_leaf_levels(int total, int cap, QftTune t) {
  int LL = t.LL;
  if (LL == 0) {
    LL = 3;
    for (int c = 4; c >= 2; --c)
      if ((total - c) % t.LB == 0) { LL = c; break; }
  }
  if (LL > cap) LL = cap;
  return LL;
}

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
  // a phase without tasks (the C/S table build)
  void end_empty() {
    open = false;
    P->phase_ntasks[P->nphase] = 0;
    P->nphase++;
    P->phase_seg0[P->nphase] = P->nseg;
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
// nt > 0 (threads per CTA) balances the phases for that CTA size: the F1 tasks
// of the small classes and the base cells move to the next plain phase when
// that saves an F1 round, and (nt >= 128) the special FINAL tasks, which do
// not use the C/S tables, run in the table phase on the warps that do not
// build the tables.
static inline int qft_build_row_plan(int r, QftTune t, QftRowPlan* P, int nt = 0) {
  using qft_planner_detail::Builder;
  memset(P, 0, sizeof *P);
  if (r < 2 || r > 24) return -1;
  if (t.L1 < 0 || t.L1 > 4 || t.LS < 1 || t.LS > 4 || t.LL < 0 || t.LL > 4 || t.LB < 1 || t.LB > 4 ||
      t.LF < 0 || t.LF > 3)
    return -1;
  int LF = t.LF;
  if (LF > r - 2) LF = r - 2;
  P->r = r; P->L1 = t.L1; P->LF = LF;
  int LLj[32];
  for (int j = 0; j < r - 1; ++j) LLj[j] = qft_leaf_levels(r - 2 - j, r - 2 - j - t.L1, t);
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
  int n_big = 0, n_small = 1;
  for (int j = 0; j < ncls; ++j) {
    if (big[j]) n_big += 1 << (r - 2 - j - t.L1);
    else ++n_small;
  }
  const bool defer_small = nt > 0 && n_big > 0 && (n_big + n_small + nt - 1) / nt > (n_big + nt - 1) / nt;
  const auto add_small = [&]() -> bool {
    for (int j = 0; j < ncls; ++j)
      if (!big[j] && !B.add(QFT_SEG_F1_SMALL, 0, j, r - 2 - j, 0, 1)) return false;
    return B.add(QFT_SEG_F1_BASE, 0, 0, 0, 0, 1);
  };
  B.begin(0);
  for (int j = 0; j < ncls; ++j)
    if (big[j] && !B.add(QFT_SEG_F1_BIG, 0, j, t.L1, 0, 1 << (r - 2 - j - t.L1))) return -1;
  if (!defer_small && !add_small()) return -1;
  B.end();
  bool small_pending = defer_small;
  // ---- DIF phases
  for (;;) {
    int Ls[32];
    bool any = false;
    for (int j = 0; j < ncls; ++j) {
      Ls[j] = 0;
      if (!big[j]) continue;
      const int rem = (r - 2 - j) - depth[j];
      int L = rem - LLj[j];
      if (L > t.LS) L = t.LS;
      if (L > 0) { Ls[j] = L; any = true; }
    }
    if (!any) break;
    B.begin(0);
    for (int side = 0; side < 2; ++side)
      for (int j = 0; j < ncls; ++j)
        if (Ls[j] > 0 && !B.add(QFT_SEG_DIF, side, j, Ls[j], depth[j], 1 << (r - 2 - j - Ls[j]))) return -1;
    if (small_pending) {
      if (!add_small()) return -1;
      small_pending = false;
      P->in_last_phase = P->nphase;
    }
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
  if (small_pending) {
    if (!add_small()) return -1;
    small_pending = false;
    P->in_last_phase = P->nphase;
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
  // ---- tables of C_Mt, S_Mt for the FINAL tasks (built by warps 0 and 1; the
  // other warps may run the special FINAL tasks meanwhile)
  const bool spec_in_tab = nt >= 128;
  B.begin(2);
  if (spec_in_tab) {
    if (!B.add(QFT_SEG_FIN_SPEC, 0, 0, LF, 0, (1 << LF) + 1)) return -1;
    B.end();
  } else {
    B.end_empty();
  }
  // ---- FINAL
  B.begin(0);
  const int W = 1 << (r - LF - 1);
  if (W >= 2 && !B.add(QFT_SEG_FIN_REG, 0, 0, LF, 0, W - 1)) return -1;
  if (!spec_in_tab && !B.add(QFT_SEG_FIN_SPEC, 0, 0, LF, 0, (1 << LF) + 1)) return -1;
  B.end();
  return 0;
}

// Number of classes (of each side) whose trees the library evaluates on
// compensated pairs by default: the FP32 error of the improved QFT grows like
// ~3.5e-8 sqrt(N) (the secant conversion of eq qft_38A); running the J largest
// classes on pairs h + l divides it by about 2^J, so J = floor((log2 N - 14)/2)
// from N = 2^16 keeps it near 5e-6 for every N up to 2^24.
static inline int qft_comp_classes(int r) { return r >= 16 ? (r - 14) / 2 : 0; }

// ---------------------------------------------------------------------------
// Schedule for rows longer than one CTA's shared memory (see qft_plan.h).
// NB: log2 of the largest node (group) a CTA transforms in shared memory.
// J: classes 0..J-1 run on compensated pairs (their segments get pad[2] = 1).
// inplace: one scratch copy; every phase reads and writes copy A (the global
// SLICE levels run in place, at most 3 a phase).
static inline int qft_build_large_plan(int r, QftTune t, int NB, int node_threads, QftLargePlan* P, int J = 0,
                                       int inplace = 0) {
  memset(P, 0, sizeof *P);
  if (r < 4 || r > 24 || NB < 4 || NB > 14) return -1;
  if (t.L1 < 1 || t.L1 > 4 || t.LS < 1 || t.LS > 4 || t.LL < 0 || t.LL > 4 || t.LB < 1 || t.LB > 4 ||
      t.LF < 0 || t.LF > 3)
    return -1;
  int LF = t.LF;
  if (LF > r - 2) LF = r - 2;
  P->r = r; P->L1 = t.L1; P->LF = LF; P->NB = NB;
  if (J < 0 || J > r - 2) return -1;
  P->comp_classes = J;
  P->inplace = inplace ? 1 : 0;
  const int LBg = inplace && t.LB > 3 ? 3 : t.LB;   // backward levels of a global SLICE phase
  const int ncls = r - 1;
  int depth[32], Dn[32], nsl[32], cur[32];
  bool big[32];
  for (int j = 0; j < ncls; ++j) {
    const int b = r - 2 - j;
    big[j] = b > t.L1;
    depth[j] = big[j] ? t.L1 : 0;
    Dn[j] = big[j] ? (b - NB > t.L1 ? b - NB : t.L1) : 0;
    nsl[j] = big[j] ? (Dn[j] + LBg - 1) / LBg : 0;     // global SLICE phases of class j
    cur[j] = (!inplace && (nsl[j] & 1)) ? 1 : 0;       // copy holding the node outputs
  }
  auto add_seg = [&](int type, int side, int cls, int L, int D, int count, int src, int dst) -> bool {
    if (P->nseg >= QFT_LP_MAX_SEGS) return false;
    QftLargePhase& ph = P->phases[P->nphase];
    QftSeg& s = P->segs[P->nseg++];
    memset(&s, 0, sizeof s);
    s.type = (uint8_t)type; s.side = (uint8_t)side; s.cls = (uint8_t)cls; s.L = (uint8_t)L; s.D = (uint8_t)D;
    s.pad[0] = (uint8_t)src; s.pad[1] = (uint8_t)dst;
    s.pad[2] = (uint8_t)((type == QFT_SEG_F1_BIG || type == QFT_SEG_DIF || type == QFT_SEG_SLICE) && cls < J ? 1 : 0);
    s.begin = ph.ntasks; s.count = count;
    ph.ntasks += count;
    ph.nseg++;
    return true;
  };
  auto begin_phase = [&](int kind) {
    QftLargePhase& ph = P->phases[P->nphase];
    ph.kind = kind; ph.seg0 = P->nseg; ph.nseg = 0; ph.ntasks = 0;
  };
  auto end_phase = [&]() { if (P->phases[P->nphase].nseg > 0) P->nphase++; };
  // ---- F1
  begin_phase(QFT_LPH_GLOBAL);
  for (int j = 0; j < ncls; ++j)
    if (big[j] && !add_seg(QFT_SEG_F1_BIG, 0, j, t.L1, 0, 1 << (r - 2 - j - t.L1), 0, 0)) return -1;
  for (int j = 0; j < ncls; ++j)
    if (!big[j] && !add_seg(QFT_SEG_F1_SMALL, 0, j, r - 2 - j, 0, 1, 0, 0)) return -1;
  if (!add_seg(QFT_SEG_F1_BASE, 0, 0, 0, 0, 1, 0, 0)) return -1;
  end_phase();
  // ---- global DIF phases down to the node depth
  for (;;) {
    int Ls[32];
    bool any = false;
    for (int j = 0; j < ncls; ++j) {
      Ls[j] = 0;
      if (!big[j] || depth[j] >= Dn[j]) continue;
      Ls[j] = Dn[j] - depth[j] < t.LS ? Dn[j] - depth[j] : t.LS;
      if (j < J && Ls[j] > 3) Ls[j] = 3;   // compensated tiles hold at most 8 cells
      any = true;
    }
    if (!any) break;
    if (P->nphase >= QFT_LP_MAX_PHASES) return -1;
    begin_phase(QFT_LPH_GLOBAL);
    for (int side = 0; side < 2; ++side)
      for (int j = 0; j < ncls; ++j)
        if (Ls[j] > 0 && !add_seg(QFT_SEG_DIF, side, j, Ls[j], depth[j], 1 << (r - 2 - j - Ls[j]), 0, 0)) return -1;
    end_phase();
    for (int j = 0; j < ncls; ++j) depth[j] += Ls[j];
  }
  // ---- node phase: one sub-plan per (side, class)
  if (P->nphase >= QFT_LP_MAX_PHASES) return -1;
  P->phases[P->nphase].kind = QFT_LPH_NODE;
  P->nphase++;
  int cta = 0;
  for (int side = 0; side < 2; ++side)
    for (int j = 0; j < ncls; ++j) {
      if (!big[j]) continue;
      if (P->nsub >= QFT_LP_MAX_SUB) return -1;
      QftNodeSub& S = P->subs[P->nsub++];
      const int b = r - 2 - j;
      const int D = Dn[j];
      const int nb = b - D;
      S.side = side; S.cls = j; S.D = D; S.nb = nb;
      S.nodes = 1 << D;
      S.group = (nb < NB) ? (1 << (NB - nb)) : 1;
      if (S.group > S.nodes) S.group = S.nodes;
      S.dst = cur[j];
      S.cta_begin = cta;
      S.comp = j < J ? 1 : 0;
      cta += S.nodes / S.group;
      // sub-plan: the row-plan phases of class j below depth D, counts per group
      QftRowPlan& Q = S.plan;
      memset(&Q, 0, sizeof Q);
      Q.r = r; Q.L1 = t.L1; Q.LF = LF;
      const int gshift = D - __builtin_ctz((unsigned)S.group);   // log2(groups per row)
      auto qbegin = [&](int is_slice) {
        Q.phase_seg0[Q.nphase] = Q.nseg; Q.phase_is_slice[Q.nphase] = is_slice; Q.phase_ntasks[Q.nphase] = 0;
      };
      auto qadd = [&](int type, int L, int Dd, int count_row) -> bool {
        if (Q.nseg >= QFT_MAX_SEGS) return false;
        QftSeg& s = Q.segs[Q.nseg++];
        memset(&s, 0, sizeof s);
        s.type = (uint8_t)type; s.side = (uint8_t)side; s.cls = (uint8_t)j; s.L = (uint8_t)L; s.D = (uint8_t)Dd;
        s.pad[2] = (uint8_t)(j < J ? 1 : 0);
        s.begin = Q.phase_ntasks[Q.nphase];
        s.count = count_row >> gshift;
        Q.phase_ntasks[Q.nphase] += s.count;
        return true;
      };
      auto qend = [&]() { Q.nphase++; Q.phase_seg0[Q.nphase] = Q.nseg; };
      int dd = D;
      // compensated subs keep at most QFT_COMP_NODE_LB backward levels per
      // SLICE phase inside the node: their tasks hold h and l parts across
      // the phase's barrier
      QftTune tn = t;
      if (j < J && tn.LB > QFT_COMP_NODE_LB) tn.LB = QFT_COMP_NODE_LB;
      int LLn = qft_leaf_levels(nb, nb, tn);
      if (j < J && LLn > 3) LLn = 3;   // compensated tiles hold at most 8 cells
      while (b - dd > LLn) {   // DIF inside the node
        int L = b - dd - LLn;
        if (L > t.LS) L = t.LS;
        if (j < J && L > 3) L = 3;
        qbegin(0);
        if (!qadd(QFT_SEG_DIF, L, dd, 1 << (b - L))) return -1;
        qend();
        dd += L;
      }
      qbegin(0);                // LEAF
      if (!qadd(QFT_SEG_LEAF, b - dd, dd, 1 << dd)) return -1;
      qend();
      while (dd > D) {          // SLICE inside the node (remainder first)
        int L = (dd - D) % tn.LB;
        if (L == 0) L = tn.LB;
        qbegin(1);
        if (!qadd(QFT_SEG_SLICE, L, dd, 1 << (b - L))) return -1;
        qend();
        const int Snode = 1 << (b - dd);
        if (Snode > P->max_slice_nodes) P->max_slice_nodes = Snode;
        dd -= L;
      }
      if (P->max_slice_nodes > node_threads) return -1;
    }
  P->node_ctas = cta;
  // ---- global SLICE phases (remainder first), ping-pong between the copies, or in place in copy A
  for (int j = 0; j < ncls; ++j) depth[j] = big[j] ? Dn[j] : 0;
  for (;;) {
    int Ls[32];
    bool any = false;
    for (int j = 0; j < ncls; ++j) {
      Ls[j] = 0;
      if (!big[j] || depth[j] == 0) continue;
      Ls[j] = depth[j] % LBg;
      if (Ls[j] == 0) Ls[j] = LBg;
      any = true;
    }
    if (!any) break;
    if (P->nphase >= QFT_LP_MAX_PHASES) return -1;
    begin_phase(QFT_LPH_SLICE);
    for (int side = 0; side < 2; ++side)
      for (int j = 0; j < ncls; ++j)
        if (Ls[j] > 0 && !add_seg(QFT_SEG_SLICE, side, j, Ls[j], depth[j], 1 << (r - 2 - j - Ls[j]),
                                  cur[j], inplace ? 0 : cur[j] ^ 1)) return -1;
    end_phase();
    for (int j = 0; j < ncls; ++j)
      if (Ls[j] > 0) { depth[j] -= Ls[j]; if (!inplace) cur[j] ^= 1; }
  }
  for (int j = 0; j < ncls; ++j)
    if (big[j] && cur[j] != 0) return -1;   // every class output must end in copy A
  // ---- C_Mt / S_Mt tables of the FINAL tasks (Mt = N / 2^LF)
  if (P->nphase >= QFT_LP_MAX_PHASES) return -1;
  P->phases[P->nphase].kind = QFT_LPH_TAB;
  P->phases[P->nphase].seg0 = P->nseg;
  P->phases[P->nphase].nseg = 0;
  P->phases[P->nphase].ntasks = 0;
  P->nphase++;
  // ---- FINAL
  if (P->nphase >= QFT_LP_MAX_PHASES) return -1;
  begin_phase(QFT_LPH_GLOBAL);
  const int W = 1 << (r - LF - 1);
  if (W >= 2 && !add_seg(QFT_SEG_FIN_REG, 0, 0, LF, 0, W - 1, 0, 0)) return -1;
  if (!add_seg(QFT_SEG_FIN_SPEC, 0, 0, LF, 0, (1 << LF) + 1, 0, 0)) return -1;
  end_phase();
  return 0;
}
