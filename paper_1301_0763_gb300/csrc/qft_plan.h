// qft_plan.h -- schedule tables of the improved-QFT row engine (host + device POD).
//
// A row of length N = 2^r is transformed by the improved QFT (Sec. 5 of the
// paper) as a sequence of phases separated by block-wide barriers.  Every phase
// is a flat list of independent tasks grouped in segments; a segment names the
// signal being worked on (DCT or DST side, 2-adic class j) and how many levels
// of the decomposition tree one task performs in registers.
//
//   F1     load the row, fold it (rdft forward relations, Sec. 4.2) and do the
//          first L1 mirror-butterfly levels of every large class (eqs qft_1,
//          qft_2, qft_38A); small classes are transformed completely.
//   DIF    further mirror-butterfly levels, in place.
//   LEAF   the last forward levels of a node plus its whole backward phase.
//   SLICE  backward levels (eqs qft_4B, qft_38B/C) of the upper tree.
//   FINAL  class combines (eqs qft_5C, qft_5D, qft_6) and the CDFT combine
//          (Sec. 4.1), then the store of the spectrum.
#pragma once
#include <stdint.h>

#define QFT_MAX_PHASES 16
#define QFT_MAX_SEGS 128

enum QftSegType {
  QFT_SEG_F1_BIG = 1,   // one task = 2^L1 Gray slots of a large class, both sides
  QFT_SEG_F1_SMALL = 2, // one task = a whole small class (forward + backward), both sides
  QFT_SEG_F1_BASE = 3,  // c(0), c(N/2)
  QFT_SEG_DIF = 4,      // one task = 2^L slots of one node, L mirror levels
  QFT_SEG_LEAF = 5,     // one task = one node of 2^L cells, forward + backward
  QFT_SEG_SLICE = 6,    // one task = one output chunk of 2^L values of one node
  QFT_SEG_FIN_REG = 7,  // one task = the 2^(LF+1) outputs of one frequency orbit
  QFT_SEG_FIN_SPEC = 8  // one task = one output pair at a multiple of N/2^(LF+1)
};

struct QftSeg {
  uint8_t type;   // QftSegType
  uint8_t side;   // 0: DCT side (s_dc_*), 1: DST side (s_ds_*)
  uint8_t cls;    // 2-adic class j: time indices n = 2^j * odd
  uint8_t L;      // levels done by one task
  uint8_t D;      // depth of the class tree before this phase
  uint8_t pad[3];
  int32_t begin;  // first task index of the segment within its phase
  int32_t count;  // number of tasks
};

struct QftRowPlan {
  int32_t r;        // log2 N
  int32_t L1;       // levels done in F1
  int32_t LF;       // class-combine levels done per FINAL task
  int32_t nphase;
  int32_t nseg;
  int32_t max_slice_nodes;  // largest number of tasks sharing one node in a SLICE phase
  int32_t phase_ntasks[QFT_MAX_PHASES];
  int32_t phase_seg0[QFT_MAX_PHASES + 1];
  int32_t phase_is_slice[QFT_MAX_PHASES];
  QftSeg segs[QFT_MAX_SEGS];
};
