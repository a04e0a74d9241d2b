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
  int32_t in_last_phase;    // last phase whose tasks read the input row (F1 tasks)
  int32_t phase_ntasks[QFT_MAX_PHASES];
  int32_t phase_seg0[QFT_MAX_PHASES + 1];
  int32_t phase_is_slice[QFT_MAX_PHASES];   // 0 plain, 1 SLICE, 2 C/S tables
  QftSeg segs[QFT_MAX_SEGS];
};


// ---------------------------------------------------------------------------
// Rows too long for one CTA's shared memory (N > 2^14) are transformed by a
// sequence of launches over the whole batch, with the class data of every row
// in a scratch buffer in global memory (two copies, A and B):
//   GLOBAL  F1, further mirror levels (DIF) and the FINAL phase, run by the
//           same task functions as the row engine on the scratch rows;
//   NODE    every class tree is cut at the depth where a node holds at most
//           2^NB cells; a CTA loads a group of such nodes into shared memory,
//           finishes their forward phase and does their whole backward phase
//           (the row engine's phase loop on a sub-plan), and writes the node
//           outputs back (to A or B);
//   SLICE   the backward levels above the node depth, reading one scratch copy
//           and writing the other (no in-place hazard between CTAs).
#define QFT_LP_MAX_PHASES 16
// most backward levels one SLICE task of a compensated class does inside a
// NODE group (its pairs stay in registers across the SLICE round's barrier)
#ifndef QFT_COMP_NODE_LB
#define QFT_COMP_NODE_LB 3
#endif
#define QFT_LP_MAX_SEGS 160
#define QFT_LP_MAX_SUB 48

// TAB: the C_Mt / S_Mt tables of the FINAL tasks, one CTA per row
enum QftLargePhaseKind { QFT_LPH_GLOBAL = 0, QFT_LPH_SLICE = 1, QFT_LPH_NODE = 2, QFT_LPH_TAB = 3 };

struct QftLargePhase {
  int32_t kind;     // QftLargePhaseKind
  int32_t seg0;     // first segment (GLOBAL / SLICE phases)
  int32_t nseg;
  int32_t ntasks;   // tasks per row
};

// Node phase of one (side, class): nodes at depth D hold 2^nb cells; `group`
// consecutive nodes are transformed by one CTA.  Segment counts in `plan` are
// per group; a CTA for group g runs task indices g*count + [0, count).
struct QftNodeSub {
  int32_t side, cls, D, nb;
  int32_t nodes;      // nodes per row and side (2^D)
  int32_t group;      // nodes per CTA
  int32_t dst;        // 0: results to scratch A, 1: to scratch B
  int32_t cta_begin;  // first CTA (within one row) of this sub
  int32_t comp;       // 1: the class tree runs on compensated pairs (lo parts loaded and stored too)
  int32_t pad_;
  QftRowPlan plan;
};

// Segments of classes whose trees run on compensated pairs carry pad[2] = 1.
struct QftLargePlan {
  int32_t r, L1, LF, NB;
  int32_t comp_classes;           // J: classes 0..J-1 (both sides) run on compensated pairs
  int32_t nphase;
  QftLargePhase phases[QFT_LP_MAX_PHASES];
  int32_t nseg;
  QftSeg segs[QFT_LP_MAX_SEGS];   // pad[0] = source copy, pad[1] = destination copy (SLICE)
  int32_t nsub;
  int32_t node_ctas;              // CTAs per row in the node phase
  int32_t max_slice_nodes;        // largest per-node task count of a node sub-plan SLICE phase
  int32_t inplace;                // 1: one scratch copy; the SLICE levels run in place (QFT_IP_TASKS a block)
  int32_t pad_;
  QftNodeSub subs[QFT_LP_MAX_SUB];
};
// Tasks of one block of an in-place SLICE level (one CTA): a block reads all
// its cells before it writes any; blocks exchange only the neighbour cells at
// their edges, through a halo copy of QFT_IP_HALO cells per block edge.
#define QFT_IP_TASKS 256
#define QFT_IP_HALO 8
// block edges per row any in-place SLICE level of a row of 2^r can have (its
// tasks number at most N/2)
#define QFT_IP_EDGES(r) (((1 << (r)) / 2) / QFT_IP_TASKS + 2)
