// qft_large.cuh -- rows longer than one CTA's shared memory (N > 2^14).
//
// The class data of every row lives in two scratch copies (A, B) in global
// memory, laid out exactly like the row engine's shared-memory side arrays;
// in-place plans keep copy A only (their SLICE levels write over the cells
// they read, k_large_slice_ip).  One execute is a short sequence of launches
// over the whole batch (see the phase list of QftLargePlan in qft_plan.h);
// launch boundaries order the phases, so no CTA ever waits on another.
#pragma once
#include "qft_rows.cuh"

struct LargeArgs {
  const QftLargePlan* plan;   // device copy of the plan
  const float* gsec;          // Gray-ordered secants, N/4 + 1 entries
  qc* scrA;                   // scratch copy A: rows * 2 * side_len cells
  qc* scrB;                   // scratch copy B
  int64_t row0;               // first row (item) of this launch chunk
  int side_len;               // padded cells per side (even: rows and sides start 16-byte aligned)
  int r;
  int* status;                // device status word (QFT_ERR_TIMEOUT), or null
  qc* tab;                    // C_Mt / S_Mt tables of the FINAL tasks: rows * tab_stride cells, or null
  int tab_stride;             // cells per row of the tables
  int tabS_off;               // S_Mt starts tabS_off cells after C_Mt (Mt/2 + 1)
  uint64_t wait_ns;           // limit of the NODE kernel's wait for a staged window
  int withhold;               // test: each NODE CTA's first window copy is not issued (its wait runs out)
  qc* loA;                    // lo parts of the compensated cells of copy A (same layout), or null
  qc* loB;                    // lo parts of copy B
  // one-scratch (in-place) plans: class outputs in the in-place order, and the
  // halo copies of the SLICE levels' block edges (ip_edges * QFT_IP_HALO cells a row)
  int lay_nb;                 // node size log2 of the layout (0: natural order, two copies)
  int lay_l1;
  int ip_edges;
  qc* haloH;
  qc* haloL;                  // lo parts of the halo cells (compensated plans), or null
};


// The NODE and SLICE kernels do not depend on the IO of the transform; they
// are compiled once (qft_k_node.cu) and launched through these helpers, which
// return the CUDA error of the launch.
// comp != 0 selects the kernels that also run the compensated segments.
cudaError_t qft_large_node_prepare(int nt, size_t smem, int comp);
cudaError_t qft_large_node_launch(const LargeArgs& a, int64_t rows, int64_t items, int nt, size_t smem,
                                  cudaStream_t st, int comp);
cudaError_t qft_large_slice_launch(const LargeArgs& a, int phase, dim3 grid, cudaStream_t st, int comp);
// in-place SLICE phase of `nblk` blocks: the halo copy of its block edges, then the level
cudaError_t qft_large_slice_ip_launch(const LargeArgs& a, int phase, int nblk, int64_t rows, cudaStream_t st,
                                      int comp);
cudaError_t qft_large_tab_launch(const LargeArgs& a, int64_t rows, int LF, cudaStream_t st);

namespace {

constexpr int kLargeNT = 256;   // threads of the GLOBAL / SLICE kernels
constexpr int kLargeTPT = 4;    // tasks per thread per CTA in those kernels
// tasks per thread of the F1 launch (the first phase, which reads the input
// row), of the DIF launches and of the FINAL launch (the last phase)
#ifndef QFT_F1_TPT
#define QFT_F1_TPT 2
#endif
#ifndef QFT_DIF_TPT
#define QFT_DIF_TPT 8
#endif
#ifndef QFT_FIN_TPT
#define QFT_FIN_TPT kLargeTPT
#endif
// tasks per thread of the (two-copy) SLICE kernel
#ifndef QFT_SLICE_TPT
#define QFT_SLICE_TPT 8
#endif
// resident CTAs per SM the GLOBAL and SLICE kernels' register allocation targets
#ifndef QFT_GLOBAL_MINB
#define QFT_GLOBAL_MINB 2
#endif
#ifndef QFT_SLICE_MINB
#define QFT_SLICE_MINB 2
#endif
// 1: the GLOBAL (DIF tasks) and SLICE kernels prefetch each thread's next task into L2
#ifndef QFT_LARGE_PF
#define QFT_LARGE_PF 1
#endif
#ifndef QFT_SLICE_PF
#define QFT_SLICE_PF QFT_LARGE_PF
#endif

__device__ __forceinline__ Eng large_eng(const LargeArgs& a, int copy, int64_t row) {
  Eng e;
  qc* base = (copy ? a.scrB : a.scrA) + row * 2 * (int64_t)a.side_len;
  e.side0 = base;
  e.side1 = base + a.side_len;
  e.sec = a.gsec;
  e.r = a.r;
  e.N = 1 << a.r;
  e.tabC = a.tab ? a.tab + row * (int64_t)a.tab_stride : nullptr;
  e.tabS = a.tab ? e.tabC + a.tabS_off : nullptr;
  qc* lb = copy ? a.loB : a.loA;
  e.lo0 = lb ? lb + row * 2 * (int64_t)a.side_len : nullptr;
  e.lo1 = lb ? e.lo0 + a.side_len : nullptr;
  e.lay_nb = a.lay_nb;
  e.lay_l1 = a.lay_l1;
  return e;
}

// GLOBAL phase (F1, DIF, FINAL): blockIdx.y = row within the chunk, blockIdx.x
// = block of kLargeNT * tpt consecutive tasks of that row's phase.
template <class FAC, int L1, bool COMP>
__global__ void __launch_bounds__(kLargeNT, QFT_GLOBAL_MINB) k_large_global(LargeArgs a, int phase, FAC fac,
                                                                            int tpt) {
  const QftLargePlan* P = a.plan;
  const QftLargePhase ph = P->phases[phase];
  const int64_t row = blockIdx.y;
  const Eng e = large_eng(a, 0, row);
  const auto io = fac.make(a.row0 + row);
  // this thread's tasks: T0 + k * kLargeNT, k < tpt, T0 = block start + tid
  const int T0 = blockIdx.x * (kLargeNT * tpt) + (int)threadIdx.x;
  const int T1 = blockIdx.x * (kLargeNT * tpt) + kLargeNT * tpt;
  for (int s = ph.seg0; s < ph.seg0 + ph.nseg; ++s) {
    const QftSeg sg = P->segs[s];
    if (sg.begin >= T1 || sg.begin + sg.count <= T0 - (int)threadIdx.x) continue;
    int first = T0 - sg.begin;
    if (first < 0) first += ((-first + kLargeNT - 1) / kLargeNT) * kLargeNT;
    int end = T1 - sg.begin;
    if (end > sg.count) end = sg.count;
    run_plain_segment<L1, decltype(io), COMP, QFT_LARGE_PF>(P->LF, sg, e, io, first, end, kLargeNT, 0);
  }
}

// cells of one NODE buffer: the largest group window, rounded up to an even
// count so that a bulk copy of it is a multiple of 16 bytes
__host__ __device__ inline int node_buf_cells(int NB) { return (qft_pidx(1 << NB) + 2) & ~1; }
// plan | secants | two cell buffers (the current item and the prefetched next
// one) | with compensation, two more buffers for their lo parts
__host__ __device__ inline size_t node_smem_bytes(int NB, int comp = 0) {
  return qft_lib::align16(sizeof(QftRowPlan)) + qft_lib::align16(sizeof(float) * (((size_t)1 << NB) + 1)) +
         (comp ? 4 : 2) * qft_lib::align16(8 * (size_t)node_buf_cells(NB));
}

#ifdef QFT_NODE_TU
// SLICE phase above the node depth: reads copy sg.pad[0], writes copy sg.pad[1].
// Output store of one warp of SLICE tasks whose 2^L-cell outputs are one
// contiguous run (lane i at base0 + i 2^L): through a per-warp buffer
// (hb/lb: 32 (2^L + 1) cells each), so that store j writes cells
// base0 + 32 j + lane, 32 consecutive cells per store instead of one cell of
// each of 32 lanes 2^L cells apart.  The cells and values are those of
// task_slice_write(_c) (the rounded h + l for a class output, `root`).
template <int L, bool C>
__device__ __forceinline__ void slice_write_warp(const QftSeg& sg, const Eng& ed, const SliceRegs& p, const qc* wl,
                                                 bool root, qc* hb, qc* lb, int lane, int base0) {
  constexpr int W = (1 << L) + 1;
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    hb[lane * W + t] = (C && root) ? cadd(p.w[t], wl[t]) : p.w[t];
    if (C && !root) lb[lane * W + t] = wl[t];
  }
  __syncwarp();
  qc* A = side_ptr(ed, sg.side);
  qc* Al = lo_ptr(ed, sg.side);
#pragma unroll
  for (int j = 0; j < (1 << L); ++j) {
    const int idx = j * 32 + lane;
    const int o = (idx >> L) * W + (idx & ((1 << L) - 1));
    const int pi = qft_pidx(base0 + idx);
    A[pi] = hb[o];
    if (C && !root) Al[pi] = lb[o];
  }
  __syncwarp();   // the buffer is reused by the next round
}

template <bool COMP>
__global__ void __launch_bounds__(kLargeNT, QFT_SLICE_MINB) k_large_slice(LargeArgs a, int phase) {
  constexpr int kW = 9 * 32;                     // cells of a warp's buffer (L <= 3)
  __shared__ qc s_hb[kLargeNT / 32][kW];
  __shared__ qc s_lb[COMP ? kLargeNT / 32 : 1][COMP ? kW : 1];
  const QftLargePlan* P = a.plan;
  const QftLargePhase ph = P->phases[phase];
  const int64_t row = blockIdx.y;
  const int t0 = blockIdx.x * (kLargeNT * QFT_SLICE_TPT);
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  int sgi = ph.seg0;
  const int sge = ph.seg0 + ph.nseg;
  for (int k = 0; k < QFT_SLICE_TPT; ++k) {
    const int tau = t0 + k * kLargeNT + (int)threadIdx.x;
    if (t0 + k * kLargeNT >= ph.ntasks) break;   // uniform over the CTA
    const bool active = tau < ph.ntasks;
    if (active)
      while (sgi + 1 < sge && P->segs[sgi + 1].begin <= tau) ++sgi;
    const QftSeg sg = P->segs[sgi];
    const bool comp = COMP && sg.pad[2];
    SliceRegsC s;
    if (active) {
      const Eng es = large_eng(a, sg.pad[0], row);
      // the cells of this thread's next task go to L2 while this one is read
      const int taun = tau + kLargeNT;
      if (QFT_SLICE_PF && k + 1 < QFT_SLICE_TPT && taun < ph.ntasks && taun < sg.begin + sg.count)
        run_slice_prefetch(sg, es, taun - sg.begin, comp);
      if (comp) run_slice_read_c(sg, es, tau - sg.begin, s);
      else run_slice_read(sg, es, tau - sg.begin, s.p);
    }
    // the warp's outputs form one contiguous run: store them coalesced
    const int base0 = __shfl_sync(0xffffffffu, s.p.base, 0);
    const int sg0 = __shfl_sync(0xffffffffu, sgi, 0);
    const bool run = __all_sync(0xffffffffu, active && sgi == sg0 && s.p.base == base0 + (lane << sg.L));
    const Eng ed = large_eng(a, sg.pad[1], row);
    if (run) {
      const bool root = comp && sg.D == sg.L;
      qc* hb = s_hb[wq];
      qc* lb = COMP ? &s_lb[wq][0] : hb;
#define QFT_SWW(LL)                                                                        \
  if (comp) slice_write_warp<LL, COMP>(sg, ed, s.p, s.wl, root, hb, lb, lane, base0);     \
  else slice_write_warp<LL, false>(sg, ed, s.p, s.wl, false, hb, lb, lane, base0);
      switch (sg.L) {
      case 1: QFT_SWW(1) break;
      case 2: QFT_SWW(2) break;
      case 3: QFT_SWW(3) break;
      default: break;
      }
#undef QFT_SWW
    } else if (active) {
      if (comp) run_slice_write_c(sg, ed, s);
      else run_slice_write(sg, ed, s.p);
    }
  }
}


// In-place SLICE phase (one-scratch plans), blockIdx.y = row.
// k_large_halo: thread k copies the neighbour cells that cross block edge k
// (1 <= k < nblk) into the row's halo copy, before any block of the level runs.
template <bool COMP>
__global__ void __launch_bounds__(256) k_large_halo(LargeArgs a, int phase, int nblk) {
  const QftLargePlan* P = a.plan;
  const QftLargePhase ph = P->phases[phase];
  const int k = 1 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (k >= nblk) return;
  const int64_t row = blockIdx.y;
  const Eng e = large_eng(a, 0, row);
  const int64_t off = (row * a.ip_edges + k) * QFT_IP_HALO;
  slice_ip_edge(P->segs, ph.seg0, ph.nseg, e, k, a.haloH + off, COMP ? a.haloL + off : nullptr);
}

// k_large_slice_ip: block blockIdx.x = tasks [QFT_IP_TASKS bx, + QFT_IP_TASKS)
// of the phase.  Every thread reads its task's cells and runs its levels,
// the CTA barrier orders all reads of the block before its writes, and each
// task writes over the cells it read.  Within the block, thread i takes task
// x = transpose of i over (2^dp x QFT_IP_TASKS/2^dp), dp the levels already
// in place below the first task's segment: a warp's lanes then take chunks
// 2^dp apart, whose cells are adjacent.
template <bool COMP>
__global__ void __launch_bounds__(QFT_IP_TASKS, 2) k_large_slice_ip(LargeArgs a, int phase) {
  const QftLargePlan* P = a.plan;
  const QftLargePhase ph = P->phases[phase];
  const int64_t row = blockIdx.y;
  const Eng e = large_eng(a, 0, row);
  const int t0 = blockIdx.x * QFT_IP_TASKS;
  const int sge = ph.seg0 + ph.nseg;
  int sgi = ph.seg0;
  while (sgi + 1 < sge && P->segs[sgi + 1].begin <= t0) ++sgi;
  int dp = cls_lay_depth(e, P->segs[sgi].cls) - P->segs[sgi].D;
  dp = dp < 0 ? 0 : (dp > 8 ? 8 : dp);
  const int cols = QFT_IP_TASKS >> dp;
  const int x = (((int)threadIdx.x % cols) << dp) | ((int)threadIdx.x / cols);
  const int tau = t0 + x;
  const bool active = tau < ph.ntasks;
  SliceIp s;
  if (active) {
    while (sgi + 1 < sge && P->segs[sgi + 1].begin <= tau) ++sgi;
    const QftSeg& sg = P->segs[sgi];
    const int slot = slice_ip_halo_slot(sg.side, x, blockIdx.x);
    const int64_t hoff = row * a.ip_edges * QFT_IP_HALO + slot;
    run_slice_ip_read(sg, e, tau - sg.begin, slot >= 0 ? a.haloH + hoff : nullptr,
                      (COMP && slot >= 0) ? a.haloL + hoff : nullptr, COMP && sg.pad[2], s);
  }
  __syncthreads();
  if (active) run_slice_ip_write(P->segs[sgi], e, COMP && P->segs[sgi].pad[2], s);
}

// NODE phase: blockIdx.x = node group (over all subs), blockIdx.y = row.  The
// group's cells [base, base + group * 2^nb) of one side (copy A) are loaded
// into shared memory, the sub-plan runs on them, and they are written to copy
// `dst`.  base is a multiple of 16, so the padded layout of the window is the
// padded layout of the scratch row shifted by qft_pidx(base).
// Window of item `it` (= node CTA index * rows + row): sub k (advanced from
// its previous value; the node CTA index never decreases along a CTA's items),
// group g, the padded cell offset pb and count pn, and the source row.
struct NodeItem {
  int k, g, pb, pn;
  int64_t row;
};
__device__ __forceinline__ void node_item(const QftLargePlan* LP, int r, int64_t it, int64_t rows, int& k,
                                          NodeItem& w) {
  const int cta = (int)(it / rows);
  w.row = it - (int64_t)cta * rows;
  while (k + 1 < LP->nsub && LP->subs[k + 1].cta_begin <= cta) ++k;
  const QftNodeSub& S = LP->subs[k];
  w.k = k;
  w.g = cta - S.cta_begin;
  const int ncell = S.group << S.nb;
  const int base = cls_off(r, S.cls) + w.g * ncell;
  w.pb = qft_pidx(base);
  w.pn = qft_pidx(ncell - 1) + 1;
}

template <int L1, int NT, bool COMP>
__global__ void __launch_bounds__(NT, 512 / NT) k_large_node(LargeArgs a, int64_t rows) {
  // Persistent: item = node CTA index * rows + row, visited in steps of the
  // grid, so one CTA's items keep the same sub (and sub-plan) for long runs;
  // the secants are loaded once per CTA and the sub-plan only when the sub
  // changes.  While an item is transformed, thread 0 copies the next item's
  // cells into the other buffer with one bulk copy (completion on an mbarrier,
  // waits bounded); windows that are not 16-byte aligned are loaded directly.
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_staged[2];
  const QftLargePlan* LP = a.plan;
  QftRowPlan& Q = *reinterpret_cast<QftRowPlan*>(smem);
  const int NB = LP->NB;
  float* sec = reinterpret_cast<float*>(smem + qft_lib::align16(sizeof(QftRowPlan)));
  qc* buf[2];
  buf[0] = reinterpret_cast<qc*>(smem + qft_lib::align16(sizeof(QftRowPlan)) +
                                 qft_lib::align16(sizeof(float) * ((1 << NB) + 1)));
  buf[1] = buf[0] + qft_lib::align16(8 * (size_t)node_buf_cells(NB)) / 8;
  qc* lbuf[2];   // lo parts of the compensated subs' cells (COMP kernels only)
  lbuf[0] = buf[1] + qft_lib::align16(8 * (size_t)node_buf_cells(NB)) / 8;
  lbuf[1] = lbuf[0] + qft_lib::align16(8 * (size_t)node_buf_cells(NB)) / 8;
  const int64_t items = (int64_t)LP->node_ctas * rows;
  const auto src_of = [&](const NodeItem& w) {
    return side_ptr(large_eng(a, 0, w.row), LP->subs[w.k].side) + w.pb;
  };
  const auto lsrc_of = [&](const NodeItem& w) {
    return lo_ptr(large_eng(a, 0, w.row), LP->subs[w.k].side) + w.pb;
  };
  // thread 0: bulk copy of item w's window (and, for a compensated sub, of its
  // lo parts) into buffer b, if everything is 16-byte aligned
  const auto issue = [&](const NodeItem& w, int b) {
    const qc* src = src_of(w);
    const bool comp = COMP && LP->subs[w.k].comp;
    const uint32_t bytes = (uint32_t)(((w.pn + 1) & ~1) * 8);
    const bool ok = ((uintptr_t)src & 15) == 0 && (bytes & 15) == 0 && (smem_u32(buf[b]) & 15) == 0 &&
                    (!comp || (((uintptr_t)lsrc_of(w) & 15) == 0 && (smem_u32(lbuf[b]) & 15) == 0));
    s_staged[b] = ok ? 1 : 0;
    if (ok) {
      fence_proxy_async_smem();
      mbar_expect_tx(smem_u32(&mbar[b]), comp ? 2 * bytes : bytes);
      bulk_g2s(smem_u32(buf[b]), src, bytes, smem_u32(&mbar[b]));
      if (comp) bulk_g2s(smem_u32(lbuf[b]), lsrc_of(w), bytes, smem_u32(&mbar[b]));
    }
  };
  for (int m = threadIdx.x; m <= (1 << NB); m += NT) sec[m] = a.gsec[m];
  int kc = 0, kn = 0;   // sub positions of the current and of the prefetched item
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    fence_mbar_init();
  }
  __syncthreads();
  // a withheld copy is never issued: nothing is in flight when its wait runs out
  bool withheld = a.withhold != 0;
  if (threadIdx.x == 0 && (int64_t)blockIdx.x < items) {
    NodeItem w;
    node_item(LP, a.r, blockIdx.x, rows, kn, w);
    if (withheld) s_staged[0] = 1;
    else issue(w, 0);
  }
  __syncthreads();
  uint32_t parity[2] = {0, 0};
  int cur = -1;
  int b = 0;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x, b ^= 1) {
    NodeItem w;
    node_item(LP, a.r, it, rows, kc, w);
    const QftNodeSub& S = LP->subs[w.k];
    qc* cells = buf[b];
    if (s_staged[b]) {
      const uint64_t t0 = global_ns();
      bool ok = true;
      while (!mbar_try_wait(smem_u32(&mbar[b]), parity[b])) {
        if (global_ns() - t0 > a.wait_ns) { ok = false; break; }
      }
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          if (a.status) atomicExch(a.status, QFT_ERR_TIMEOUT);
          // the copy in flight writes this CTA's shared memory: a second bounded wait (long limit)
          const uint64_t t1 = global_ns();
          while (!withheld && !mbar_try_wait(smem_u32(&mbar[b]), parity[b]) && global_ns() - t1 < kWaitLimitNs) {
          }
        }
        __syncthreads();
        return;
      }
      parity[b] ^= 1;
    } else {
      const qc* srcp = src_of(w);
      for (int i = threadIdx.x; i < w.pn; i += NT) cells[i] = srcp[i];
      if (COMP && S.comp) {
        const qc* lsrc = lsrc_of(w);
        for (int i = threadIdx.x; i < w.pn; i += NT) lbuf[b][i] = lsrc[i];
      }
    }
    withheld = false;
    // the next item's copy goes to the other buffer, free since the last barrier
    const int64_t next = it + gridDim.x;
    if (threadIdx.x == 0 && next < items) {
      NodeItem wn;
      node_item(LP, a.r, next, rows, kn, wn);
      issue(wn, b ^ 1);
    }
    if (w.k != cur) {
      const int* src = reinterpret_cast<const int*>(&S.plan);
      int* dst = reinterpret_cast<int*>(smem);
      for (int i = threadIdx.x; i < (int)(sizeof(QftRowPlan) / 4); i += NT) dst[i] = src[i];
      cur = w.k;
    }
    __syncthreads();
    Eng e;
    e.side0 = cells - w.pb;   // the window maps class-level index base -> cells[0]
    e.side1 = cells - w.pb;
    e.sec = sec;
    e.r = a.r;
    e.N = 1 << a.r;
    e.tabC = nullptr;
    e.tabS = nullptr;
    e.lo0 = lbuf[b] - w.pb;
    e.lo1 = lbuf[b] - w.pb;
    run_row_phases<L1, NT, NoIO, NoHook, COMP>(Q, e, NoIO(), w.g);
    const Eng ed = large_eng(a, S.dst, w.row);
    qc* dstp = side_ptr(ed, S.side) + w.pb;
    for (int i = threadIdx.x; i < w.pn; i += NT) dstp[i] = cells[i];
    if (COMP && S.comp) {
      qc* ldst = lo_ptr(ed, S.side) + w.pb;
      for (int i = threadIdx.x; i < w.pn; i += NT) ldst[i] = lbuf[b][i];
    }
    __syncthreads();   // this buffer (and maybe the sub-plan) is reused two items on
  }
}
// TAB phase: the C_Mt / S_Mt tables of one row (one CTA), level by level from
// the dct(2) / dst(4) base cases with the class outputs in copy A (eqs qft_5C,
// qft_5D, qft_6 and their DST forms), as the row engine builds them in shared
// memory; a CTA barrier separates the levels.
// NT threads a CTA (one row): the launch takes more threads a row when the
// chunk has fewer rows (qft_large_tab_launch).
template <int NT>
__global__ void __launch_bounds__(NT) k_large_tab(LargeArgs a, int LF) {
  const Eng e = large_eng(a, 0, blockIdx.x);
  const int mt = a.r - LF;
  for (int m = 1; m <= mt; ++m) {
    tab_level_c(e, m, threadIdx.x, NT);
    if (m >= 2) tab_level_s(e, m, threadIdx.x, NT);
    __syncthreads();
  }
}
#endif  // QFT_NODE_TU

// One execute on the large-row path: every phase of the plan, in order, for
// `items` rows (or real row pairs) starting at row0, in chunks that fit the
// plan's scratch.
template <class FAC>
static inline int launch_large(qft_plan p, FAC fac, int64_t items, cudaStream_t st) {
  const QftLargePlan& H = *p->large_host;
  const int comp = H.comp_classes > 0 ? 1 : 0;
  LargeArgs a;
  a.plan = p->d_large;
  a.gsec = p->d_sec;
  // scratch: copy A | copy B | C/S tables | (compensated plans) lo parts of A | of B;
  // in-place plans: copy A | C/S tables | (lo parts of A) | halos | (their lo parts)
  const int ip = H.inplace;
  const size_t copy_cells = (size_t)p->scratch_rows * 2 * p->side_len;
  a.scrA = reinterpret_cast<qc*>(p->scratch);
  a.scrB = ip ? a.scrA : a.scrA + copy_cells;
  a.side_len = p->side_len;
  a.r = p->r;
  a.status = p->d_status;
  a.wait_ns = p->wait_ns > 0 ? (uint64_t)p->wait_ns : kWaitLimitNs;
  a.withhold = p->withhold_copy;
  a.tab_stride = qft_lib::large_tab_cells(1 << p->r, H.LF);
  a.tabS_off = ((1 << p->r) >> H.LF) / 2 + 1;
  // tables after the two copies; a CTA builds one row's tables, which pays off
  // only with enough rows of moderate length (the plan's large_tab)
  qc* tab0 = (ip ? a.scrA : a.scrB) + copy_cells;
  a.tab = p->large_tab ? tab0 : nullptr;
  qc* lo0 = tab0 + (size_t)p->scratch_rows * qft_lib::large_tab_cells(1 << p->r, qft_lib::kLargeMinLF);
  a.loA = comp ? lo0 : nullptr;
  a.loB = comp ? (ip ? lo0 : lo0 + copy_cells) : nullptr;
  a.lay_nb = ip ? H.NB : 0;
  a.lay_l1 = ip ? H.L1 : 0;
  a.ip_edges = QFT_IP_EDGES(p->r);
  qc* halo0 = lo0 + (comp ? copy_cells : 0);
  a.haloH = ip ? halo0 : nullptr;
  a.haloL = ip && comp ? halo0 + (size_t)p->scratch_rows * a.ip_edges * QFT_IP_HALO : nullptr;
  const size_t node_smem = node_smem_bytes(H.NB, comp);
  // node kernel: 512 threads (one CTA per SM) unless the plan asks for 256
  const int node_nt = p->node_nt == 256 ? 256 : 512;
  cudaError_t e = qft_large_node_prepare(node_nt, node_smem, comp);
  if (e != cudaSuccess) return qft_set_cuda(p, e);
  const int64_t chunk = p->chunk_rows > 0 && p->chunk_rows < p->scratch_rows ? p->chunk_rows : p->scratch_rows;
  for (int64_t r0 = 0; r0 < items; r0 += chunk) {
    const int64_t rows = items - r0 < chunk ? items - r0 : chunk;
    a.row0 = r0;
    for (int ph = 0; ph < H.nphase; ++ph) {
      const QftLargePhase& P = H.phases[ph];
      if (P.kind == QFT_LPH_TAB) {
        if (!a.tab) continue;
        qft_time_begin(p, st, QFT_KERNEL_GLOBAL);
        e = qft_large_tab_launch(a, rows, H.LF, st);
        if (e != cudaSuccess) return qft_set_cuda(p, e);
      } else if (P.kind == QFT_LPH_NODE) {
        qft_time_begin(p, st, QFT_KERNEL_NODE);
        e = qft_large_node_launch(a, rows, (int64_t)H.node_ctas * rows, node_nt, node_smem, st, comp);
        if (e != cudaSuccess) return qft_set_cuda(p, e);
      } else {
        const unsigned bx = (unsigned)((P.ntasks + kLargeNT * QFT_SLICE_TPT - 1) / (kLargeNT * QFT_SLICE_TPT));
        if (P.kind == QFT_LPH_SLICE) {
          qft_time_begin(p, st, QFT_KERNEL_SLICE);
          e = ip ? qft_large_slice_ip_launch(a, ph, (P.ntasks + QFT_IP_TASKS - 1) / QFT_IP_TASKS, rows, st, comp)
                 : qft_large_slice_launch(a, ph, dim3(bx, (unsigned)rows), st, comp);
          if (e != cudaSuccess) return qft_set_cuda(p, e);
        } else {
          qft_time_begin(p, st, QFT_KERNEL_GLOBAL);
          const int tpt = ph == 0 ? QFT_F1_TPT : (ph == H.nphase - 1 ? QFT_FIN_TPT : QFT_DIF_TPT);
          const unsigned gx = (unsigned)((P.ntasks + kLargeNT * tpt - 1) / (kLargeNT * tpt));
          if (comp) k_large_global<FAC, qft_lib::kL1, true><<<dim3(gx, (unsigned)rows), kLargeNT, 0, st>>>(a, ph, fac, tpt);
          else k_large_global<FAC, qft_lib::kL1, false><<<dim3(gx, (unsigned)rows), kLargeNT, 0, st>>>(a, ph, fac, tpt);
        }
      }
      qft_time_end(p, st);
      e = cudaGetLastError();
      if (e != cudaSuccess) return qft_set_cuda(p, e);
    }
  }
  return QFT_OK;
}

template <class FAC>
static inline int launch_any(qft_plan p, FAC fac, int64_t items, cudaStream_t st, size_t stage_bytes = 0,
                             bool stage_ok = false) {
  if (p->large_host) return launch_large<FAC>(p, fac, items, st);
  return launch_rows<FAC>(p, fac, items, st, stage_bytes, stage_ok);
}

}  // namespace

template <class ST>
static inline int exec_c2c(qft_plan p, int op, const void* in, void* out, cudaStream_t st) {
  FacC2C<ST> f;
  f.in = static_cast<const typename ST::elem*>(in);
  f.out = static_cast<typename ST::elem*>(out);
  f.N = (int)p->n;
  f.scale = 1.f; f.scaled = 0;
  switch (op) {
  case QFT_OP_FORWARD: f.in_op = QFT_LANE_ID; f.out_op = QFT_LANE_ID; break;
  case QFT_OP_INVERSE: f.in_op = QFT_LANE_SWAP; f.out_op = QFT_LANE_SWAP; f.scale = 1.f / (float)p->n; f.scaled = 1; break;
  case QFT_OP_FORWARD_ADJOINT: f.in_op = QFT_LANE_CONJ; f.out_op = QFT_LANE_CONJ; break;
  case QFT_OP_INVERSE_ADJOINT: f.in_op = QFT_LANE_ID; f.out_op = QFT_LANE_ID; f.scale = 1.f / (float)p->n; f.scaled = 1; break;
  default: return QFT_ERR_INVALID_ARG;
  }
  if (p->r == 1) {
    const int64_t blocks = (p->batch + 127) / 128;
    k_c2c_n2<ST><<<(unsigned)blocks, 128, 0, st>>>(f, p->batch);
    return qft_set_cuda(p, cudaGetLastError());
  }
  return launch_any<FacC2C<ST>>(p, f, p->batch, st, (size_t)p->n * sizeof(typename ST::elem),
                                ((uintptr_t)in % 16) == 0);
}

