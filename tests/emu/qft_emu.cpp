// Host emulation of the row engine (test infrastructure only).
//
// Compiles the library's engine header (qft_engine.cuh / qft_io.cuh) and its
// planner for the host with QFT_HOST_EMULATION, and runs the phases of one CTA
// the way the kernel does: every phase loops over its tasks, SLICE phases run
// in rounds (all reads of a round, then all writes).  The test-suite compares
// its output bit for bit with the improved-QFT oracle built in FP32, which
// checks the engine's index logic without a GPU.  The product never loads this.
#define QFT_HOST_EMULATION 1
#define QFT_MAX_LB 4
#include "../../paper_1301_0763_gb300/csrc/qft_io.cuh"
#include "../../paper_1301_0763_gb300/csrc/qft_planner.h"
#include "../../paper_1301_0763_gb300/csrc/qft_consts.h"
#include <vector>
#include <stdint.h>

using namespace qft;

template <class IO, bool COMP = false>
static void run_row(const QftRowPlan& P, const Eng& e, const IO& io, int nthr, int g = 0) {
  for (int p = 0; p < P.nphase; ++p) {
    const int nt = P.phase_ntasks[p];
    if (P.phase_is_slice[p] == 2) {
      const int mt = P.r - P.LF;
      for (int m = 1; m <= mt; ++m) for (int lane = 0; lane < 32; ++lane) tab_level_c(e, m, lane, 32);
      for (int m = 2; m <= mt; ++m) for (int lane = 0; lane < 32; ++lane) tab_level_s(e, m, lane, 32);
      for (int tau = 0; tau < nt; ++tau) {
        const QftSeg& sg = find_seg(P, p, tau);
        switch (P.L1) {
        case 0: run_plain_task<0, IO, COMP>(P.LF, sg, e, io, g * sg.count + tau - sg.begin); break;
        case 1: run_plain_task<1, IO, COMP>(P.LF, sg, e, io, g * sg.count + tau - sg.begin); break;
        case 2: run_plain_task<2, IO, COMP>(P.LF, sg, e, io, g * sg.count + tau - sg.begin); break;
        case 3: run_plain_task<3, IO, COMP>(P.LF, sg, e, io, g * sg.count + tau - sg.begin); break;
        default: run_plain_task<4, IO, COMP>(P.LF, sg, e, io, g * sg.count + tau - sg.begin); break;
        }
      }
      continue;
    }
    if (!P.phase_is_slice[p]) {
      for (int tid = 0; tid < nthr; ++tid)
        for (int s = P.phase_seg0[p]; s < P.phase_seg0[p + 1]; ++s) {
          const QftSeg& sg = P.segs[s];
          int first = (tid - sg.begin) % nthr;
          if (first < 0) first += nthr;
          switch (P.L1) {
          case 0: run_plain_segment<0, IO, COMP>(P.LF, sg, e, io, first, sg.count, nthr, g); break;
          case 1: run_plain_segment<1, IO, COMP>(P.LF, sg, e, io, first, sg.count, nthr, g); break;
          case 2: run_plain_segment<2, IO, COMP>(P.LF, sg, e, io, first, sg.count, nthr, g); break;
          case 3: run_plain_segment<3, IO, COMP>(P.LF, sg, e, io, first, sg.count, nthr, g); break;
          default: run_plain_segment<4, IO, COMP>(P.LF, sg, e, io, first, sg.count, nthr, g); break;
          }
        }
    } else {
      std::vector<SliceRegsC> regs(nthr);
      std::vector<int> segi(nthr);
      for (int rb = 0; rb < nt; rb += nthr) {
        for (int tid = 0; tid < nthr; ++tid) {
          const int tau = rb + tid;
          segi[tid] = -1;
          if (tau < nt) {
            const QftSeg& sg = find_seg(P, p, tau);
            segi[tid] = (int)(&sg - P.segs);
            if (COMP && sg.pad[2]) run_slice_read_c<QFT_COMP_NODE_LB>(sg, e, g * sg.count + tau - sg.begin, regs[tid]);
            else run_slice_read(sg, e, g * sg.count + tau - sg.begin, regs[tid].p);
          }
        }
        for (int tid = 0; tid < nthr; ++tid)
          if (segi[tid] >= 0) {
            const QftSeg& sg = P.segs[segi[tid]];
            if (COMP && sg.pad[2]) run_slice_write_c<QFT_COMP_NODE_LB>(sg, e, regs[tid]);
            else run_slice_write(sg, e, regs[tid].p);
          }
      }
    }
  }
}

struct Row {
  std::vector<qc> s0, s1, tab;
  std::vector<float> sec;
  QftRowPlan P;
  Eng e;
  int ok;
  Row(int N, const int* tune, int& nthr) {
    int r = 0; while ((1 << r) < N) ++r;
    if (nthr <= 0) nthr = qft_default_threads(r);
    QftTune t = qft_default_tune(r);
    if (tune) { t.L1 = tune[0]; t.LS = tune[1]; t.LL = tune[2]; t.LB = tune[3]; t.LF = tune[4]; }
    ok = qft_build_row_plan(r, t, &P, nthr) == 0 && P.max_slice_nodes <= nthr;
    s0.assign(qft_side_len(N), mkc(NAN, NAN));
    s1.assign(qft_side_len(N), mkc(NAN, NAN));
    sec.assign(N / 4 + 1, 0.f);
    qft_fill_gray_secants(r, sec.data());
    e.side0 = s0.data(); e.side1 = s1.data(); e.sec = sec.data(); e.r = r; e.N = N;
    tab.assign((N >> P.LF) + 2, mkc(NAN, NAN));
    e.tabC = tab.data();
    e.tabS = tab.data() + (N >> P.LF) / 2 + 1;
    e.lo0 = nullptr; e.lo1 = nullptr;
  }
};

extern "C" int emu_plan_info(int N, const int* tune, int* nphase, int* nseg, int* max_slice) {
  int big = 1 << 20;
  Row R(N, tune, big);
  *nphase = R.P.nphase; *nseg = R.P.nseg; *max_slice = R.P.max_slice_nodes;
  return R.ok ? 0 : -1;
}

// op: 0 forward, 1 inverse, 2 forward adjoint, 3 inverse adjoint; data complex64 interleaved
extern "C" int emu_c2c(int N, int64_t batch, const float* in, float* out, int op, const int* tune, int nthr) {
  if (N < 4) return -1;
  Row R(N, tune, nthr);
  if (!R.ok) return -2;
  for (int64_t b = 0; b < batch; ++b) {
    IoC2C<StC64> io;
    io.in = reinterpret_cast<const qc*>(in) + b * N;
    io.out = reinterpret_cast<qc*>(out) + b * N;
    io.N = N; io.scale = 1.f; io.scaled = false;
    io.in_op = io.out_op = QFT_LANE_ID;
    if (op == 1) { io.in_op = io.out_op = QFT_LANE_SWAP; io.scale = 1.f / N; io.scaled = true; }
    if (op == 2) { io.in_op = io.out_op = QFT_LANE_CONJ; }
    if (op == 3) { io.scale = 1.f / N; io.scaled = true; }
    run_row(R.P, R.e, io, nthr);
  }
  return 0;
}

// DCT-0 (dst = 0, rows of N/2+1) or DST-0 (dst = 1, rows of N/2-1) of
// periodization N, two rows per pass as on the device.
extern "C" int emu_r2r(int N, int64_t batch, const float* in, float* out, int dst, int nthr) {
  Row R(N, nullptr, nthr);
  if (!R.ok) return -2;
  const int64_t L = dst ? N / 2 - 1 : N / 2 + 1;
  for (int64_t it = 0; it < (batch + 1) / 2; ++it) {
    const int64_t a = 2 * it, b = 2 * it + 1;
    if (dst) {
      IoR2R<true> io;
      io.ina = in + a * L; io.inb = b < batch ? in + b * L : nullptr;
      io.outa = out + a * L; io.outb = b < batch ? out + b * L : nullptr; io.N = N;
      run_row(R.P, R.e, io, nthr);
    } else {
      IoR2R<false> io;
      io.ina = in + a * L; io.inb = b < batch ? in + b * L : nullptr;
      io.outa = out + a * L; io.outb = b < batch ? out + b * L : nullptr; io.N = N;
      run_row(R.P, R.e, io, nthr);
    }
  }
  return 0;
}

// dtype 1: fp16 pairs, 2: bf16 pairs (uint16 pairs in memory)
extern "C" int emu_c2c_half(int N, int64_t batch, const uint16_t* in, uint16_t* out, int dtype, int op, int nthr) {
  Row R(N, nullptr, nthr);
  if (!R.ok) return -2;
  for (int64_t b = 0; b < batch; ++b) {
    if (dtype == 1) {
      IoC2C<StC16> io;
      io.in = reinterpret_cast<const h2pair*>(in) + b * N; io.out = reinterpret_cast<h2pair*>(out) + b * N;
      io.N = N; io.scale = 1.f; io.scaled = false; io.in_op = io.out_op = QFT_LANE_ID;
      if (op == 1) { io.in_op = io.out_op = QFT_LANE_SWAP; io.scale = 1.f / N; io.scaled = true; }
      run_row(R.P, R.e, io, nthr);
    } else {
      IoC2C<StBF16> io;
      io.in = reinterpret_cast<const h2pair*>(in) + b * N; io.out = reinterpret_cast<h2pair*>(out) + b * N;
      io.N = N; io.scale = 1.f; io.scaled = false; io.in_op = io.out_op = QFT_LANE_ID;
      if (op == 1) { io.in_op = io.out_op = QFT_LANE_SWAP; io.scale = 1.f / N; io.scaled = true; }
      run_row(R.P, R.e, io, nthr);
    }
  }
  return 0;
}

// R2C family: op 0 forward (real->half spectrum), 1 inverse (half->real),
// 2 forward adjoint (half->real, w=1), 3 inverse adjoint (real->half, weights w/N)
extern "C" int emu_r2c(int N, int64_t batch, const float* in, float* out, int op, int nthr) {
  Row R(N, nullptr, nthr);
  if (!R.ok) return -2;
  const int64_t H = N / 2 + 1;
  for (int64_t it = 0; it < (batch + 1) / 2; ++it) {
    const int64_t a = 2 * it, b = 2 * it + 1;
    if (op == 0 || op == 3) {
      IoR2C<StC64> io;
      io.ina = in + a * N; io.inb = b < batch ? in + b * N : nullptr;
      io.outa = reinterpret_cast<qc*>(out) + a * H; io.outb = b < batch ? reinterpret_cast<qc*>(out) + b * H : nullptr;
      io.N = N; io.wscale = op == 0 ? 0.f : 1.f / N;
      run_row(R.P, R.e, io, nthr);
    } else {
      IoC2R<StC64> io;
      io.ina = reinterpret_cast<const qc*>(in) + a * H; io.inb = b < batch ? reinterpret_cast<const qc*>(in) + b * H : nullptr;
      io.outa = out + a * N; io.outb = b < batch ? out + b * N : nullptr;
      io.N = N;
      if (op == 1) { io.wmid = 2.f; io.scale = 1.f / N; } else { io.wmid = 1.f; io.scale = 1.f; }
      run_row(R.P, R.e, io, nthr);
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Large-row path (N > 2^14): the launches of qft_large.cuh, emulated phase by
// phase, row by row (each GLOBAL / SLICE task and each NODE group in turn).
static QftLargePlan g_lp;

template <class IO>
static void run_large_row(const QftLargePlan& LP, std::vector<qc>& A, std::vector<qc>& B, int side_len,
                          const float* gsec, const IO& io) {
  std::vector<qc> tab(((1 << LP.r) >> LP.LF) + 4, mkc(NAN, NAN));
  std::vector<qc> Alo(2 * side_len, mkc(NAN, NAN)), Blo(2 * side_len, mkc(NAN, NAN));
  auto eng = [&](int copy) {
    Eng e;
    qc* base = copy ? B.data() : A.data();
    qc* lb = copy ? Blo.data() : Alo.data();
    e.side0 = base; e.side1 = base + side_len; e.sec = gsec; e.r = LP.r; e.N = 1 << LP.r;
    e.tabC = tab.data(); e.tabS = tab.data() + ((1 << LP.r) >> LP.LF) / 2 + 1;
    e.lo0 = lb; e.lo1 = lb + side_len;
    if (LP.inplace) { e.lay_nb = LP.NB; e.lay_l1 = LP.L1; }
    return e;
  };
  for (int ph = 0; ph < LP.nphase; ++ph) {
    const QftLargePhase& P = LP.phases[ph];
    if (P.kind == QFT_LPH_TAB) {
      const Eng e = eng(0);
      for (int m = 1; m <= LP.r - LP.LF; ++m) {
        tab_level_c(e, m, 0, 1);
        if (m >= 2) tab_level_s(e, m, 0, 1);
      }
    } else if (P.kind == QFT_LPH_GLOBAL) {
      const Eng e = eng(0);
      const int NT = 256, TPT = 4;
      const int nblk = (P.ntasks + NT * TPT - 1) / (NT * TPT);
      for (int bx = 0; bx < nblk; ++bx)
        for (int tid = 0; tid < NT; ++tid) {
          const int T0 = bx * NT * TPT + tid, T1 = bx * NT * TPT + NT * TPT;
          for (int s = P.seg0; s < P.seg0 + P.nseg; ++s) {
            const QftSeg& sg = LP.segs[s];
            if (sg.begin >= T1 || sg.begin + sg.count <= T0 - tid) continue;
            int first = T0 - sg.begin;
            if (first < 0) first += ((-first + NT - 1) / NT) * NT;
            int end = T1 - sg.begin;
            if (end > sg.count) end = sg.count;
            run_plain_segment<3, IO, true>(LP.LF, sg, e, io, first, end, NT, 0);
          }
        }
    } else if (P.kind == QFT_LPH_SLICE && LP.inplace) {
      // in place: the halo copies first (a launch of its own), then each
      // block reads all its tasks' cells before it writes any
      const Eng e = eng(0);
      const int nblk = (P.ntasks + QFT_IP_TASKS - 1) / QFT_IP_TASKS;
      std::vector<qc> hh((size_t)(nblk + 1) * QFT_IP_HALO, mkc(NAN, NAN)), hl(hh.size(), mkc(NAN, NAN));
      for (int k = 1; k < nblk; ++k)
        slice_ip_edge(LP.segs, P.seg0, P.nseg, e, k, &hh[(size_t)k * QFT_IP_HALO], &hl[(size_t)k * QFT_IP_HALO]);
      std::vector<SliceIp> regs(QFT_IP_TASKS);
      std::vector<int> segi(QFT_IP_TASKS);
      // odd blocks before even ones: at every edge one of the two blocks has
      // already written when the other reads, as CTAs may run on the GPU
      for (int it = 0; it < nblk; ++it) {
        const int bx = it < nblk / 2 ? 2 * it + 1 : 2 * (it - nblk / 2);
        for (int x = 0; x < QFT_IP_TASKS; ++x) {
          const int tau = bx * QFT_IP_TASKS + x;
          segi[x] = -1;
          if (tau >= P.ntasks) continue;
          int s = P.seg0;
          while (s + 1 < P.seg0 + P.nseg && LP.segs[s + 1].begin <= tau) ++s;
          segi[x] = s;
          const QftSeg& sg = LP.segs[s];
          const int slot = slice_ip_halo_slot(sg.side, x, bx);
          run_slice_ip_read(sg, e, tau - sg.begin, slot >= 0 ? &hh[slot] : nullptr, slot >= 0 ? &hl[slot] : nullptr,
                            sg.pad[2] != 0, regs[x]);
        }
        for (int x = 0; x < QFT_IP_TASKS; ++x)
          if (segi[x] >= 0) run_slice_ip_write(LP.segs[segi[x]], e, LP.segs[segi[x]].pad[2] != 0, regs[x]);
      }
    } else if (P.kind == QFT_LPH_SLICE) {
      for (int tau = 0; tau < P.ntasks; ++tau) {
        int s = P.seg0;
        while (s + 1 < P.seg0 + P.nseg && LP.segs[s + 1].begin <= tau) ++s;
        const QftSeg& sg = LP.segs[s];
        if (sg.pad[2]) {
          SliceRegsC regs;
          run_slice_read_c(sg, eng(sg.pad[0]), tau - sg.begin, regs);
          run_slice_write_c(sg, eng(sg.pad[1]), regs);
        } else {
          SliceRegs regs;
          run_slice_read(sg, eng(sg.pad[0]), tau - sg.begin, regs);
          run_slice_write(sg, eng(sg.pad[1]), regs);
        }
      }
    } else {
      std::vector<float> secp(gsec, gsec + (1 << LP.NB) + 1);
      for (int k = 0; k < LP.nsub; ++k) {
        const QftNodeSub& S = LP.subs[k];
        const int ngroups = S.nodes / S.group;
        for (int g = 0; g < ngroups; ++g) {
          const int ncell = S.group << S.nb;
          const int base = cls_off(LP.r, S.cls) + g * ncell;
          const int pb = qft_pidx(base), pn = qft_pidx(ncell - 1) + 1;
          std::vector<qc> win(pn), lwin(pn, mkc(NAN, NAN));
          const Eng ea = eng(0);
          const qc* src = side_ptr(ea, S.side) + pb;
          for (int i = 0; i < pn; ++i) win[i] = src[i];
          if (S.comp) {
            const qc* lsrc = lo_ptr(ea, S.side) + pb;
            for (int i = 0; i < pn; ++i) lwin[i] = lsrc[i];
          }
          Eng e;
          e.side0 = win.data() - pb; e.side1 = win.data() - pb;
          e.sec = secp.data(); e.r = LP.r; e.N = 1 << LP.r; e.tabC = nullptr; e.tabS = nullptr;
          e.lo0 = lwin.data() - pb; e.lo1 = lwin.data() - pb;
          run_row<NoIO, true>(S.plan, e, NoIO(), 512, g);
          const Eng ed = eng(S.dst);
          qc* dst = side_ptr(ed, S.side) + pb;
          for (int i = 0; i < pn; ++i) dst[i] = win[i];
          if (S.comp) {
            qc* ldst = lo_ptr(ed, S.side) + pb;
            for (int i = 0; i < pn; ++i) ldst[i] = lwin[i];
          }
        }
      }
    }
  }
}

// op as in emu_c2c (complex64 rows)
// plain = 1: every class tree in plain FP32 (else the library's compensated classes)
// plain = 1: J = 0; plain < 0: J = -plain (another count, for tests)
// inplace = 1: the one-scratch schedule (every phase in copy A)
extern "C" int emu_c2c_large(int N, int64_t batch, const float* in, float* out, int op, int plain, int NB,
                             int inplace) {
  int r = 0; while ((1 << r) < N) ++r;
  QftTune t = qft_default_tune(r);
  const int J = plain > 0 ? 0 : (plain < 0 ? -plain : qft_comp_classes(r));
  if (qft_build_large_plan(r, t, NB, 512, &g_lp, J, inplace) != 0) return -2;
  std::vector<float> gsec(N / 4 + 1, 0.f);
  qft_fill_gray_secants(r, gsec.data());
  const int side_len = qft_side_len(N);
  std::vector<qc> A(2 * side_len, mkc(NAN, NAN)), B(2 * side_len, mkc(NAN, NAN));
  for (int64_t b = 0; b < batch; ++b) {
    IoC2C<StC64> io;
    io.in = reinterpret_cast<const qc*>(in) + b * N;
    io.out = reinterpret_cast<qc*>(out) + b * N;
    io.N = N; io.scale = 1.f; io.scaled = false;
    io.in_op = io.out_op = QFT_LANE_ID;
    if (op == 1) { io.in_op = io.out_op = QFT_LANE_SWAP; io.scale = 1.f / N; io.scaled = true; }
    if (op == 2) { io.in_op = io.out_op = QFT_LANE_CONJ; }
    if (op == 3) { io.scale = 1.f / N; io.scaled = true; }
    run_large_row(g_lp, A, B, side_len, gsec.data(), io);
  }
  return 0;
}

// R2C family on the large path (op as in emu_r2c)
extern "C" int emu_r2c_large(int N, int64_t batch, const float* in, float* out, int op, int plain, int inplace) {
  int r = 0; while ((1 << r) < N) ++r;
  QftTune t = qft_default_tune(r);
  const int J = plain ? 0 : qft_comp_classes(r);
  if (qft_build_large_plan(r, t, 12, 512, &g_lp, J, inplace) != 0) return -2;
  std::vector<float> gsec(N / 4 + 1, 0.f);
  qft_fill_gray_secants(r, gsec.data());
  const int side_len = qft_side_len(N);
  std::vector<qc> A(2 * side_len), B(2 * side_len);
  const int64_t H = N / 2 + 1;
  for (int64_t it = 0; it < (batch + 1) / 2; ++it) {
    const int64_t a = 2 * it, b = 2 * it + 1;
    if (op == 0 || op == 3) {
      IoR2C<StC64> io;
      io.ina = in + a * N; io.inb = b < batch ? in + b * N : nullptr;
      io.outa = reinterpret_cast<qc*>(out) + a * H; io.outb = b < batch ? reinterpret_cast<qc*>(out) + b * H : nullptr;
      io.N = N; io.wscale = op == 0 ? 0.f : 1.f / N;
      run_large_row(g_lp, A, B, side_len, gsec.data(), io);
    } else {
      IoC2R<StC64> io;
      io.ina = reinterpret_cast<const qc*>(in) + a * H; io.inb = b < batch ? reinterpret_cast<const qc*>(in) + b * H : nullptr;
      io.outa = out + a * N; io.outb = b < batch ? out + b * N : nullptr;
      io.N = N;
      if (op == 1) { io.wmid = 2.f; io.scale = 1.f / N; } else { io.wmid = 1.f; io.scale = 1.f; }
      run_large_row(g_lp, A, B, side_len, gsec.data(), io);
    }
  }
  return 0;
}

// The in-place order of the large-row path's one-scratch schedule (ip_perm),
// exported for its host tests.
extern "C" int emu_ip_perm(int i, int dp, int sb) { return ip_perm(i, dp, sb); }
