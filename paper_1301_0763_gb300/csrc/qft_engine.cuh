// qft_engine.cuh -- the improved-QFT row engine (Pasquini, "Improved QFT
// algorithm for power-of-two FFT", Sec. 3-5), written once for the sm_103a
// kernels and, with QFT_HOST_EMULATION, for a host build used only by the
// test-suite to check the engine's index logic without a GPU.
//
// Data layout of one row (N = 2^r, r >= 2) in shared memory
// ----------------------------------------------------------
// The CDFT is split (Sec. 4.1/4.2; complex data pushed through the
// real-coefficient network, re and im lanes together) into
//   c(n) = z(n) + z(N-n)  (s_dc_tt, n in [0, N/2]) and
//   d(n) = z(n) - z(N-n)  (s_ds_tt, n in [1, N/2-1]).
// dct and dst first separate even from odd time indices (Sec. 3.1) and halve
// the even ones (Sec. 3.4), recursively; unrolled, this partitions the time
// indices by their 2-adic valuation: class j holds n = 2^j * (2c+1),
// c in [0, P_j), P_j = N / 2^(j+2), and is one dct_ot / dst_ot of
// periodization N / 2^j.  DCT classes are j = 0..r-2, DST classes j = 0..r-3.
// Each side (DCT, DST) is one array of N/2+1 complex cells:
//   class j occupies [N/2 - 2^(r-1-j), N/2 - 2^(r-2-j)),
//   DCT: c(0) at N/2-1, c(N/2) at N/2;  DST: d(N/4) (the dst(4) base) at N/2-2.
// Shared-memory addresses are padded by one cell every 16 (qft_pidx) so that
// strided task accesses do not collide on banks.
//
// Forward phase of a class (Sec. 3.2 + 3.3, eqs qft_1, qft_2, qft_9, qft_10,
// and the secant conversion of dct_oo / dst_oo, eq qft_38A): a node of
// 2^b cells (own time index n = 2c+1, periodization M = 2^(b+2)) splits by
// the mirror butterfly s(n) +- s(M/2-n) into its even-harmonic child (a
// dct_ot / dst_ot of periodization M/2) and its odd-harmonic child, which is
// scaled by 1/(2cos(2 pi n/M)) and is then also a dct_ot / dst_ot of
// periodization M/2.  Cells are stored in Gray order: slot g holds own cell
// invgray(g).  In that order the mirror partner of a cell differs only in the
// node's top slot bit, the even-harmonic child keeps the lower half, the
// odd-harmonic child the upper half, and both children are again in their own
// Gray order -- so the whole forward phase is an in-place radix-2 network.
//
// Backward phase (eqs qft_4B, qft_38B (read as X(M/4-1) = Y(M/8-1)),
// qft_38C): outputs are kept in natural frequency order per node; a node's
// output interleaves E (even harmonics) with Y(j) + Y(j+1) (odd harmonics,
// DCT) or Z(j-1) + Z(j) (DST, stored at k-1).
//
// Final phase (eqs qft_5C, qft_5D, qft_6 and their DST forms; Sec. 4.1):
// C_M(k) = C_{M/2}(k) + O(k), C_M(M/2-k) = C_{M/2}(k) - O(k), C_M(M/4) =
// C_{M/2}(M/4); S_M(k) = S_{M/2}(k) + O(k), S_M(M/2-k) = O(k) - S_{M/2}(k),
// S_M(M/4) = O(M/4); X(k) = C(k) - i S(k), X(N-k) = C(k) + i S(k).
//
// Every arithmetic operation is a single round-to-nearest fp32 operation on
// each lane (never contracted into an FMA), and the operands of every
// operation are exactly the ones the recursion of Sec. 5 prescribes, so the
// engine's result does not depend on the order in which tasks run.
#pragma once

#include <stdint.h>
#include "qft_plan.h"

#if defined(__CUDACC__) && !defined(QFT_HOST_EMULATION)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#define QFT_HD __host__ __device__ __forceinline__
// tasks that run a few times per row (inlined like the others: out-of-line calls cost spills)
#define QFT_RARE __host__ __device__ __forceinline__
typedef float2 qc;
#else
#include <string.h>
#include <math.h>
#define QFT_HD inline
#define QFT_RARE inline
struct qc { float x, y; };
#endif

namespace qft {

// ------------------------------------------------------------ arithmetic
QFT_HD qc mkc(float x, float y) { qc r; r.x = x; r.y = y; return r; }

// Complex adds and subtracts use the packed two-lane FP32 instructions
// (add/sub.rn.f32x2, one instruction per complex value); multiplies by a
// secant or a scale use the scalar round-to-nearest intrinsic per lane.  With
// both packed multiplies (mul/fma.rn.f32x2) and packed adds in one kernel,
// sm_103a builds did not reproduce the FP32 evaluation of the recursion bit
// for bit (checked again with the compensated products: N = 16 already
// differs), so the packed multiply is not used.  QFT_SCALAR_ARITH selects
// scalar adds too.
#if defined(__CUDA_ARCH__) && !defined(QFT_SCALAR_ARITH)
QFT_HD qc cadd(qc a, qc b) {
  qc r;
  asm("{\n\t.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\t"
      "add.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0,%1}, rc;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
QFT_HD qc csub(qc a, qc b) {
  qc r;
  asm("{\n\t.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\t"
      "sub.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0,%1}, rc;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
QFT_HD qc cmul(qc a, float s) { return mkc(__fmul_rn(a.x, s), __fmul_rn(a.y, s)); }
QFT_HD float fmul(float a, float b) { return __fmul_rn(a, b); }
QFT_HD float fadd(float a, float b) { return __fadd_rn(a, b); }
QFT_HD float fsub(float a, float b) { return __fsub_rn(a, b); }
QFT_HD float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#elif defined(__CUDA_ARCH__)
// scalar round-to-nearest intrinsics (never contracted), one per lane
QFT_HD qc cadd(qc a, qc b) { return mkc(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
QFT_HD qc csub(qc a, qc b) { return mkc(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
QFT_HD qc cmul(qc a, float s) { return mkc(__fmul_rn(a.x, s), __fmul_rn(a.y, s)); }
QFT_HD float fmul(float a, float b) { return __fmul_rn(a, b); }
QFT_HD float fadd(float a, float b) { return __fadd_rn(a, b); }
QFT_HD float fsub(float a, float b) { return __fsub_rn(a, b); }
QFT_HD float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
// host emulation: plain IEEE single precision (built with -ffp-contract=off)
QFT_HD qc cadd(qc a, qc b) { return mkc(a.x + b.x, a.y + b.y); }
QFT_HD qc csub(qc a, qc b) { return mkc(a.x - b.x, a.y - b.y); }
QFT_HD qc cmul(qc a, float s) { return mkc(a.x * s, a.y * s); }
QFT_HD float fmul(float a, float b) { return a * b; }
QFT_HD float fadd(float a, float b) { return a + b; }
QFT_HD float fsub(float a, float b) { return a - b; }
QFT_HD float ffma(float a, float b, float c) { return fmaf(a, b, c); }
#endif

// ------------------------------------------------ compensated arithmetic
// In the compensated class trees every value is an unevaluated pair h + l of
// FP32 numbers: h is exactly the plain FP32 value, l carries the rounding
// errors (the FP32 error of the improved QFT comes from the secant conversion
// of eq qft_38A, whose large factors make every value below them large).
//   add: s = ah + bh, z = s - ah, e = (ah - (s - z)) + (bh - z)  (TwoSum,
//        Knuth: s + e = ah + bh exactly), l = (al + bl) + e
//   sub: the add of (-bh, -bl), written out without the negations
//   mul by a constant c: p = ah c, e = fma(ah, c, -p) (exact), l = fma(al, c, e)
// Each class output is rounded once, h + l.  e is exact, so the results do not
// depend on operand order.
QFT_HD void p_add(qc ah, qc al, qc bh, qc bl, qc& sh, qc& sl) {
  const qc s = cadd(ah, bh);
  const qc z = csub(s, ah);
  const qc e = cadd(csub(ah, csub(s, z)), csub(bh, z));
  sl = cadd(cadd(al, bl), e);
  sh = s;
}
QFT_HD void p_sub(qc ah, qc al, qc bh, qc bl, qc& sh, qc& sl) {
  const qc s = csub(ah, bh);
  const qc z = csub(s, ah);
  const qc e = csub(csub(ah, csub(s, z)), cadd(bh, z));   // (ah - (s - z)) + (-bh - z)
  sl = cadd(csub(al, bl), e);
  sh = s;
}
QFT_HD void p_mul(qc ah, qc al, float c, qc& ph, qc& pl) {
  ph = cmul(ah, c);
  const float ex = ffma(ah.x, c, -ph.x), ey = ffma(ah.y, c, -ph.y);
  pl = mkc(ffma(al.x, c, ex), ffma(al.y, c, ey));
}

// ------------------------------------------------------------ geometry
QFT_HD int qft_pidx(int i) { return i + (i >> 4); }
// Padded index of cell base + t*2^h (h >= 4, base's low 4 bits below 2^h):
// pidx(base) + t * qft_pstride(h), one add per access instead of a shift and two adds.
QFT_HD int qft_pstride(int h) { return (1 << h) + (1 << (h - 4)); }
// padded cells per side of a scratch row, rounded up to even so that every
// row and both sides start on a 16-byte boundary
QFT_HD int qft_side_len(int N) { return (qft_pidx(N / 2) + 2) & ~1; }
QFT_HD int cls_off(int r, int j) { return (1 << (r - 1)) - (1 << (r - 1 - j)); }
QFT_HD int cls_bits(int r, int j) { return r - 2 - j; }
// Bit reversal of the low n bits of x (1 <= n <= 31).
QFT_HD unsigned qft_brev(unsigned x, int n) {
#if defined(__CUDA_ARCH__)
  return __brev(x) >> (32 - n);
#else
  unsigned y = 0;
  for (int i = 0; i < n; ++i) y |= ((x >> i) & 1u) << (n - 1 - i);
  return y;
#endif
}
// In-place backward order of a node of 2^sb cells whose top dp backward levels
// ran in place: natural index i sits at bitrev_dp(i mod 2^dp) 2^(sb-dp) +
// floor(i / 2^dp).  One in-place level over descendants t of 2^s cells keeps
// output u of chunk i in descendant bitrev(u)'s cell i, which composes to this.
QFT_HD int ip_perm(int i, int dp, int sb) {
  return dp > 0 ? (int)((qft_brev((unsigned)i & ((1u << dp) - 1u), dp) << (sb - dp)) | (unsigned)(i >> dp)) : i;
}
QFT_HD unsigned invgray(unsigned g) {
  g ^= g >> 1; g ^= g >> 2; g ^= g >> 4; g ^= g >> 8; g ^= g >> 16;
  return g;
}
#if defined(__CUDACC__) && !defined(QFT_HOST_EMULATION)
__host__ __device__ constexpr int ig_c(int x) { return x ^ (x >> 1) ^ (x >> 2) ^ (x >> 3) ^ (x >> 4) ^ (x >> 5); }
#else
static constexpr int ig_c(int x) { return x ^ (x >> 1) ^ (x >> 2) ^ (x >> 3) ^ (x >> 4) ^ (x >> 5); }
#endif

// Everything a phase needs about the row being transformed.
struct Eng {
  qc* side0;          // DCT side (padded), N/2+1 cells
  qc* side1;          // DST side (padded)
  const float* sec;   // Gray-ordered secants (qft_fill_gray_secants): node of 2^b cells,
                      // lower butterfly slot g -> sec[2^(b-1) + g]
  int r;              // log2 N
  int N;
  qc* tabC;           // C_Mt(k), k in [0, Mt/2]   (Mt = N >> LF), or null
  qc* tabS;           // S_Mt(k), k in [1, Mt/2-1], or null
  qc* lo0;            // lo parts of the DCT side's compensated cells (same indexing), or null
  qc* lo1;            // lo parts of the DST side
  // Layout of the class outputs.  lay_nb = 0: natural order.  Otherwise (the
  // large-row path's in-place schedule, node size 2^lay_nb, F1 levels lay_l1)
  // the backward levels above each class's node depth ran in place and left
  // the outputs in the order cls_pos gives.
  int lay_nb = 0;
  int lay_l1 = 0;
};

QFT_HD qc* side_ptr(const Eng& e, int s) { return s ? e.side1 : e.side0; }
QFT_HD qc* lo_ptr(const Eng& e, int s) { return s ? e.lo1 : e.lo0; }

// Backward levels of class j that ran in place (0: natural order): the levels
// above its node depth, max(b - NB, L1) for the classes the large-row path
// cuts into nodes (b > L1), none for the others.
QFT_HD int cls_lay_depth(const Eng& e, int j) {
  const int b = cls_bits(e.r, j);
  if (e.lay_nb == 0 || b <= e.lay_l1) return 0;
  return b - e.lay_nb > e.lay_l1 ? b - e.lay_nb : e.lay_l1;
}
// Padded position of stored output i of class j (DCT: k = i, DST: k = i + 1).
// Indices past the class (dummy reads of the chain walks) stay natural.
QFT_HD int cls_pos(const Eng& e, int j, int i) {
  const int b = cls_bits(e.r, j);
  const int d = cls_lay_depth(e, j);
  return qft_pidx(cls_off(e.r, j) + ((d > 0 && i < (1 << b)) ? ip_perm(i, d, b) : i));
}

// L2 prefetch of one cell of a scratch row in global memory (a hint; the
// large-row kernels give it the cells of the task a thread runs next)
QFT_HD void prefetch_cell(const qc* p) {
#if defined(__CUDA_ARCH__)
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
#else
  (void)p;
#endif
}

// ------------------------------------------------- forward mirror levels
// L levels of the forward phase on registers v[t], t in [0, 2^L).  Register t
// holds node slot t*H + lo (H = 2^(nb-L)) of a node of 2^nb cells.  Level l
// pairs t and t + 2^(L-l); the node at that level has 2^bp cells
// (bp = nb-l+1) and the lower element sits in its slot hi*H + lo
// (hi = t mod 2^(L-l)), so its secant is sec[2^(bp-1) + hi*H + lo].
// DCT (eqs qft_1, qft_2, qft_38A): e = a + b, o = (a - b) sec.
// DST (roles swapped, Sec. 3.2):   e = a - b, o = (a + b) sec.
template <int L, int SIDE>
QFT_HD void dif_regs(qc (&v)[1 << L], int nb, int lo, const float* sec) {
  const int h = nb - L;
  const float* sl = sec + lo;
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    const int half = 1 << (L - l);
    const float* sb = sl + (1 << (nb - l));
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) {
      if (t & half) continue;
      const float s = sb[(t & (half - 1)) << h];
      const qc a = v[t], b = v[t | half];
      if (SIDE == 0) { v[t] = cadd(a, b); v[t | half] = cmul(csub(a, b), s); }
      else           { v[t] = csub(a, b); v[t | half] = cmul(cadd(a, b), s); }
    }
  }
}

// The same levels on compensated pairs (v = h parts, w = l parts).
template <int L, int SIDE>
QFT_HD void dif_regs_c(qc (&v)[1 << L], qc (&w)[1 << L], int nb, int lo, const float* sec) {
  const int h = nb - L;
  const float* sl = sec + lo;
#pragma unroll
  for (int l = 1; l <= L; ++l) {
    const int half = 1 << (L - l);
    const float* sb = sl + (1 << (nb - l));
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) {
      if (t & half) continue;
      const float s = sb[(t & (half - 1)) << h];
      const qc a = v[t], al = w[t], b = v[t | half], bl = w[t | half];
      qc dh, dl;
      if (SIDE == 0) { p_add(a, al, b, bl, v[t], w[t]); p_sub(a, al, b, bl, dh, dl); }
      else           { p_sub(a, al, b, bl, v[t], w[t]); p_add(a, al, b, bl, dh, dl); }
      p_mul(dh, dl, s, v[t | half], w[t | half]);
    }
  }
}

// ------------------------------------------------------ backward levels
// Backward phase of L tree levels on w[t] (t = path of a depth-L descendant,
// MSB first, 0 = even-harmonic child, 1 = odd-harmonic child).  On entry w[t]
// holds one frequency value of descendant t (the chunk of this task); on exit
// w holds 2^L consecutive outputs of the top node.  h[t] (t >= 1) is the
// neighbouring value of descendant t (next chunk for DCT, previous chunk for
// DST) used at a chunk edge when hv is true; at a node edge hv is false.
// DCT (dct_ot, eqs qft_4B, qft_38B, qft_38C): X(2i) = E(i),
//   X(2i+1) = Y(i) + Y(i+1), last X(B-1) = Y(B/2-1).
// DST (dst_ot, outputs k = 1..B stored at k-1): X(2i+1) = E(i), X(0) = Z(0),
//   X(2i) = Z(i-1) + Z(i).
template <int L, int SIDE>
QFT_HD void bwd_chunk(qc (&w)[1 << L], const qc* h, bool hv) {
#pragma unroll
  for (int s = 2; s <= (1 << L); s <<= 1) {
    const int hs = s >> 1;
#pragma unroll
    for (int base = 0; base < (1 << L); base += s) {
      qc tmp[1 << L];
#pragma unroll
      for (int i = 0; i < hs; ++i) {
        const qc E = w[base + i];
        const qc Y = w[base + hs + i];
        if (SIDE == 0) {
          tmp[2 * i] = E;
          if (i + 1 < hs) tmp[2 * i + 1] = cadd(Y, w[base + hs + i + 1]);
          else tmp[2 * i + 1] = hv ? cadd(Y, h[base + hs]) : Y;
        } else {
          tmp[2 * i + 1] = E;
          if (i >= 1) tmp[2 * i] = cadd(w[base + hs + i - 1], Y);
          else tmp[2 * i] = hv ? cadd(h[base + hs], Y) : Y;
        }
      }
#pragma unroll
      for (int i = 0; i < s; ++i) w[base + i] = tmp[i];
    }
  }
}

// The same backward levels on compensated pairs.
template <int L, int SIDE>
QFT_HD void bwd_chunk_c(qc (&w)[1 << L], qc (&wl)[1 << L], const qc* h, const qc* hl, bool hv) {
#pragma unroll
  for (int s = 2; s <= (1 << L); s <<= 1) {
    const int hs = s >> 1;
#pragma unroll
    for (int base = 0; base < (1 << L); base += s) {
      qc tmp[1 << L], tml[1 << L];
#pragma unroll
      for (int i = 0; i < hs; ++i) {
        const qc E = w[base + i], El = wl[base + i];
        const qc Y = w[base + hs + i], Yl = wl[base + hs + i];
        if (SIDE == 0) {
          tmp[2 * i] = E; tml[2 * i] = El;
          if (i + 1 < hs) p_add(Y, Yl, w[base + hs + i + 1], wl[base + hs + i + 1], tmp[2 * i + 1], tml[2 * i + 1]);
          else if (hv) p_add(Y, Yl, h[base + hs], hl[base + hs], tmp[2 * i + 1], tml[2 * i + 1]);
          else { tmp[2 * i + 1] = Y; tml[2 * i + 1] = Yl; }
        } else {
          tmp[2 * i + 1] = E; tml[2 * i + 1] = El;
          if (i >= 1) p_add(w[base + hs + i - 1], wl[base + hs + i - 1], Y, Yl, tmp[2 * i], tml[2 * i]);
          else if (hv) p_add(h[base + hs], hl[base + hs], Y, Yl, tmp[2 * i], tml[2 * i]);
          else { tmp[2 * i] = Y; tml[2 * i] = Yl; }
        }
      }
#pragma unroll
      for (int i = 0; i < s; ++i) { w[base + i] = tmp[i]; wl[base + i] = tml[i]; }
    }
  }
}

// ------------------------------------------------------------------ F1
// Large class j: one task = the 2^L1 Gray slots t*H + lo (H = 2^(b-L1),
// lo = gray(ilo)) of both sides.  The cells are loaded straight from the row:
// own cell c -> time index n = 2^j (2c+1); the IO object returns the folded
// pair (c(n), d(n)).
template <int L1, class IO>
QFT_HD void task_f1_big(const Eng& e, const IO& io, int j, int ilo) {
  const int b = cls_bits(e.r, j);
  const int h = b - L1;
  const int H = 1 << h;
  const int lo = ilo ^ (ilo >> 1);
  qc vc[1 << L1], vs[1 << L1];
#pragma unroll
  for (int t = 0; t < (1 << L1); ++t) {
    const int ig = ig_c(t);
    const int c = (ig << h) | ((ig & 1) ? (H - 1 - ilo) : ilo);
    io.get_cd((2 * c + 1) << j, vc[t], vs[t]);
  }
  dif_regs<L1, 0>(vc, b, lo, e.sec);
  dif_regs<L1, 1>(vs, b, lo, e.sec);
  const int off = cls_off(e.r, j);
  if (h >= 4) {   // off is a multiple of 16 here
    const int p0 = qft_pidx(off + lo), ps = qft_pstride(h);
#pragma unroll
    for (int t = 0; t < (1 << L1); ++t) {
      e.side0[p0 + t * ps] = vc[t];
      e.side1[p0 + t * ps] = vs[t];
    }
  } else {
#pragma unroll
    for (int t = 0; t < (1 << L1); ++t) {
      e.side0[qft_pidx(off + t * H + lo)] = vc[t];
      e.side1[qft_pidx(off + t * H + lo)] = vs[t];
    }
  }
}

// The same task for a compensated class: the folded cells enter the class tree
// as pairs (l = 0); h and l parts are stored.
template <int L1, class IO>
QFT_HD void task_f1_big_c(const Eng& e, const IO& io, int j, int ilo) {
  const int b = cls_bits(e.r, j);
  const int h = b - L1;
  const int H = 1 << h;
  const int lo = ilo ^ (ilo >> 1);
  qc vc[1 << L1], vs[1 << L1], wc[1 << L1], ws[1 << L1];
#pragma unroll
  for (int t = 0; t < (1 << L1); ++t) {
    const int ig = ig_c(t);
    const int c = (ig << h) | ((ig & 1) ? (H - 1 - ilo) : ilo);
    io.get_cd((2 * c + 1) << j, vc[t], vs[t]);
    wc[t] = mkc(0.f, 0.f);
    ws[t] = wc[t];
  }
  dif_regs_c<L1, 0>(vc, wc, b, lo, e.sec);
  dif_regs_c<L1, 1>(vs, ws, b, lo, e.sec);
  const int off = cls_off(e.r, j);
  const bool lin = h >= 4;   // off is a multiple of 16 then
  const int p0 = qft_pidx(off + lo), ps = lin ? qft_pstride(h) : 0;
#pragma unroll
  for (int t = 0; t < (1 << L1); ++t) {
    const int pi = lin ? p0 + t * ps : qft_pidx(off + t * H + lo);
    e.side0[pi] = vc[t];
    e.side1[pi] = vs[t];
    e.lo0[pi] = wc[t];
    e.lo1[pi] = ws[t];
  }
}

// Small class j (2^L cells, L = r-2-j): forward and backward in one task.
// Class r-2 (one cell, n = N/4) has no DST class; its DST value d(N/4) is the
// dst(4) base case and goes to the DST base cell.
template <int L, class IO>
QFT_RARE void task_f1_small(const Eng& e, const IO& io, int j) {
  qc vc[1 << L], vs[1 << L];
#pragma unroll
  for (int g = 0; g < (1 << L); ++g) io.get_cd((2 * ig_c(g) + 1) << j, vc[g], vs[g]);
  // off is a multiple of 2^(L+1): the 2^L <= 16 cells lie in one padded block
  const int p0 = qft_pidx(cls_off(e.r, j));
  dif_regs<L, 0>(vc, L, 0, e.sec);
  bwd_chunk<L, 0>(vc, vc, false);
#pragma unroll
  for (int k = 0; k < (1 << L); ++k) e.side0[p0 + k] = vc[k];
  if (j <= e.r - 3) {
    dif_regs<L, 1>(vs, L, 0, e.sec);
    bwd_chunk<L, 1>(vs, vs, false);
#pragma unroll
    for (int k = 0; k < (1 << L); ++k) e.side1[p0 + k] = vs[k];
  } else {
    e.side1[qft_pidx(e.N / 2 - 2)] = vs[0];
  }
}

template <class IO>
QFT_HD void task_f1_base(const Eng& e, const IO& io) {
  e.side0[qft_pidx(e.N / 2 - 1)] = io.get_c(0);
  e.side0[qft_pidx(e.N / 2)] = io.get_c(e.N / 2);
}

// ------------------------------------------------------------ DIF, LEAF
template <int L, int SIDE>
QFT_HD void task_dif(const Eng& e, int j, int D, int tau) {
  const int nb = cls_bits(e.r, j) - D;
  const int h = nb - L;
  const int q = tau >> h;
  const int lo = tau & ((1 << h) - 1);
  qc* A = side_ptr(e, SIDE);
  const int base = cls_off(e.r, j) + (q << nb) + lo;
  qc v[1 << L];
  const bool lin = h >= 4;   // then base - lo is a multiple of 16
  const int p0 = qft_pidx(base), ps = lin ? qft_pstride(h) : 0;
  if (lin) {
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) v[t] = A[p0 + t * ps];
  } else {
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) v[t] = A[qft_pidx(base + (t << h))];
  }
  dif_regs<L, SIDE>(v, nb, lo, e.sec);
  if (lin) {
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) A[p0 + t * ps] = v[t];
  } else {
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) A[qft_pidx(base + (t << h))] = v[t];
  }
}

template <int L, int SIDE>
QFT_HD void task_leaf(const Eng& e, int j, int q) {
  qc* A = side_ptr(e, SIDE);
  const int base = cls_off(e.r, j) + (q << L);
  // base is a multiple of 2^L <= 16: the node's cells lie in one padded block
  const int p0 = qft_pidx(base);
  qc v[1 << L];
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) v[t] = A[p0 + t];
  dif_regs<L, SIDE>(v, L, 0, e.sec);
  bwd_chunk<L, SIDE>(v, v, false);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) A[p0 + t] = v[t];
}

template <int L, int SIDE>
QFT_HD void task_dif_c(const Eng& e, int j, int D, int tau) {
  const int nb = cls_bits(e.r, j) - D;
  const int h = nb - L;
  const int q = tau >> h;
  const int lo = tau & ((1 << h) - 1);
  qc* A = side_ptr(e, SIDE);
  qc* Al = lo_ptr(e, SIDE);
  const int base = cls_off(e.r, j) + (q << nb) + lo;
  qc v[1 << L], w[1 << L];
  const bool lin = h >= 4;
  const int p0 = qft_pidx(base), ps = lin ? qft_pstride(h) : 0;
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    const int pi = lin ? p0 + t * ps : qft_pidx(base + (t << h));
    v[t] = A[pi];
    w[t] = Al[pi];
  }
  dif_regs_c<L, SIDE>(v, w, nb, lo, e.sec);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    const int pi = lin ? p0 + t * ps : qft_pidx(base + (t << h));
    A[pi] = v[t];
    Al[pi] = w[t];
  }
}

// The cells task_dif / task_dif_c(tau) reads (and their lo parts if `lo`),
// prefetched into L2.
template <int L, int SIDE>
QFT_HD void task_dif_prefetch(const Eng& e, int j, int D, int tau, bool lo) {
  const int nb = cls_bits(e.r, j) - D;
  const int h = nb - L;
  const int base = cls_off(e.r, j) + ((tau >> h) << nb) + (tau & ((1 << h) - 1));
  const qc* A = side_ptr(e, SIDE);
  const qc* Al = lo_ptr(e, SIDE);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    const int pi = qft_pidx(base + (t << h));
    prefetch_cell(A + pi);
    if (lo) prefetch_cell(Al + pi);
  }
}

template <int L, int SIDE>
QFT_HD void task_leaf_c(const Eng& e, int j, int q) {
  qc* A = side_ptr(e, SIDE);
  qc* Al = lo_ptr(e, SIDE);
  const int base = cls_off(e.r, j) + (q << L);
  const int p0 = qft_pidx(base);
  qc v[1 << L], w[1 << L];
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) { v[t] = A[p0 + t]; w[t] = Al[p0 + t]; }
  dif_regs_c<L, SIDE>(v, w, L, 0, e.sec);
  bwd_chunk_c<L, SIDE>(v, w, v, w, false);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) { A[p0 + t] = v[t]; Al[p0 + t] = w[t]; }
}

// --------------------------------------------------------------- SLICE
// Node at depth D-L (2^nb cells) whose depth-D descendants (2^(b-D) cells
// each, natural frequency order, descendant t at offset t*S) are known.  Task
// (q, r_) produces node outputs [r_ 2^L, (r_+1) 2^L).  The neighbour value
// needed at a chunk edge for the odd-harmonic child of every sub-node is, by
// the even-harmonic copies of the recursion, a raw value of descendant t at
// slice r_+1 (DCT) or r_-1 (DST), for every t >= 1.
#ifndef QFT_MAX_LB
#define QFT_MAX_LB 3    // largest number of backward levels one SLICE task does
#endif
struct SliceRegs {
  qc w[1 << QFT_MAX_LB];
  qc h[1 << QFT_MAX_LB];
  int base;   // node base + r_ * 2^L  (write position)
  bool hv;
};
// compensated SLICE tasks: the l parts as well; `root` marks the tasks that
// produce the class outputs (node at depth 0), which are rounded once, h + l
struct SliceRegsC {
  SliceRegs p;    // h parts, halo flag and write position
  qc wl[1 << QFT_MAX_LB];
  qc hl[1 << QFT_MAX_LB];
  bool root;
};

template <int L, int SIDE>
QFT_HD void task_slice_read(const Eng& e, int j, int D, int tau, SliceRegs& s) {
  const int b = cls_bits(e.r, j);
  const int sb = b - D;                   // log2 S
  const int S = 1 << sb;
  const int nb = b - (D - L);
  const int q = tau >> sb;
  const int rr = tau & (S - 1);
  const qc* A = side_ptr(e, SIDE);
  const int nbase = cls_off(e.r, j) + (q << nb);
  const bool hv = SIDE == 0 ? (rr + 1 < S) : (rr >= 1);
  const int hoff = SIDE == 0 ? rr + 1 : rr - 1;
  if (sb >= 4) {   // nbase is a multiple of 16 here
    const int ps = qft_pstride(sb);
    const int pw = qft_pidx(nbase + rr);
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) s.w[t] = A[pw + t * ps];
    if (hv) {
      const int ph = qft_pidx(nbase + hoff);
#pragma unroll
      for (int t = 1; t < (1 << L); ++t) s.h[t] = A[ph + t * ps];
    }
  } else {
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) s.w[t] = A[qft_pidx(nbase + t * S + rr)];
    if (hv) {
#pragma unroll
      for (int t = 1; t < (1 << L); ++t) s.h[t] = A[qft_pidx(nbase + t * S + hoff)];
    }
  }
  s.hv = hv;
  s.base = nbase + (rr << L);
  // the backward levels run here, so that only the 2^L outputs stay live until
  // the write (across the SLICE round's barrier in the row kernel)
  qc w[1 << L];
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) w[t] = s.w[t];
  bwd_chunk<L, SIDE>(w, s.h, hv);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) s.w[t] = w[t];
}

// The cells task_slice_read / task_slice_read_c(tau) reads from its node's
// descendants (not the halo: a neighbour lane's cells), and their lo parts if
// `lo`, prefetched into L2.
template <int L, int SIDE>
QFT_HD void task_slice_prefetch(const Eng& e, int j, int D, int tau, bool lo) {
  const int b = cls_bits(e.r, j);
  const int sb = b - D;
  const int S = 1 << sb;
  const int nb = b - (D - L);
  const int nbase = cls_off(e.r, j) + ((tau >> sb) << nb) + (tau & (S - 1));
  const qc* A = side_ptr(e, SIDE);
  const qc* Al = lo_ptr(e, SIDE);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    const int pi = qft_pidx(nbase + t * S);
    prefetch_cell(A + pi);
    if (lo) prefetch_cell(Al + pi);
  }
}

template <int L, int SIDE>
QFT_HD void task_slice_write(const Eng& e, SliceRegs& s) {
  qc* A = side_ptr(e, SIDE);
  const int p0 = qft_pidx(s.base);   // s.base is a multiple of 2^L <= 16
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) A[p0 + t] = s.w[t];
}

template <int L, int SIDE>
QFT_HD void task_slice_read_c(const Eng& e, int j, int D, int tau, SliceRegsC& s) {
  const int b = cls_bits(e.r, j);
  const int sb = b - D;
  const int S = 1 << sb;
  const int nb = b - (D - L);
  const int q = tau >> sb;
  const int rr = tau & (S - 1);
  const qc* A = side_ptr(e, SIDE);
  const qc* Al = lo_ptr(e, SIDE);
  const int nbase = cls_off(e.r, j) + (q << nb);
  const bool hv = SIDE == 0 ? (rr + 1 < S) : (rr >= 1);
  const int hoff = SIDE == 0 ? rr + 1 : rr - 1;
  const bool lin = sb >= 4;
  const int ps = lin ? qft_pstride(sb) : 0;
  const int pw = qft_pidx(nbase + rr);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    const int pi = lin ? pw + t * ps : qft_pidx(nbase + t * S + rr);
    s.p.w[t] = A[pi];
    s.wl[t] = Al[pi];
  }
  if (hv) {
    const int ph = qft_pidx(nbase + hoff);
#pragma unroll
    for (int t = 1; t < (1 << L); ++t) {
      const int pi = lin ? ph + t * ps : qft_pidx(nbase + t * S + hoff);
      s.p.h[t] = A[pi];
      s.hl[t] = Al[pi];
    }
  }
  s.p.hv = hv;
  s.root = D == L;
  s.p.base = nbase + (rr << L);
  // backward levels now: only the outputs stay live until the write
  qc w[1 << L], wl[1 << L];
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) { w[t] = s.p.w[t]; wl[t] = s.wl[t]; }
  bwd_chunk_c<L, SIDE>(w, wl, s.p.h, s.hl, hv);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) { s.p.w[t] = w[t]; s.wl[t] = wl[t]; }
}

template <int L, int SIDE>
QFT_HD void task_slice_write_c(const Eng& e, SliceRegsC& s) {
  qc* A = side_ptr(e, SIDE);
  qc* Al = lo_ptr(e, SIDE);
  const int p0 = qft_pidx(s.p.base);
  if (s.root) {
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) A[p0 + t] = cadd(s.p.w[t], s.wl[t]);   // class output, rounded once
  } else {
#pragma unroll
    for (int t = 0; t < (1 << L); ++t) { A[p0 + t] = s.p.w[t]; Al[p0 + t] = s.wl[t]; }
  }
}

// ------------------------------------------------- in-place SLICE (large rows)
// The large-row path's one-scratch schedule runs the backward levels above the
// node depth in place.  A task reads the cells of its chunk i (natural index)
// in the 2^L descendants of its node, at the positions the levels below left
// them (ip_perm), and writes output u of the chunk over descendant
// bitrev_L(u)'s cell: the cells it writes are the cells it read.  So a block
// of tasks can read, wait for its own reads (a CTA barrier), and write; only
// the neighbour cells of a chunk (eqs qft_38B/C) at a block edge belong to
// another block, and those are copied out before the level starts
// (task_slice_ip_halo).
struct SliceIp {
  qc w[1 << QFT_MAX_LB];    // outputs (h parts)
  qc wl[1 << QFT_MAX_LB];   // lo parts (compensated segments)
  int nbase;                // class-level index of the node
  int sb;                   // log2 of a descendant's cells
  int prr;                  // position of chunk i within a descendant
  bool root;                // compensated class output: stored rounded, h + l
};

// Neighbour cells (descendants t = 1 .. 2^L-1) of the chunk that task `loc`
// of segment (j, D, L) at a block edge takes from the other block: for the
// DCT side the cells of chunk i = loc's (the task before it needs them), for
// the DST side those of chunk i - 1 (loc needs them).  Nothing when loc starts
// a node.  Returns whether it copied.
template <int SIDE>
QFT_HD bool task_slice_ip_halo(const Eng& e, int j, int D, int L, int loc, qc* xh, qc* xl) {
  const int b = cls_bits(e.r, j);
  const int sb = b - D;
  const int rr = loc & ((1 << sb) - 1);
  if (rr == 0) return false;
  const int nbase = cls_off(e.r, j) + ((loc >> sb) << (sb + L));
  const int ph = ip_perm(SIDE == 0 ? rr : rr - 1, cls_lay_depth(e, j) - D, sb);
  const qc* A = side_ptr(e, SIDE);
  const qc* Al = lo_ptr(e, SIDE);
  for (int t = 1; t < (1 << L); ++t) {
    const int pi = qft_pidx(nbase + (t << sb) + ph);
    xh[t] = A[pi];
    if (xl) xl[t] = Al[pi];
  }
  return true;
}

// xh / xl: the chunk's neighbour cells from the halo copy (a task at a block
// edge), or null to read them from the scratch.
template <int L, int SIDE, bool C>
QFT_HD void task_slice_ip_read(const Eng& e, int j, int D, int tau, const qc* xh, const qc* xl, SliceIp& s) {
  const int b = cls_bits(e.r, j);
  const int sb = b - D;
  const int S = 1 << sb;
  const int rr = tau & (S - 1);
  const int dp = cls_lay_depth(e, j) - D;
  const int nbase = cls_off(e.r, j) + ((tau >> sb) << (sb + L));
  const int prr = ip_perm(rr, dp, sb);
  const qc* A = side_ptr(e, SIDE);
  const qc* Al = lo_ptr(e, SIDE);
  qc w[1 << L], wl[1 << L], h[1 << L], hl[1 << L];
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    const int pi = qft_pidx(nbase + (t << sb) + prr);
    w[t] = A[pi];
    if (C) wl[t] = Al[pi];
  }
  const bool hv = SIDE == 0 ? (rr + 1 < S) : (rr >= 1);
  if (hv) {
    if (xh) {
#pragma unroll
      for (int t = 1; t < (1 << L); ++t) {
        h[t] = xh[t];
        if (C) hl[t] = xl[t];
      }
    } else {
      const int ph = ip_perm(SIDE == 0 ? rr + 1 : rr - 1, dp, sb);
#pragma unroll
      for (int t = 1; t < (1 << L); ++t) {
        const int pi = qft_pidx(nbase + (t << sb) + ph);
        h[t] = A[pi];
        if (C) hl[t] = Al[pi];
      }
    }
  }
  if (C) bwd_chunk_c<L, SIDE>(w, wl, h, hl, hv);
  else bwd_chunk<L, SIDE>(w, h, hv);
#pragma unroll
  for (int t = 0; t < (1 << L); ++t) {
    s.w[t] = w[t];
    if (C) s.wl[t] = wl[t];
  }
  s.nbase = nbase;
  s.sb = sb;
  s.prr = prr;
  s.root = C && D == L;
}

template <int L, int SIDE, bool C>
QFT_HD void task_slice_ip_write(const Eng& e, const SliceIp& s) {
  qc* A = side_ptr(e, SIDE);
  qc* Al = lo_ptr(e, SIDE);
#pragma unroll
  for (int u = 0; u < (1 << L); ++u) {
    const int pi = qft_pidx(s.nbase + ((int)qft_brev((unsigned)u, L) << s.sb) + s.prr);
    if (C && s.root) {
      A[pi] = cadd(s.w[u], s.wl[u]);   // class output, rounded once
    } else {
      A[pi] = s.w[u];
      if (C) Al[pi] = s.wl[u];
    }
  }
}

// Block edge k (task B = k QFT_IP_TASKS) of an in-place SLICE phase whose
// segments are segs[seg0, seg0 + nseg): copies the neighbour cells that cross
// it into xh (and their lo parts into xl, if xl and the segment is
// compensated).  Returns false where the edge is not inside one node.
QFT_HD bool slice_ip_edge(const QftSeg* segs, int seg0, int nseg, const Eng& e, int k, qc* xh, qc* xl) {
  const int B = k * QFT_IP_TASKS;
  int s = seg0;
  while (s + 1 < seg0 + nseg && segs[s + 1].begin <= B) ++s;
  const QftSeg& sg = segs[s];
  if (B - 1 < sg.begin || B >= sg.begin + sg.count) return false;
  qc* l = sg.pad[2] ? xl : nullptr;
  return sg.side ? task_slice_ip_halo<1>(e, sg.cls, sg.D, sg.L, B - sg.begin, xh, l)
                 : task_slice_ip_halo<0>(e, sg.cls, sg.D, sg.L, B - sg.begin, xh, l);
}
// Offset (in halo cells) of the copy a task at position x of block bx takes
// its neighbour cells from, or -1 (they are in its own block): the last task
// of a block on the DCT side, the first on the DST side.
QFT_HD int slice_ip_halo_slot(int side, int x, int bx) {
  if (side == 0 && x == QFT_IP_TASKS - 1) return (bx + 1) * QFT_IP_HALO;
  if (side == 1 && x == 0) return bx * QFT_IP_HALO;
  return -1;
}

// dispatch on the segment's L (1..3), side and compensation
QFT_HD void run_slice_ip_read(const QftSeg& sg, const Eng& e, int loc, const qc* xh, const qc* xl, bool comp,
                              SliceIp& s) {
#define QFT_IPR(LL)                                                                       \
  case LL:                                                                                \
    if (comp) {                                                                           \
      if (sg.side) task_slice_ip_read<LL, 1, true>(e, sg.cls, sg.D, loc, xh, xl, s);      \
      else task_slice_ip_read<LL, 0, true>(e, sg.cls, sg.D, loc, xh, xl, s);              \
    } else {                                                                              \
      if (sg.side) task_slice_ip_read<LL, 1, false>(e, sg.cls, sg.D, loc, xh, xl, s);     \
      else task_slice_ip_read<LL, 0, false>(e, sg.cls, sg.D, loc, xh, xl, s);             \
    }                                                                                     \
    break;
  switch (sg.L) {
    QFT_IPR(1) QFT_IPR(2) QFT_IPR(3)
    default: break;
  }
#undef QFT_IPR
}

QFT_HD void run_slice_ip_write(const QftSeg& sg, const Eng& e, bool comp, const SliceIp& s) {
#define QFT_IPW(LL)                                                                       \
  case LL:                                                                                \
    if (comp) {                                                                           \
      if (sg.side) task_slice_ip_write<LL, 1, true>(e, s); else task_slice_ip_write<LL, 0, true>(e, s);   \
    } else {                                                                              \
      if (sg.side) task_slice_ip_write<LL, 1, false>(e, s); else task_slice_ip_write<LL, 0, false>(e, s); \
    }                                                                                     \
    break;
  switch (sg.L) {
    QFT_IPW(1) QFT_IPW(2) QFT_IPW(3)
    default: break;
  }
#undef QFT_IPW
}

// --------------------------------------------------------------- FINAL
// Class output O_j(k) of side s: DCT k in [0, P_j) at off+k; DST k in [1, P_j]
// at off+k-1.
// IP = false: the caller knows the outputs are in natural order (e.lay_nb = 0).
template <bool IP = true>
QFT_HD qc cls_out(const Eng& e, int s, int j, int k) {
  return side_ptr(e, s)[IP ? cls_pos(e, j, k - s) : qft_pidx(cls_off(e.r, j) + k - s)];
}

// C_M(k) for M = 2^m, k in [0, M/2]: walk down the dct recursion (recording
// which of eqs qft_5C / qft_5D / qft_6 applies at each level), then add the
// class outputs bottom-up in the recursion's order.  Branch-free: every lane
// executes the same instructions (the eq qft_6 case keeps v; v - O is computed
// as v + (-O), which is the same IEEE operation).
QFT_RARE qc chain_c(const Eng& e, int m, int k) {
  uint64_t ops = 0;
  const int nl = m - 1;
  for (int i = 0; i < nl; ++i) {
    const int M = 1 << (m - i);
    const int qq = M >> 2;
    const uint64_t op = k < qq ? 0u : (k > qq ? 1u : 2u);
    k = op == 1 ? (M >> 1) - k : k;
    ops |= op << (2 * i);
  }
  const qc c0 = e.side0[qft_pidx(e.N / 2 - 1)];
  const qc c1 = e.side0[qft_pidx(e.N / 2)];
  const qc cm = k == 0 ? c1 : mkc(-c1.x, -c1.y);
  qc v = cadd(c0, cm);                                  // dct(2): c0 + c1 or c0 - c1
  for (int i = nl - 1; i >= 0; --i) {
    const int op = (int)((ops >> (2 * i)) & 3);
    const int mm = m - i;                             // log2 of this level's periodization
    const int j = e.r - mm;
    qc o = e.side0[cls_pos(e, j, k)];    // O_j(k) (k = M/4 reads a neighbour, unused)
    if (op == 1) o = mkc(-o.x, -o.y);
    const qc w = cadd(v, o);
    v = op == 2 ? v : w;
    k = op == 1 ? (1 << (mm - 1)) - k : k;
  }
  return v;
}

// S_M(k), k in [1, M/2-1]: same walk for the dst recursion; it stops at
// k = M/4 (S_M(M/4) = O(M/4)) or at the dst(4) base.  The walk runs over every
// level in every lane; levels below the stop only carry a dummy in-range index.
QFT_RARE qc chain_s(const Eng& e, int m, int k) {
  uint64_t ops = 0;
  const int nl = m - 2;                  // levels M = 2^m .. 8 above the dst(4) base
  int stop = nl;                         // first level (from the top) with k == M/4
  for (int i = 0; i < nl; ++i) {
    const int M = 1 << (m - i);
    const int qq = M >> 2;
    const bool hit = stop == nl && k == qq;
    stop = hit ? i : stop;
    const uint64_t op = k > qq ? 1u : 0u;
    k = (stop == nl && op == 1) ? (M >> 1) - k : k;
    ops |= op << i;
  }
  qc v = e.side1[qft_pidx(e.N / 2 - 2)];   // dst(4) base, used when no level stops
  for (int i = nl - 1; i >= 0; --i) {
    const int mm = m - i;
    const int j = e.r - mm;
    const int P = 1 << (mm - 2);
    const int kk = k & (P - 1 + P);        // keeps the dummy index inside class j's cells
    const qc o = e.side1[cls_pos(e, j, kk > 0 ? kk - 1 : 0)];
    const int op = (int)((ops >> i) & 1);
    const qc negv = mkc(-v.x, -v.y);
    const qc w = cadd(op ? negv : v, o);   // S(k) = E + O  or  S(M/2-k) = O - E
    v = i == stop ? o : (i < stop ? w : v);
    k = (i < stop && op == 1) ? (1 << (mm - 1)) - k : k;
  }
  return v;
}

// Tables of C_Mt and S_Mt (Mt = N / 2^LF) for the FINAL tasks, built level by
// level from the dct(2) / dst(4) base cases with the class outputs (eqs qft_5C,
// qft_5D, qft_6 and their DST forms), in the same operation order as the
// recursion.  tab_level_c(m) builds C_{2^m} from C_{2^(m-1)} in place
// (m = 1 builds C_2 from c(0), c(N/2)); tab_level_s(m) builds S_{2^m}
// (m = 2 is the dst(4) base).  Lanes split the k range; levels are separated
// by a (warp) barrier.
QFT_RARE void tab_level_c(const Eng& e, int m, int lane, int nl) {
  if (m == 1) {
    if (lane == 0) {
      const qc c0 = e.side0[qft_pidx(e.N / 2 - 1)], c1 = e.side0[qft_pidx(e.N / 2)];
      e.tabC[0] = cadd(c0, c1);
      e.tabC[1] = csub(c0, c1);
    }
    return;
  }
  const int M = 1 << m;
  const int j = e.r - m;
  for (int k = lane; k < M / 4; k += nl) {
    const qc E = e.tabC[k];
    const qc O = e.side0[cls_pos(e, j, k)];
    e.tabC[k] = cadd(E, O);
    e.tabC[M / 2 - k] = csub(E, O);
  }
}

QFT_RARE void tab_level_s(const Eng& e, int m, int lane, int nl) {
  if (m == 2) {
    if (lane == 0) e.tabS[1] = e.side1[qft_pidx(e.N / 2 - 2)];
    return;
  }
  const int M = 1 << m;
  const int j = e.r - m;
  for (int k = 1 + lane; k < M / 4; k += nl) {
    const qc E = e.tabS[k];
    const qc O = e.side1[cls_pos(e, j, k - 1)];
    e.tabS[k] = cadd(E, O);
    e.tabS[M / 2 - k] = csub(O, E);
  }
  if (lane == 0) e.tabS[M / 4] = e.side1[cls_pos(e, j, M / 4 - 1)];
}

// Regular frequency orbit: k0 in [1, N/2^(LF+1)).  The task builds C and S
// on the orbit {+-k0 + m N/2^LF} level by level and emits X at 2^(LF+1) bins.
template <int LF, class IO, bool IP = false>
QFT_HD void task_fin_reg(const Eng& e, const IO& io, int k0) {
  qc C[1 << LF], S[1 << LF];
  int K[1 << LF];
  if (e.tabC) {
    C[0] = e.tabC[k0];
    S[0] = e.tabS[k0];
  } else {
    C[0] = chain_c(e, e.r - LF, k0);
    S[0] = chain_s(e, e.r - LF, k0);
  }
  K[0] = k0;
#pragma unroll
  for (int l = LF; l >= 1; --l) {
    const int n = 1 << (LF - l);
    const int j = l - 1;
    const int Mh = e.N >> l;    // M/2 with M = N/2^(l-1)
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const qc oc = cls_out<IP>(e, 0, j, K[i]);
      const qc os = cls_out<IP>(e, 1, j, K[i]);
      C[n + i] = csub(C[i], oc);
      C[i] = cadd(C[i], oc);
      S[n + i] = csub(os, S[i]);
      S[i] = cadd(S[i], os);
      K[n + i] = Mh - K[i];
    }
  }
#pragma unroll
  for (int i = 0; i < (1 << LF); ++i) io.emit(K[i], C[i], S[i]);
}

// Multiples of N/2^(LF+1): one bin pair per task, full chain from periodization N.
template <class IO>
QFT_RARE void task_fin_spec(const Eng& e, const IO& io, int LF, int mi) {
  const int k = mi * (e.N >> (LF + 1));
  const qc C = chain_c(e, e.r, k);
  const qc S = (k > 0 && k < e.N / 2) ? chain_s(e, e.r, k) : mkc(0.f, 0.f);
  io.emit(k, C, S);
}

// ------------------------------------------------------------ dispatch
// IO of the node sub-plans of the large-row path (they have no F1 / FINAL tasks).
struct NoIO {
  QFT_HD void get_cd(int, qc& c, qc& d) const { c = mkc(0.f, 0.f); d = c; }
  QFT_HD qc get_c(int) const { return mkc(0.f, 0.f); }
  QFT_HD void emit(int, qc, qc) const {}
};

QFT_HD const QftSeg& find_seg(const QftRowPlan& P, int p, int tau) {
  int s = P.phase_seg0[p];
  const int e = P.phase_seg0[p + 1];
  while (s + 1 < e && P.segs[s + 1].begin <= tau) ++s;
  return P.segs[s];
}

// COMP kernels (large-row path) also run the compensated variants of the
// segments flagged in pad[2] (classes whose trees run on pairs); their register
// tiles hold at most 8 cells (the planner caps L at 3 for those segments).
template <int L1, class IO, bool COMP = false>
QFT_HD void run_plain_task(int LF, const QftSeg& sg, const Eng& e, const IO& io, int loc) {
  if (COMP && sg.pad[2]) {
    switch (sg.type) {
    case QFT_SEG_F1_BIG: task_f1_big_c<L1>(e, io, sg.cls, loc); return;
    case QFT_SEG_DIF:
#define QFT_DIFC_CASE(LL) case LL: if (sg.side) task_dif_c<LL, 1>(e, sg.cls, sg.D, loc); else task_dif_c<LL, 0>(e, sg.cls, sg.D, loc); return;
      switch (sg.L) { QFT_DIFC_CASE(1) QFT_DIFC_CASE(2) QFT_DIFC_CASE(3) default: return; }
#undef QFT_DIFC_CASE
    case QFT_SEG_LEAF:
#define QFT_LEAFC_CASE(LL) case LL: if (sg.side) task_leaf_c<LL, 1>(e, sg.cls, loc); else task_leaf_c<LL, 0>(e, sg.cls, loc); return;
      switch (sg.L) { QFT_LEAFC_CASE(1) QFT_LEAFC_CASE(2) QFT_LEAFC_CASE(3) default: return; }
#undef QFT_LEAFC_CASE
    default: break;
    }
  }
  switch (sg.type) {
  case QFT_SEG_F1_BIG: task_f1_big<L1>(e, io, sg.cls, loc); break;
  case QFT_SEG_F1_SMALL:
    switch (sg.L) {
    case 0: task_f1_small<0>(e, io, sg.cls); break;
    case 1: task_f1_small<1>(e, io, sg.cls); break;
    case 2: task_f1_small<2>(e, io, sg.cls); break;
    case 3: task_f1_small<3>(e, io, sg.cls); break;
    case 4: task_f1_small<4>(e, io, sg.cls); break;
    default: break;
    }
    break;
  case QFT_SEG_F1_BASE: task_f1_base(e, io); break;
  case QFT_SEG_DIF:
#define QFT_DIF_CASE(LL) case LL: if (sg.side) task_dif<LL, 1>(e, sg.cls, sg.D, loc); else task_dif<LL, 0>(e, sg.cls, sg.D, loc); break;
    switch (sg.L) { QFT_DIF_CASE(1) QFT_DIF_CASE(2) QFT_DIF_CASE(3) QFT_DIF_CASE(4) default: break; }
#undef QFT_DIF_CASE
    break;
  case QFT_SEG_LEAF:
#define QFT_LEAF_CASE(LL) case LL: if (sg.side) task_leaf<LL, 1>(e, sg.cls, loc); else task_leaf<LL, 0>(e, sg.cls, loc); break;
    switch (sg.L) { QFT_LEAF_CASE(1) QFT_LEAF_CASE(2) QFT_LEAF_CASE(3) QFT_LEAF_CASE(4) default: break; }
#undef QFT_LEAF_CASE
    break;
  case QFT_SEG_FIN_REG:
    switch (LF) {
    case 0: if (e.lay_nb) task_fin_reg<0, IO, true>(e, io, loc + 1); else task_fin_reg<0, IO, false>(e, io, loc + 1); break;
    case 1: if (e.lay_nb) task_fin_reg<1, IO, true>(e, io, loc + 1); else task_fin_reg<1, IO, false>(e, io, loc + 1); break;
    case 2: if (e.lay_nb) task_fin_reg<2, IO, true>(e, io, loc + 1); else task_fin_reg<2, IO, false>(e, io, loc + 1); break;
    case 3:
      if (e.lay_nb) task_fin_reg<3, IO, true>(e, io, loc + 1);
      else task_fin_reg<3, IO, false>(e, io, loc + 1);
      break;
    default: break;
    }
    break;
  case QFT_SEG_FIN_SPEC: task_fin_spec(e, io, LF, loc); break;
  default: break;
  }
}

// All of one thread's tasks of one segment: local task indices
// l = first, first + step, ... < end (task index g*count + l).  The switch on
// the task kind is taken once per segment; the loop body is specialised, so
// the class geometry is loop-invariant.
// PF (large-row kernels, scratch in global memory): each DIF task first
// prefetches the cells of the thread's next task into L2.
template <int L1, class IO, bool COMP = false, bool PF = false>
QFT_HD void run_plain_segment(int LF, const QftSeg& sg, const Eng& e, const IO& io, int first, int end,
                              int step, int g) {
  const int off = g * sg.count;
#define QFT_LOOP(CALL) for (int l = first; l < end; l += step) { const int loc = off + l; (void)loc; CALL; }
#define QFT_LOOP_PF(LL, SD, LO, CALL)                                                  \
  for (int l = first; l < end; l += step) {                                           \
    const int loc = off + l;                                                          \
    if (PF && l + step < end) task_dif_prefetch<LL, SD>(e, sg.cls, sg.D, loc + step, LO); \
    CALL;                                                                             \
  }
  if (COMP && sg.pad[2]) {
    switch (sg.type) {
    case QFT_SEG_F1_BIG: QFT_LOOP(task_f1_big_c<L1>(e, io, sg.cls, loc)) return;
    case QFT_SEG_DIF:
#define QFT_DIFC_CASE(LL) case LL: if (sg.side) { QFT_LOOP_PF(LL, 1, true, (task_dif_c<LL, 1>(e, sg.cls, sg.D, loc))) } else { QFT_LOOP_PF(LL, 0, true, (task_dif_c<LL, 0>(e, sg.cls, sg.D, loc))) } return;
      switch (sg.L) { QFT_DIFC_CASE(1) QFT_DIFC_CASE(2) QFT_DIFC_CASE(3) default: return; }
#undef QFT_DIFC_CASE
    case QFT_SEG_LEAF:
#define QFT_LEAFC_CASE(LL) case LL: if (sg.side) { QFT_LOOP((task_leaf_c<LL, 1>(e, sg.cls, loc))) } else { QFT_LOOP((task_leaf_c<LL, 0>(e, sg.cls, loc))) } return;
      switch (sg.L) { QFT_LEAFC_CASE(1) QFT_LEAFC_CASE(2) QFT_LEAFC_CASE(3) default: return; }
#undef QFT_LEAFC_CASE
    default: break;
    }
  }
  switch (sg.type) {
  case QFT_SEG_F1_BIG: QFT_LOOP(task_f1_big<L1>(e, io, sg.cls, loc)) break;
  case QFT_SEG_F1_SMALL:
    switch (sg.L) {
    case 0: QFT_LOOP(task_f1_small<0>(e, io, sg.cls)) break;
    case 1: QFT_LOOP(task_f1_small<1>(e, io, sg.cls)) break;
    case 2: QFT_LOOP(task_f1_small<2>(e, io, sg.cls)) break;
    case 3: QFT_LOOP(task_f1_small<3>(e, io, sg.cls)) break;
    case 4: QFT_LOOP(task_f1_small<4>(e, io, sg.cls)) break;
    default: break;
    }
    break;
  case QFT_SEG_F1_BASE: QFT_LOOP(task_f1_base(e, io)) break;
  case QFT_SEG_DIF:
#define QFT_DIF_CASE(LL) case LL: if (sg.side) { QFT_LOOP_PF(LL, 1, false, (task_dif<LL, 1>(e, sg.cls, sg.D, loc))) } else { QFT_LOOP_PF(LL, 0, false, (task_dif<LL, 0>(e, sg.cls, sg.D, loc))) } break;
    switch (sg.L) { QFT_DIF_CASE(1) QFT_DIF_CASE(2) QFT_DIF_CASE(3) QFT_DIF_CASE(4) default: break; }
#undef QFT_DIF_CASE
    break;
  case QFT_SEG_LEAF:
#define QFT_LEAF_CASE(LL) case LL: if (sg.side) { QFT_LOOP((task_leaf<LL, 1>(e, sg.cls, loc))) } else { QFT_LOOP((task_leaf<LL, 0>(e, sg.cls, loc))) } break;
    switch (sg.L) { QFT_LEAF_CASE(1) QFT_LEAF_CASE(2) QFT_LEAF_CASE(3) QFT_LEAF_CASE(4) default: break; }
#undef QFT_LEAF_CASE
    break;
  case QFT_SEG_FIN_REG:
    switch (LF) {
    case 0:
      if (e.lay_nb) { QFT_LOOP((task_fin_reg<0, IO, true>(e, io, loc + 1))) }
      else { QFT_LOOP((task_fin_reg<0, IO, false>(e, io, loc + 1))) }
      break;
    case 1:
      if (e.lay_nb) { QFT_LOOP((task_fin_reg<1, IO, true>(e, io, loc + 1))) }
      else { QFT_LOOP((task_fin_reg<1, IO, false>(e, io, loc + 1))) }
      break;
    case 2:
      if (e.lay_nb) { QFT_LOOP((task_fin_reg<2, IO, true>(e, io, loc + 1))) }
      else { QFT_LOOP((task_fin_reg<2, IO, false>(e, io, loc + 1))) }
      break;
    case 3:   // the large-row path's FINAL: in-place plans read the class outputs through cls_pos
      if (e.lay_nb) { QFT_LOOP((task_fin_reg<3, IO, true>(e, io, loc + 1))) }
      else { QFT_LOOP((task_fin_reg<3, IO, false>(e, io, loc + 1))) }
      break;
    default: break;
    }
    break;
  case QFT_SEG_FIN_SPEC: QFT_LOOP(task_fin_spec(e, io, LF, loc)) break;
  default: break;
  }
#undef QFT_LOOP
#undef QFT_LOOP_PF
}

QFT_HD void run_slice_read(const QftSeg& sg, const Eng& e, int loc, SliceRegs& s) {
#define QFT_SR_CASE(LL) case LL: if (sg.side) task_slice_read<LL, 1>(e, sg.cls, sg.D, loc, s); else task_slice_read<LL, 0>(e, sg.cls, sg.D, loc, s); break;
  switch (sg.L) {
    QFT_SR_CASE(1) QFT_SR_CASE(2) QFT_SR_CASE(3)
#if QFT_MAX_LB >= 4
    QFT_SR_CASE(4)
#endif
    default: break;
  }
#undef QFT_SR_CASE
}

QFT_HD void run_slice_prefetch(const QftSeg& sg, const Eng& e, int loc, bool lo) {
  switch (sg.L) {
  case 1: if (sg.side) task_slice_prefetch<1, 1>(e, sg.cls, sg.D, loc, lo); else task_slice_prefetch<1, 0>(e, sg.cls, sg.D, loc, lo); break;
  case 2: if (sg.side) task_slice_prefetch<2, 1>(e, sg.cls, sg.D, loc, lo); else task_slice_prefetch<2, 0>(e, sg.cls, sg.D, loc, lo); break;
  case 3: if (sg.side) task_slice_prefetch<3, 1>(e, sg.cls, sg.D, loc, lo); else task_slice_prefetch<3, 0>(e, sg.cls, sg.D, loc, lo); break;
  default: break;
  }
}

// MAXL: the largest L the caller's plans give compensated SLICE segments (the
// NODE kernel's sub-plans use at most 2, which keeps its registers in budget).
template <int MAXL = 3>
QFT_HD void run_slice_read_c(const QftSeg& sg, const Eng& e, int loc, SliceRegsC& s) {
  switch (sg.L) {
  case 1: if (sg.side) task_slice_read_c<1, 1>(e, sg.cls, sg.D, loc, s); else task_slice_read_c<1, 0>(e, sg.cls, sg.D, loc, s); break;
  case 2: if (sg.side) task_slice_read_c<2, 1>(e, sg.cls, sg.D, loc, s); else task_slice_read_c<2, 0>(e, sg.cls, sg.D, loc, s); break;
  case 3:
    if constexpr (MAXL >= 3) {
      if (sg.side) task_slice_read_c<3, 1>(e, sg.cls, sg.D, loc, s); else task_slice_read_c<3, 0>(e, sg.cls, sg.D, loc, s);
    }
    break;
  default: break;
  }
}

template <int MAXL = 3>
QFT_HD void run_slice_write_c(const QftSeg& sg, const Eng& e, SliceRegsC& s) {
  switch (sg.L) {
  case 1: if (sg.side) task_slice_write_c<1, 1>(e, s); else task_slice_write_c<1, 0>(e, s); break;
  case 2: if (sg.side) task_slice_write_c<2, 1>(e, s); else task_slice_write_c<2, 0>(e, s); break;
  case 3:
    if constexpr (MAXL >= 3) {
      if (sg.side) task_slice_write_c<3, 1>(e, s); else task_slice_write_c<3, 0>(e, s);
    }
    break;
  default: break;
  }
}

QFT_HD void run_slice_write(const QftSeg& sg, const Eng& e, SliceRegs& s) {
#define QFT_SW_CASE(LL) case LL: if (sg.side) task_slice_write<LL, 1>(e, s); else task_slice_write<LL, 0>(e, s); break;
  switch (sg.L) {
    QFT_SW_CASE(1) QFT_SW_CASE(2) QFT_SW_CASE(3)
#if QFT_MAX_LB >= 4
    QFT_SW_CASE(4)
#endif
    default: break;
  }
#undef QFT_SW_CASE
}

}  // namespace qft
