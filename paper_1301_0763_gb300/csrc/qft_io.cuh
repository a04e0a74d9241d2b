// qft_io.cuh -- what the row engine reads at its first phase and writes at its
// last one, for each transform the library offers.  All variants feed the same
// DCT-0 / DST-0 network (real coefficients, two fp32 lanes per cell):
//
//  IoC2C   complex z -> c(n) = z(n) + z(N-n), d(n) = z(n) - z(N-n) (Sec. 4.2
//          applied to both lanes); out X(k) = C(k) - i S(k), X(N-k) = C(k) + i S(k)
//          (Sec. 4.1).  Input/output lanes may be swapped (re <-> im) or
//          conjugated and the output scaled, which gives the inverse
//          IDFT(X) = swap(DFT(swap X))/N and the adjoint F^H g = conj(F conj g).
//  IoR2C   two real rows a, b in the two lanes (the cdft of Sec. 4.1 read
//          backwards: its two rdft children are computed together); out
//          X_a(k) = C_a(k) - i S_a(k), X_b(k) likewise, k in [0, N/2].
//  IoC2R   two Hermitian half spectra Y_a, Y_b: the real inverse
//          x(n) = s (A(n) - B(n)), x(N-n) = s (A(n) + B(n)) with A = DCT-0 of
//          w Re Y and B = DST-0 of w Im Y (eqs qft_0B, qft_0C; DCT-0 and DST-0
//          are symmetric matrices), w = 2 inside, 1 at k = 0, N/2.
//
// Storage types: fp32 complex (interleaved), fp16 or bf16 pairs; arithmetic is
// always fp32 (loads widen exactly, stores round to nearest even).
#pragma once
#include "qft_engine.cuh"

namespace qft {

// ------------------------------------------------------------ storage
struct StC64 {
  typedef qc elem;
  QFT_HD static qc ld(const elem* p, int64_t i) { return p[i]; }
  QFT_HD static void st(elem* p, int64_t i, qc v) { p[i] = v; }
};

#if defined(__CUDACC__) && !defined(QFT_HOST_EMULATION)
struct StC16 {
  typedef __half2 elem;
  QFT_HD static qc ld(const elem* p, int64_t i) { return __half22float2(p[i]); }
  QFT_HD static void st(elem* p, int64_t i, qc v) { p[i] = __float22half2_rn(v); }
};
struct StBF16 {
  typedef __nv_bfloat162 elem;
  QFT_HD static qc ld(const elem* p, int64_t i) { return __bfloat1622float2(p[i]); }
  QFT_HD static void st(elem* p, int64_t i, qc v) { p[i] = __float22bfloat162_rn(v); }
};
#else
// host emulation: bit-level conversions, round to nearest even
static inline float h2f_bits(uint16_t h) {
  const uint32_t s = (uint32_t)(h & 0x8000u) << 16;
  uint32_t e = (h >> 10) & 0x1f, m = h & 0x3ffu, u;
  if (e == 0) {
    if (m == 0) u = s;
    else { e = 127 - 15 + 1; while (!(m & 0x400u)) { m <<= 1; --e; } m &= 0x3ffu; u = s | (e << 23) | (m << 13); }
  } else if (e == 31) u = s | 0x7f800000u | (m << 13);
  else u = s | ((e + 127 - 15) << 23) | (m << 13);
  float f; memcpy(&f, &u, 4); return f;
}
static inline uint16_t f2h_bits(float f) {
  uint32_t u; memcpy(&u, &f, 4);
  const uint32_t s = (u >> 16) & 0x8000u;
  const int32_t e = (int32_t)((u >> 23) & 0xff) - 127 + 15;
  uint32_t m = u & 0x7fffffu;
  if (((u >> 23) & 0xff) == 0xff) return (uint16_t)(s | 0x7c00u | (m ? 0x200u : 0));
  if (e >= 31) return (uint16_t)(s | 0x7c00u);
  if (e <= 0) {
    if (e < -10) return (uint16_t)s;
    m |= 0x800000u;
    const int sh = 14 - e;
    uint32_t r = m >> sh, rem = m & ((1u << sh) - 1), half = 1u << (sh - 1);
    if (rem > half || (rem == half && (r & 1))) ++r;
    return (uint16_t)(s | r);
  }
  uint32_t r = ((uint32_t)e << 10) | (m >> 13);
  const uint32_t rem = m & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (r & 1))) ++r;
  return (uint16_t)(s | r);
}
static inline float bf2f_bits(uint16_t h) { uint32_t u = (uint32_t)h << 16; float f; memcpy(&f, &u, 4); return f; }
static inline uint16_t f2bf_bits(float f) {
  uint32_t u; memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
struct h2pair { uint16_t x, y; };
struct StC16 {
  typedef h2pair elem;
  static qc ld(const elem* p, int64_t i) { return mkc(h2f_bits(p[i].x), h2f_bits(p[i].y)); }
  static void st(elem* p, int64_t i, qc v) { h2pair o; o.x = f2h_bits(v.x); o.y = f2h_bits(v.y); p[i] = o; }
};
struct StBF16 {
  typedef h2pair elem;
  static qc ld(const elem* p, int64_t i) { return mkc(bf2f_bits(p[i].x), bf2f_bits(p[i].y)); }
  static void st(elem* p, int64_t i, qc v) { h2pair o; o.x = f2bf_bits(v.x); o.y = f2bf_bits(v.y); p[i] = o; }
};
#endif

// lane transforms applied on load / store
enum { QFT_LANE_ID = 0, QFT_LANE_SWAP = 1, QFT_LANE_CONJ = 2 };
QFT_HD qc lane_op(qc v, int op) {
  if (op == QFT_LANE_SWAP) return mkc(v.y, v.x);
  if (op == QFT_LANE_CONJ) return mkc(v.x, -v.y);
  return v;
}

// ---------------------------------------------------------------- C2C
template <class ST>
struct IoC2C {
  const typename ST::elem* in;
  typename ST::elem* out;
  int N;
  int in_op, out_op;
  float scale;      // output scale (1 or 1/N, exact powers of two)
  bool scaled;

  QFT_HD qc ld(int n) const { return lane_op(ST::ld(in, n), in_op); }
  QFT_HD void get_cd(int n, qc& c, qc& d) const {
    const qc a = ld(n), b = ld(N - n);
    c = cadd(a, b);
    d = csub(a, b);
  }
  QFT_HD qc get_c(int n) const { return ld(n); }
  QFT_HD void st(int k, qc v) const {
    v = lane_op(v, out_op);
    if (scaled) v = mkc(fmul(v.x, scale), fmul(v.y, scale));
    ST::st(out, k, v);
  }
  // X(k) = C(k) - i S(k), X(N-k) = C(k) + i S(k); -i S = (S.y, -S.x).
  QFT_HD void emit(int k, qc C, qc S) const {
    if (k == 0 || 2 * k == N) { st(k, C); return; }
    const qc t = mkc(S.y, -S.x);
    st(k, cadd(C, t));
    st(N - k, csub(C, t));
  }
};

// ---------------------------------------------------------- DCT-0 / DST-0
// The standalone real transforms of periodization N (eqs qft_0B, qft_0C) on
// two real rows (a in lane x, b in lane y; b may be absent):
//   DCT-0: c(n), n in [0, N/2]   -> C(k) = sum_n c(n) cos(2 pi n k / N), k in [0, N/2];
//   DST-0: d(n), n in [1, N/2-1] -> S(k) = sum_n d(n) sin(2 pi n k / N), k in [1, N/2-1],
//          stored at n-1 and k-1.
// The input feeds one side of the network directly (no fold); the other side
// carries zeros.
template <bool DST>
struct IoR2R {
  const float* ina;
  const float* inb;
  float* outa;
  float* outb;
  int N;
  QFT_HD qc ld(int i) const { return mkc(ina[i], inb ? inb[i] : 0.f); }
  QFT_HD void get_cd(int n, qc& c, qc& d) const {
    const qc z = mkc(0.f, 0.f);
    if (DST) { c = z; d = ld(n - 1); }
    else { c = ld(n); d = z; }
  }
  QFT_HD qc get_c(int n) const { return DST ? mkc(0.f, 0.f) : ld(n); }
  QFT_HD void emit(int k, qc C, qc S) const {
    if (DST) {
      if (k < 1 || 2 * k >= N) return;
      outa[k - 1] = S.x;
      if (outb) outb[k - 1] = S.y;
    } else {
      outa[k] = C.x;
      if (outb) outb[k] = C.y;
    }
  }
};

// ---------------------------------------------------------------- R2C
// Two real rows (a in lane x, b in lane y).  b may be absent (odd batch).
// Output row: N/2+1 complex.  Optional per-bin weight w_k * scale (used by
// the adjoint of the real inverse: w = 1 at k = 0, N/2 and 2 elsewhere),
// with the imaginary part forced to zero at k = 0 and N/2.
template <class ST>   // ST: output storage (complex)
struct IoR2C {
  const float* ina;
  const float* inb;     // may be null
  typename ST::elem* outa;
  typename ST::elem* outb;  // may be null
  int N;
  float wscale;         // 0: no weighting; else multiply by (k==0||k==N/2 ? 1 : 2) * wscale

  QFT_HD qc ld(int n) const { return mkc(ina[n], inb ? inb[n] : 0.f); }
  QFT_HD void get_cd(int n, qc& c, qc& d) const {
    const qc a = ld(n), b = ld(N - n);
    c = cadd(a, b);
    d = csub(a, b);
  }
  QFT_HD qc get_c(int n) const { return ld(n); }
  QFT_HD void emit(int k, qc C, qc S) const {
    qc xa, xb;
    if (k == 0 || 2 * k == N) { xa = mkc(C.x, 0.f); xb = mkc(C.y, 0.f); }
    else { xa = mkc(C.x, -S.x); xb = mkc(C.y, -S.y); }
    if (wscale != 0.f) {
      const float w = (k == 0 || 2 * k == N) ? wscale : fmul(2.f, wscale);
      xa = mkc(fmul(xa.x, w), fmul(xa.y, w));
      xb = mkc(fmul(xb.x, w), fmul(xb.y, w));
    }
    ST::st(outa, k, xa);
    if (outb) ST::st(outb, k, xb);
  }
};

// ---------------------------------------------------------------- C2R
template <class ST>   // ST: input storage (complex)
struct IoC2R {
  const typename ST::elem* ina;
  const typename ST::elem* inb;   // may be null
  float* outa;
  float* outb;                    // may be null
  int N;
  float wmid;    // 2 for the real inverse, 1 for the adjoint of the forward R2C
  float scale;   // 1/N for the real inverse, 1 for the adjoint

  QFT_HD qc lda(int n) const { return ST::ld(ina, n); }
  QFT_HD qc ldb(int n) const { return inb ? ST::ld(inb, n) : mkc(0.f, 0.f); }
  QFT_HD void get_cd(int n, qc& c, qc& d) const {
    const qc a = lda(n), b = ldb(n);
    c = mkc(fmul(wmid, a.x), fmul(wmid, b.x));
    d = mkc(fmul(wmid, a.y), fmul(wmid, b.y));
  }
  QFT_HD qc get_c(int n) const { return mkc(lda(n).x, ldb(n).x); }
  QFT_HD void emit(int k, qc A, qc B) const {
    if (k == 0 || 2 * k == N) {
      outa[k] = fmul(A.x, scale);
      if (outb) outb[k] = fmul(A.y, scale);
      return;
    }
    const qc lo = csub(A, B), hi = cadd(A, B);
    outa[k] = fmul(lo.x, scale);
    outa[N - k] = fmul(hi.x, scale);
    if (outb) { outb[k] = fmul(lo.y, scale); outb[N - k] = fmul(hi.y, scale); }
  }
};

}  // namespace qft

// --------------------------------------------------------- spectral filter
// Layer y = irfft(W (.) rfft(x)) on row pairs (a, b) of one channel c.  The
// spectrum stays in shared memory between the forward (R2C) and the inverse
// (C2R) transform of the pair.  Complex products are evaluated as
// re = wr*xr - wi*xi, im = wr*xi + wi*xr, each operation rounded separately.
namespace qft {

QFT_HD qc cmulc(qc w, qc x) {   // w * x
  return mkc(fsub(fmul(w.x, x.x), fmul(w.y, x.y)), fadd(fmul(w.x, x.y), fmul(w.y, x.x)));
}
QFT_HD qc cmulcj(qc w, qc x) {  // conj(w) * x
  return mkc(fadd(fmul(w.x, x.x), fmul(w.y, x.y)), fsub(fmul(w.x, x.y), fmul(w.y, x.x)));
}

// R2C of rows a, b whose spectrum goes to shared memory (spa, spb: N/2+1 cells),
// optionally weighted like the adjoint of the real inverse (wscale != 0:
// w_k * wscale, w = 1 at k = 0, N/2 and 2 elsewhere, Im = 0 at k = 0, N/2).
struct IoR2CSpec {
  const float* ina;
  const float* inb;   // may be null
  qc* spa;
  qc* spb;
  int N;
  float wscale;
  QFT_HD qc ld(int n) const { return mkc(ina[n], inb ? inb[n] : 0.f); }
  QFT_HD void get_cd(int n, qc& c, qc& d) const {
    const qc a = ld(n), b = ld(N - n);
    c = cadd(a, b);
    d = csub(a, b);
  }
  QFT_HD qc get_c(int n) const { return ld(n); }
  QFT_HD void emit(int k, qc C, qc S) const {
    qc xa, xb;
    if (k == 0 || 2 * k == N) { xa = mkc(C.x, 0.f); xb = mkc(C.y, 0.f); }
    else { xa = mkc(C.x, -S.x); xb = mkc(C.y, -S.y); }
    if (wscale != 0.f) {
      const float w = (k == 0 || 2 * k == N) ? wscale : fmul(2.f, wscale);
      xa = mkc(fmul(xa.x, w), fmul(xa.y, w));
      xb = mkc(fmul(xb.x, w), fmul(xb.y, w));
    }
    spa[k] = xa;
    spb[k] = xb;
  }
};

// R2C of rows a, b (the layer input) that accumulates the weight gradient:
// acc[k] += G_a(k) conj(X_a(k)) + G_b(k) conj(X_b(k)), G from shared memory.
struct IoR2CAccum {
  const float* ina;
  const float* inb;   // may be null
  const qc* ga;
  const qc* gb;
  qc* acc;
  int N;
  QFT_HD qc ld(int n) const { return mkc(ina[n], inb ? inb[n] : 0.f); }
  QFT_HD void get_cd(int n, qc& c, qc& d) const {
    const qc a = ld(n), b = ld(N - n);
    c = cadd(a, b);
    d = csub(a, b);
  }
  QFT_HD qc get_c(int n) const { return ld(n); }
  QFT_HD void emit(int k, qc C, qc S) const {
    qc xa, xb;
    if (k == 0 || 2 * k == N) { xa = mkc(C.x, 0.f); xb = mkc(C.y, 0.f); }
    else { xa = mkc(C.x, -S.x); xb = mkc(C.y, -S.y); }
    qc s = cadd(acc[k], cmulcj(xa, ga[k]));   // G conj(X) = conj(X) * G
    if (inb) s = cadd(s, cmulcj(xb, gb[k]));
    acc[k] = s;
  }
};

// C2R of rows a, b whose half spectra are w (.) sp (conj(w) (.) sp if conjw),
// with w the channel's weights (global), sp in shared memory.
struct IoC2RFilt {
  const qc* spa;
  const qc* spb;   // may be null
  const qc* w;
  bool conjw;
  float* outa;
  float* outb;     // may be null
  int N;
  float wmid, scale;
  QFT_HD qc ya(int n) const { return conjw ? cmulcj(w[n], spa[n]) : cmulc(w[n], spa[n]); }
  QFT_HD qc yb(int n) const { return spb ? (conjw ? cmulcj(w[n], spb[n]) : cmulc(w[n], spb[n])) : mkc(0.f, 0.f); }
  QFT_HD void get_cd(int n, qc& c, qc& d) const {
    const qc a = ya(n), b = yb(n);
    c = mkc(fmul(wmid, a.x), fmul(wmid, b.x));
    d = mkc(fmul(wmid, a.y), fmul(wmid, b.y));
  }
  QFT_HD qc get_c(int n) const { return mkc(ya(n).x, yb(n).x); }
  QFT_HD void emit(int k, qc A, qc B) const {
    if (k == 0 || 2 * k == N) {
      outa[k] = fmul(A.x, scale);
      if (outb) outb[k] = fmul(A.y, scale);
      return;
    }
    const qc lo = csub(A, B), hi = cadd(A, B);
    outa[k] = fmul(lo.x, scale);
    outa[N - k] = fmul(hi.x, scale);
    if (outb) { outb[k] = fmul(lo.y, scale); outb[N - k] = fmul(hi.y, scale); }
  }
};

}  // namespace qft
