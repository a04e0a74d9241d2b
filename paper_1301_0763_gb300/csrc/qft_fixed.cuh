// qft_fixed.cuh -- the fixed-point variant of the improved QFT: complex int16
// (Q15) input, int32 block-floating-point arithmetic, int32 mantissas and one
// exponent per row out.  Written once for the sm_103a kernel and, with
// QFT_HOST_EMULATION, for a host build used only by the test-suite.
//
// Arithmetic (the paper names fixed point as its target, Sec. 1 and 7, and
// gives no scaling rule; this is the library's rule).  The values of one block
// share one exponent E (value = mantissa * 2^E).  NORM shifts a block so that
// its largest mantissa has 29 significant bits (left shifts exact, right
// shifts rounded half up: floor((m + 2^(s-1)) / 2^s)); an all-zero block gets
// the exponent kEZero, which never wins an alignment.  Adds and subtracts are
// exact on mantissas of one exponent; two blocks are aligned to the larger
// exponent first.  The secant of eq qft_38A is a 31-bit mantissa c in
// [2^30, 2^31) with its own exponent x; o * c is exact in 64 bits, and the
// products of one node form one block.  Blocks: the fold outputs (per class),
// the even-harmonic child of every mirror butterfly, the secant products of
// every odd-harmonic child, every node output (after the neighbour adds of
// eqs qft_38B/C and the interleave of eq qft_4B), every dct / dst output of the
// class chain (eqs qft_5C-6) and the CDFT output row (Sec. 4.1).  Every value
// is a function of block operands and block maxima only, so the order in which
// threads run does not change a bit.
//
// Shared-memory layout of one row (N = 2^r, 4 <= N <= 2^kMaxLog2), per side s
// (0: DCT network on c(n) = z(n) + z(N-n), 1: DST network on d(n) = z(n) -
// z(N-n)): cells V[s][0 .. N/2].  The class of 2-adic valuation j (a dct_ot /
// dst_ot of periodization M = N/2^j with P = N/2^(j+2) points; lp = log2 P)
// holds slots [off, off + P), off = N/2 - 2P, its time index n = 2^j (2i+1)
// at slot off + i.  The DCT chain's base pair c(0), c(N/2) sits at N/2 - 1,
// N/2; the DST chain's base d(N/4) is the DST class lp = 0.
//  - A node of a class tree with m cells (periodization 4m) keeps its input
//    s(n), odd n, at slot (n-1)/2; the mirror butterfly writes the
//    even-harmonic child to the first half and the secant products (the
//    odd-harmonic child, converted by eq qft_38A) to the second half, so a
//    tree is a perfect binary tree of nodes laid out in place.
//  - A node's output keeps natural frequency order: DCT X(k) at slot k, DST
//    X(k) at slot k - 1.
//  - The output of dct(4P) / dst(4P) of the class chain occupies the slots of
//    the class and of every smaller class (and the base), natural order.
// Block exponents: one int16 per tree node (heap order, class heap at 2 off),
// and one per chain output (ch[s][lp + 1]; ch[0][0] is dct(2)).
#pragma once
#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__) && !defined(QFT_HOST_EMULATION)
#define QFX_HD __host__ __device__ __forceinline__
#else
#define QFX_HD inline
#endif

namespace qfx {

constexpr int kBits = 29;          // significant bits of a normalized block's largest mantissa
constexpr int kEZero = -16384;     // exponent of an all-zero block
constexpr int kKeyOff = 64;        // offset that keeps product keys positive
constexpr int kMaxLog2 = 14;       // largest row one CTA transforms
constexpr int kInExp = -15;        // exponent of the Q15 input

struct Cell { int32_t x, y; };
struct Sec { int32_t c, x; };      // secant = c * 2^x

QFX_HD int blen64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return 64 - __clzll((long long)v);
#else
  return v ? 64 - __builtin_clzll(v) : 0;
#endif
}
QFX_HD uint64_t mag64(int64_t v) { return v < 0 ? (uint64_t)(-v) : (uint64_t)v; }
QFX_HD int imax(int a, int b) { return a > b ? a : b; }
QFX_HD int blen32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return 32 - __clz((int)v);
#else
  return v ? 32 - __builtin_clz(v) : 0;
#endif
}
// bit length of the larger magnitude of a cell (0 for a zero cell; |x|, |y| < 2^31)
QFX_HD int key(Cell a) {
  const uint32_t mx = (uint32_t)(a.x < 0 ? -a.x : a.x), my = (uint32_t)(a.y < 0 ? -a.y : a.y);
  return blen32(mx > my ? mx : my);
}
// v 2^-s rounded half up (floor((v + 2^(s-1)) / 2^s)); s <= 0: exact left shift
QFX_HD int64_t rs(int64_t v, int s) {
  if (s <= 0) return v * ((int64_t)1 << (-s));
  if (s >= 63) return 0;   // |v| < 2^61
  return (v + ((int64_t)1 << (s - 1))) >> s;
}
// rs() of an int32 mantissa in 32-bit arithmetic: with q = floor(v / 2^(s-1)),
// floor((v + 2^(s-1)) / 2^s) = floor((q + 1) / 2); shifts of 32 or more give
// q in {0, -1}, i.e. 0.  Left shifts stay below 2^31 (at most 29 places).
QFX_HD int32_t rs32(int32_t v, int s) {
  if (s <= 0) return (int32_t)((uint32_t)v << (-s));
  const int t = s - 1 < 31 ? s - 1 : 31;
  return ((v >> t) + 1) >> 1;
}
QFX_HD Cell rsc(Cell a, int s) {
  Cell r;
  r.x = rs32(a.x, s);
  r.y = rs32(a.y, s);
  return r;
}
QFX_HD Cell add(Cell a, Cell b) { Cell r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
QFX_HD Cell sub(Cell a, Cell b) { Cell r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
QFX_HD Cell zero() { Cell r; r.x = 0; r.y = 0; return r; }
// exponent after a NORM of a block whose largest mantissa has bl bits
QFX_HD int norm_exp(int bl, int E) { return bl ? E + bl - kBits : kEZero; }

// The constants of a row of length N: entry m/2 - 1 + i holds the secant
// 1/(2 cos(2 pi (2i+1) / (4m))) of slot i of a node of m cells (m = 2 ..
// N/4); the node of 2 cells (periodization 8) uses cos(pi/4), the base case
// of dct_oo / dst_oo (the same value).  Long double, the complementary-angle
// sine near the pole, rounded once to a 31-bit mantissa.  N/4 - 1 entries.
inline void fill_consts(int N, Sec* tab) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int m = 2; m <= N / 4; m *= 2) {
    const long M = 4L * m;
    for (int i = 0; i < m / 2; ++i) {
      const long n = 2L * i + 1;
      long double v;
      if (M == 8) v = cosl(pi / 4);
      else if (8 * n <= M) v = 1.0L / (2.0L * cosl(2 * pi * (long double)n / (long double)M));
      else v = 1.0L / (2.0L * sinl(2 * pi * (long double)(M / 4 - n) / (long double)M));
      int e;
      const long double f = frexpl(v, &e);
      long long c = (long long)floorl(f * 2147483648.0L + 0.5L);
      if (c == (1LL << 31)) { c >>= 1; ++e; }
      tab[m / 2 - 1 + i].c = (int32_t)c;
      tab[m / 2 - 1 + i].x = e - 31;
    }
  }
}

// ------------------------------------------------------------ row storage
// One row in shared memory: the cells of both sides (N/2 + 2 each), the
// tree-node exponents of both sides (int16, N each) and the chain exponents
// (32 ints).  The DST side first holds the staged input row (N words): the
// fold step reads all of it before it stores any cell.
QFX_HD size_t row_bytes(int N) { return 16 * (size_t)(N / 2 + 2) + 4 * (size_t)N + 128; }
// block-maximum slots of a CTA whose steps have up to `items` items: two
// alternating sets of two keys
QFX_HD int slot_count(int items) { return items >= 64 ? items / 32 : 2; }

struct Row {
  Cell* V0;            // DCT side
  Cell* V1;            // DST side
  int16_t* X0;         // tree-node exponents of the DCT side, N (class heap at 2 off)
  int16_t* X1;         // of the DST side
  int* ch;             // chain exponents: ch[16 s + lp + 1]
  const Sec* sec;      // fill_consts table
  int r, N;
};
QFX_HD Row make_row(unsigned char* base, int r, const Sec* sec) {
  const int N = 1 << r, L = N / 2 + 2;
  Row R;
  R.V0 = reinterpret_cast<Cell*>(base);
  R.V1 = R.V0 + L;
  R.X0 = reinterpret_cast<int16_t*>(R.V1 + L);
  R.X1 = R.X0 + N;
  R.ch = reinterpret_cast<int*>(R.X1 + N);
  R.sec = sec;
  R.r = r;
  R.N = N;
  return R;
}
QFX_HD Cell* side(const Row& R, int s) { return s ? R.V1 : R.V0; }
QFX_HD int16_t* exps(const Row& R, int s) { return s ? R.X1 : R.X0; }
// the staged input row (over the DST side)
QFX_HD uint32_t* staged(const Row& R) { return reinterpret_cast<uint32_t*>(R.V1); }

QFX_HD Cell load_z(const uint32_t* z, int n) {
  const uint32_t w = z[n];
  Cell c;
  c.x = (int32_t)(int16_t)(uint16_t)(w & 0xffffu);
  c.y = (int32_t)(int16_t)(uint16_t)(w >> 16);
  return c;
}

// Every step: items w in [0, items of the row).  An item's eval function
// reads its operands and gives its (unnormalized) values, its block key(s)
// and its block size seg (a power of two; 0: no work); after the CTA barrier
// its store function writes the values, shifted by the block maxima, in place.
struct Val {
  Cell a, b, c, d;     // values (c, d: the forward step's second pair)
  int k1, k2;          // block keys
  int seg;
  int ex;              // exponent the values are aligned to (backward, final)
};
QFX_HD void val_none(Val& v) {
  v.a = zero(); v.b = zero(); v.c = zero(); v.d = zero();
  v.k1 = 0; v.k2 = 0; v.seg = 0; v.ex = 0;
}

// ---------------------------------------------------------------- fold step
// Items w in [0, N/2): side s = w / (N/4), slots 2 w1 and 2 w1 + 1 of that
// side: the fold values c(n) or d(n) of those slots, one block per class (a
// NORM of the fold output followed by the lossless NORMs of the even/odd
// separations of Sec. 3.1 is one NORM per class).  A class of P >= 2 slots
// holds P/2 items; the last item of a side holds the class of one slot
// (c(N/4), or the DST base d(N/4)) and nothing else (slot N/2 - 1 is the DCT
// base, done by fold_base).  Reads the staged input row z.
struct FoldDec { int s, w1, lp, P, off, i; };
QFX_HD bool fold_dec(const Row& R, int w, FoldDec& d) {
  const int H = R.N / 2, Q4 = R.N / 4;
  d.s = w >= Q4;
  d.w1 = 2 * (w - d.s * Q4);   // the item's first slot
  d.lp = blen32((uint32_t)(H - 1 - d.w1)) - 1;
  d.P = 1 << d.lp;
  d.off = H - 2 * d.P;
  d.i = d.w1 - d.off;
  return true;
}
QFX_HD Cell fold_value(const Row& R, const uint32_t* z, int s, int lp, int i) {
  const int n = (2 * i + 1) << (R.r - 2 - lp);
  const Cell a = load_z(z, n), b = load_z(z, R.N - n);
  return s ? sub(a, b) : add(a, b);
}
QFX_HD void fold_eval(const Row& R, const uint32_t* z, int w, Val& v) {
  val_none(v);
  FoldDec d;
  fold_dec(R, w, d);
  v.a = fold_value(R, z, d.s, d.lp, d.i);
  if (d.P >= 2) v.b = fold_value(R, z, d.s, d.lp, d.i + 1);
  v.k1 = imax(key(v.a), key(v.b));
  v.seg = d.P >= 2 ? d.P >> 1 : 1;
}
QFX_HD void fold_store(const Row& R, int w, const Val& v, int bl) {
  FoldDec d;
  fold_dec(R, w, d);
  Cell* V = side(R, d.s);
  V[d.w1] = rsc(v.a, bl - kBits);
  if (d.P >= 2) V[d.w1 + 1] = rsc(v.b, bl - kBits);
  if (d.i == 0) {
    const int E = norm_exp(bl, kInExp);
    exps(R, d.s)[2 * d.off] = (int16_t)E;
    if (d.s == 1 && d.lp == 0) R.ch[16 + 1] = E;   // dst(4) of the chain: its input d(N/4)
  }
}
// The DCT chain's base: c(0), c(N/2) normalized, then dct(2) (eq qft_0B).
// Reads z(0), z(N/2) before the fold's barrier; the two cells it stores are
// on the DCT side, away from the staged row.
QFX_HD void fold_base(const Row& R, const uint32_t* z) {
  const int H = R.N / 2;
  Cell b0 = load_z(z, 0), b1 = load_z(z, H);
  const int bl = imax(key(b0), key(b1));
  const int E = norm_exp(bl, kInExp);
  b0 = rsc(b0, bl - kBits);
  b1 = rsc(b1, bl - kBits);
  const Cell c0 = add(b0, b1), c1 = sub(b0, b1);
  const int bl2 = imax(key(c0), key(c1));
  R.V0[H - 1] = rsc(c0, bl2 - kBits);
  R.V0[H] = rsc(c1, bl2 - kBits);
  R.ch[0] = norm_exp(bl2, E);
}

// ------------------------------------------------------- forward step (depth d)
// Items w in [0, N/4): side s = w / (N/8); item w1 takes the mirror pairs
// p = 2 w1 and 2 w1 + 1 of the side's pair layout (class lp at pairs
// [N/4 - P, N/4 - P/2), one pair (i, m-1-i), i < m/2, per pair of each of its
// 2^d nodes of m = P / 2^d cells): the butterflies of eqs qft_1, qft_2 (DST
// roles swapped, Sec. 3.2) and the secant products of the odd-harmonic half
// (eq qft_38A).
//  - m >= 4: both pairs (i, i+1) are in one node; keys: k1 for the
//    even-harmonic child, k2 for the product block (x + bits + kKeyOff); the
//    values: children a, c (pairs i, i+1) and differences b, d before the secant.
//  - m = 2: the pairs are the only pairs of nodes q and q+1 (the second pair
//    exists if lp >= 2): every child is a block of one cell, normalized by its
//    own key (seg 1, no reduction).
struct FwdDec { int s, lp, off, q, i, m, base; bool two; };
QFX_HD bool fwd_dec(const Row& R, int dep, int w, FwdDec& d) {
  const int Q8 = R.N / 8, Q4 = R.N / 4;
  d.s = w >= Q8;
  const int p = 2 * (w - d.s * Q8);
  d.lp = blen32((uint32_t)(Q4 - 1 - p));
  if (d.lp < dep + 1) return false;
  const int P = 1 << d.lp;
  d.off = R.N / 2 - 2 * P;
  const int w2 = p - (Q4 - P);
  const int hb = d.lp - dep - 1;
  d.q = w2 >> hb;
  d.i = w2 & ((1 << hb) - 1);
  d.m = 2 << hb;
  d.base = d.off + d.q * d.m;
  d.two = hb >= 1 || d.lp >= 2;
  return true;
}
// key of an odd-harmonic difference o times the secant c (0 for zero)
QFX_HD int prod_key(Cell o, Sec c) {
  const int64_t px = (int64_t)o.x * c.c, py = (int64_t)o.y * c.c;
  const uint64_t mx = mag64(px), my = mag64(py);
  const int bl = blen64(mx > my ? mx : my);
  return bl ? c.x + bl + kKeyOff : 0;
}
// the product block's member o c shifted to the block whose key is k2
QFX_HD Cell prod_val(Cell o, Sec c, int k2) {
  Cell t = zero();
  if (k2) {
    const int top = k2 - kKeyOff - kBits;
    t.x = (int32_t)rs((int64_t)o.x * c.c, top - c.x);
    t.y = (int32_t)rs((int64_t)o.y * c.c, top - c.x);
  }
  return t;
}
QFX_HD void butterfly(int s, Cell a, Cell b, Cell& e, Cell& o) {
  e = s ? sub(a, b) : add(a, b);   // even-harmonic child
  o = s ? add(a, b) : sub(a, b);   // odd-harmonic child, before the secant
}
QFX_HD void fwd_eval(const Row& R, int dep, int w, Val& v) {
  val_none(v);
  FwdDec d;
  if (!fwd_dec(R, dep, w, d)) return;
  const Cell* V = side(R, d.s);
  if (d.m >= 4) {
    butterfly(d.s, V[d.base + d.i], V[d.base + d.m - 1 - d.i], v.a, v.b);
    butterfly(d.s, V[d.base + d.i + 1], V[d.base + d.m - 2 - d.i], v.c, v.d);
    const Sec* c = R.sec + (d.m >> 1) - 1 + d.i;
    v.k1 = imax(key(v.a), key(v.c));
    v.k2 = imax(prod_key(v.b, c[0]), prod_key(v.d, c[1]));
    v.seg = d.m >> 2;
  } else {
    butterfly(d.s, V[d.base], V[d.base + 1], v.a, v.b);
    if (d.two) butterfly(d.s, V[d.base + 2], V[d.base + 3], v.c, v.d);
    v.seg = 1;
  }
}
QFX_HD void fwd_store(const Row& R, int dep, int w, const Val& v, int k1, int k2) {
  FwdDec d;
  fwd_dec(R, dep, w, d);
  Cell* V = side(R, d.s);
  int16_t* X = exps(R, d.s);
  const int h0 = 2 * d.off + (1 << dep) - 1, h1 = 2 * d.off + (2 << dep) - 1;   // heap bases: depth dep, dep + 1
  if (d.m >= 4) {
    const Sec* c = R.sec + (d.m >> 1) - 1 + d.i;
    Cell* e = V + d.base + d.i;                  // i even: both pairs 16-byte aligned
    Cell* t = V + d.base + (d.m >> 1) + d.i;
    e[0] = rsc(v.a, k1 - kBits);
    e[1] = rsc(v.c, k1 - kBits);
    t[0] = prod_val(v.b, c[0], k2);
    t[1] = prod_val(v.d, c[1], k2);
    if (d.i == 0) {
      const int Ein = X[h0 + d.q];
      X[h1 + 2 * d.q] = (int16_t)norm_exp(k1, Ein);
      X[h1 + 2 * d.q + 1] = (int16_t)(k2 ? Ein + k2 - kKeyOff - kBits : kEZero);
    }
    return;
  }
  // nodes of two cells: the secant of a node of 2 cells (periodization 8) is entry 0
  const Sec c = R.sec[0];
  for (int k = 0; k < (d.two ? 2 : 1); ++k) {
    const Cell e = k ? v.c : v.a, o = k ? v.d : v.b;
    const int q = d.q + k, ke = key(e), kt = prod_key(o, c);
    const int Ein = X[h0 + q];
    V[d.base + 2 * k] = rsc(e, ke - kBits);
    V[d.base + 2 * k + 1] = prod_val(o, c, kt);
    X[h1 + 2 * q] = (int16_t)norm_exp(ke, Ein);
    X[h1 + 2 * q + 1] = (int16_t)(kt ? Ein + kt - kKeyOff - kBits : kEZero);
  }
}

// ----------------------------------------------------- backward step (height h)
// Items w in [0, N/2): side s = w / (N/4), then, in the half-resolution layout
// of the forward step (class lp at [N/4 - P, N/4 - P/2)), u = N/4 - 1 - w1:
//  - u >= 2^(h-1): a tree item of class lp = bits(u) >= h: output cells 2j and
//    2j + 1 of a node of m = 2^h cells at depth lp - h, from its children
//    (eqs qft_4B, qft_38B, qft_38C; DST forms of Sec. 5);
//  - u < 2^(h-1): item t of the class chain's combine of class c = h - 1,
//    dct(4P) (or dst(4P), c >= 1), P = 2^c: outputs t and 2P - t (eqs qft_5C,
//    qft_5D; DCT item 0 also the middle output, eq qft_6).  The chain's P items
//    take the half-resolution slots of class c and of every smaller class.
struct BwdDec { int s, lp, P, off, w2; };
QFX_HD int bwd_dec(const Row& R, int h, int w, BwdDec& d) {
  const int Q4 = R.N / 4;
  d.s = w >= Q4;
  const int w1 = w - d.s * Q4;
  const int u = Q4 - 1 - w1;
  if (u >= (1 << (h - 1))) {                                 // tree item
    d.lp = blen32((uint32_t)u);
    d.P = 1 << d.lp;
    d.off = R.N / 2 - 2 * d.P;
    d.w2 = w1 - (Q4 - d.P);
    return 1;
  }
  d.lp = h - 1;                                              // chain item
  if (d.s == 1 && d.lp == 0) return 0;                       // dst(4) is its input
  d.P = 1 << d.lp;
  d.off = R.N / 2 - 2 * d.P;
  d.w2 = w1 - (Q4 - d.P);
  return 2;
}
QFX_HD void bwd_eval(const Row& R, int h, int w, Val& v) {
  val_none(v);
  BwdDec d;
  const int kind = bwd_dec(R, h, w, d);
  if (!kind) return;
  const Cell* V = side(R, d.s);
  const int16_t* X = exps(R, d.s);
  if (kind == 1) {
    const int dep = d.lp - h, hm = h - 1, q = d.w2 >> hm, j = d.w2 & ((1 << hm) - 1);
    const int hc = 2 * d.off + (2 << dep) - 1 + 2 * q;
    const int Ee = X[hc], Ey = X[hc + 1];
    const int Ex = imax(Ee, Ey);
    const int m = 1 << h, base = d.off + q * m, half = base + (m >> 1);
    if (d.s == 0) {            // DCT: X(2j) = E(j); X(2j+1) = Y(j) + Y(j+1), the last Y(m/2-1)
      v.a = rsc(V[base + j], Ex - Ee);
      v.b = rsc(j + 1 < (m >> 1) ? add(V[half + j], V[half + j + 1]) : V[half + j], Ex - Ey);
    } else {                   // DST, slots 2j, 2j+1 hold X(2j+1), X(2j+2): X(1) = Z(1); X(2j+1) = Z(j) + Z(j+1); X(2j+2) = E(j+1)
      v.a = rsc(j == 0 ? V[half] : add(V[half + j - 1], V[half + j]), Ex - Ey);
      v.b = rsc(V[base + j], Ex - Ee);
    }
    v.k1 = imax(key(v.a), key(v.b));
    v.seg = m >> 1;
    v.ex = Ex;
    return;
  }
  const int EO = X[2 * d.off], EE = R.ch[16 * d.s + d.lp];
  const int Ex = imax(EE, EO);
  const int t = d.w2, P = d.P, off = d.off;
  if (d.s == 0) {              // C(t) = E(t) + O(t), C(2P-t) = E(t) - O(t), C(P) = E(P)
    const Cell e = rsc(V[off + P + t], Ex - EE), o = rsc(V[off + t], Ex - EO);
    v.a = add(e, o);
    v.b = sub(e, o);
    v.k1 = imax(key(v.a), key(v.b));
    if (t == 0) v.k1 = imax(v.k1, key(rsc(V[off + 2 * P], Ex - EE)));
  } else if (t == 0) {         // S(P) = O(P)
    v.a = rsc(V[off + P - 1], Ex - EO);
    v.k1 = key(v.a);
  } else {                     // S(t) = E(t) + O(t), S(2P-t) = O(t) - E(t)
    const Cell e = rsc(V[off + P + t - 1], Ex - EE), o = rsc(V[off + t - 1], Ex - EO);
    v.a = add(e, o);
    v.b = sub(o, e);
    v.k1 = imax(key(v.a), key(v.b));
  }
  v.seg = P;
  v.ex = Ex;
}
QFX_HD void bwd_store(const Row& R, int h, int w, const Val& v, int bl) {
  BwdDec d;
  const int kind = bwd_dec(R, h, w, d);
  Cell* V = side(R, d.s);
  const int sh = bl - kBits;
  if (kind == 1) {
    const int hm = h - 1, q = d.w2 >> hm, j = d.w2 & ((1 << hm) - 1);
    Cell* o = V + d.off + (q << h) + 2 * j;   // an even slot: the pair is 16-byte aligned
    o[0] = rsc(v.a, sh);
    o[1] = rsc(v.b, sh);
    if (j == 0) exps(R, d.s)[2 * d.off + (1 << (d.lp - h)) - 1 + q] = (int16_t)norm_exp(bl, v.ex);
    return;
  }
  const int t = d.w2, P = d.P, off = d.off;
  if (d.s == 0) {
    if (t == 0) {              // E(P), read before C(2P) replaces it; only this item touches both cells
      const Cell mid = rsc(V[off + 2 * P], v.ex - R.ch[d.lp]);
      V[off + P] = rsc(mid, sh);
      R.ch[d.lp + 1] = norm_exp(bl, v.ex);
    }
    V[off + t] = rsc(v.a, sh);
    V[off + 2 * P - t] = rsc(v.b, sh);
  } else if (t == 0) {
    V[off + P - 1] = rsc(v.a, sh);
    R.ch[16 + d.lp + 1] = norm_exp(bl, v.ex);
  } else {
    V[off + t - 1] = rsc(v.a, sh);
    V[off + 2 * P - t - 1] = rsc(v.b, sh);
  }
}

// ------------------------------------------------------------- final step
// Items k in [0, N/2): X(k) = C(k) - i S(k), X(N-k) = C(k) + i S(k) (Sec.
// 4.1 on complex data), item 0: X(0) = C(0), X(N/2) = C(N/2); one block.
QFX_HD void fin_eval(const Row& R, int k, Val& v) {
  const int EC = R.ch[R.r - 1], ES = R.ch[16 + R.r - 1];
  const int Ex = imax(EC, ES);
  if (k == 0) {
    v.a = rsc(R.V0[0], Ex - EC);
    v.b = rsc(R.V0[R.N / 2], Ex - EC);
  } else {
    const Cell a = rsc(R.V0[k], Ex - EC), b = rsc(R.V1[k - 1], Ex - ES);
    v.a.x = a.x + b.y; v.a.y = a.y - b.x;
    v.b.x = a.x - b.y; v.b.y = a.y + b.x;
  }
  v.k1 = imax(key(v.a), key(v.b));
  v.k2 = 0;
  v.seg = R.N / 2;
  v.ex = Ex;
}
// out: the row's N cells; *E the row exponent (0 for a row of zeros)
QFX_HD void fin_store(const Row& R, int k, const Val& v, int bl, Cell* out, int* E) {
  out[k] = rsc(v.a, bl - kBits);
  out[k == 0 ? R.N / 2 : R.N - k] = rsc(v.b, bl - kBits);
  if (k == 0) *E = bl ? v.ex + bl - kBits : 0;
}

// N = 2: X(0) = z(0) + z(1), X(1) = z(0) - z(1), one block.
QFX_HD void row_n2(const uint32_t* z, Cell* out, int* E) {
  const Cell a = load_z(z, 0), b = load_z(z, 1);
  const Cell s = add(a, b), t = sub(a, b);
  const int bl = imax(key(s), key(t));
  out[0] = rsc(s, bl - kBits);
  out[1] = rsc(t, bl - kBits);
  *E = bl ? kInExp + bl - kBits : 0;
}

}  // namespace qfx
