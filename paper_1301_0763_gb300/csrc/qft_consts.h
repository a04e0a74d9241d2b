// qft_consts.h -- the library's trigonometric-constant table (host code).
//
// The improved QFT needs only the secants 1/(2 cos(2 pi m / N)), m in
// [1, N/4) (eq qft_38A; Sec. 6.1: N/4 constants including cos(pi/4), whose
// value is the entry m = N/8).  They are generated once per plan in FP64 and
// rounded once to FP32.  For m > N/8 the cosine is evaluated as the sine of
// the complementary small angle 2 pi (N/4 - m)/N, so that the FP64 value keeps
// full relative accuracy where the secant is large (near m = N/4).
// A table built for N serves every N' = N / 2^s: entry m of N' is entry
// m 2^s of N (the same angle).
#pragma once
#include <math.h>
#include <stdint.h>

// 1/(2 cos(2 pi m / M)) for 0 < m < M/4, evaluated in FP64 with the
// complementary-angle form near m = M/4, rounded once to FP32.
static inline float qft_secant(int64_t m, int64_t M) {
  const double two_pi = 6.283185307179586476925286766559;
  double c;
  if (8 * m <= M) c = cos(two_pi * (double)m / (double)M);
  else c = sin(two_pi * (double)(M / 4 - m) / (double)M);
  return (float)(1.0 / (2.0 * c));
}

// The secants in the order the row engine uses them.  A node of 2^b cells
// (own time index n = 2c+1, periodization M = 2^(b+2)) multiplies the
// odd-harmonic half of its mirror butterflies by 1/(2 cos(2 pi n / M))
// (eq qft_38A); the engine stores cells in Gray order, so the butterfly whose
// lower element sits in node slot g (g < 2^(b-1)) needs own cell
// c = invgray(g).  Entry 2^(b-1) + g of this table holds that secant, for
// b = 1 .. rmax-2; entry 0 is unused.  The value depends only on (b, g), so
// the table built for 2^rmax serves every N <= 2^rmax through its first N/4
// entries, and it holds exactly the N/4 - 1 secant constants of Sec. 6.1
// (b = 1 gives 1/(2 cos(pi/4)) = cos(pi/4)).
static inline void qft_fill_gray_secants(int rmax, float* gsec /* 2^(rmax-2) entries */) {
  gsec[0] = 0.f;
  for (int b = 1; b <= rmax - 2; ++b) {
    const int64_t M = (int64_t)1 << (b + 2);
    for (int64_t g = 0; g < ((int64_t)1 << (b - 1)); ++g) {
      uint64_t c = (uint64_t)g;
      c ^= c >> 1; c ^= c >> 2; c ^= c >> 4; c ^= c >> 8; c ^= c >> 16; c ^= c >> 32;
      gsec[((int64_t)1 << (b - 1)) + g] = qft_secant(2 * (int64_t)c + 1, M);
    }
  }
}

static inline void qft_fill_secants(int64_t N, float* sec /* N/4 + 1 entries */) {
  const double two_pi = 6.283185307179586476925286766559;
  sec[0] = 0.f;
  for (int64_t m = 1; m < N / 4; ++m) {
    double c;
    if (8 * m <= N) c = cos(two_pi * (double)m / (double)N);
    else c = sin(two_pi * (double)(N / 4 - m) / (double)N);
    sec[m] = (float)(1.0 / (2.0 * c));
  }
  if (N >= 4) sec[N / 4] = 0.f;
}
