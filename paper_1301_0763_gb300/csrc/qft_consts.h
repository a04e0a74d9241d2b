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
