/*
 * qft_oracle_fx.c -- plain CPU oracle of the fixed-point variant of the
 * improved QFT (Pasquini, "Improved QFT algorithm for power-of-two FFT").
 *
 * TEST INFRASTRUCTURE ONLY.  Compiled into its own shared library, loaded by
 * the test-suite, the smoke check and the benchmark's CPU baseline; the GPU
 * library never links, includes or calls it and shares no code, header or
 * constant generator with it.
 *
 * The paper names fixed-point arithmetic as the application it aims at (Sec.
 * 1 and 7) but gives no scaling rule; the rule below is this project's
 * reading.  The recursion is the one of Sec. 5 (cdft -> dct / dst ->
 * dct_ot / dct_oo / dst_ot / dst_oo), step for step as in qft_oracle.c, with
 * every value an integer:
 *
 *  - Input: complex int16 samples, value q * 2^-15 (Q15).
 *  - Block floating point.  The values of one block (a function's input or
 *    output signal, or the secant products of one dct_oo / dst_oo) are int
 *    mantissas m with one shared exponent E (value m * 2^E).  NORM shifts a
 *    block so that its largest magnitude has 29 significant bits: left
 *    shifts are exact, right shifts round half up, floor((m + 2^(s-1)) /
 *    2^s).  A block of zeros gets the exponent EZERO, which never wins an
 *    alignment.  Normalized mantissas obey |m| <= 2^29, so a sum or
 *    difference of two fits 31 bits.
 *  - Adds and subtracts (fold, mirror butterflies eqs qft_1 / qft_2,
 *    neighbour adds eqs qft_38B / qft_38C, combines eqs qft_5C-6, the CDFT
 *    combine of Sec. 4.1) are exact integer operations on mantissas of one
 *    exponent; two blocks of different exponents are first aligned to the
 *    larger one (each mantissa rounded by the same right shift).
 *  - The secant multiply (eq qft_38A) uses the constant 1/(2 cos(2 pi n/N))
 *    as a 31-bit mantissa c in [2^30, 2^31) and its own exponent x
 *    (evaluated in long double, rounded once); the product o c is exact in
 *    64 bits, and the product block is normalized once (each product by its
 *    own shift, so that all share the block exponent).
 *  - Block boundaries: the fold output (c, d), each function's output, the
 *    even-harmonic child of each mirror butterfly, and the secant products.
 *    The odd-harmonic difference o is passed to dct_oo / dst_oo unnormalized
 *    (|o| <= 2^30), and dct_oo / dst_oo return their neighbour sums
 *    unnormalized with the exponent of Y; dct_ot / dst_ot align and
 *    normalize.
 *  - Complex data go through one real-coefficient network (re and im
 *    lanes share each block exponent); the output is N int32 complex
 *    mantissas and one exponent per row (0 for a row of zeros).
 *
 * Every operation is a deterministic function of its operands and of block
 * maxima, so a parallel evaluation that takes the same blocks gets the same
 * bits in any order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FX_EZERO (-16384)
#define FX_BITS 29

typedef struct { int64_t re, im; } fxc;

static const long double FX_PI = 3.141592653589793238462643383279502884197L;

static fxc *fxalloc(long n) { return (fxc *)calloc((size_t)(n > 0 ? n : 1), sizeof(fxc)); }

static int bitlen(uint64_t v)
{
    int b = 0;
    while (v) { ++b; v >>= 1; }
    return b;
}

static uint64_t mag(int64_t v) { return v < 0 ? (uint64_t)(-v) : (uint64_t)v; }

/* v * 2^-s rounded half up; s <= 0 is an exact left shift */
static int64_t rs(int64_t v, int s)
{
    if (v == 0) return 0;
    if (s <= 0) return v * ((int64_t)1 << -s);
    if (s >= 63) return 0;                         /* |v| < 2^61 < 2^(s-1) */
    const int64_t h = (int64_t)1 << (s - 1), d = (int64_t)1 << s;
    const int64_t t = v + h;                       /* floor(t / d) */
    return t >= 0 ? t / d : -((-t + d - 1) / d);
}

static fxc rsc(fxc a, int s) { fxc r = { rs(a.re, s), rs(a.im, s) }; return r; }
static fxc fadd(fxc a, fxc b) { fxc r = { a.re + b.re, a.im + b.im }; return r; }
static fxc fsub(fxc a, fxc b) { fxc r = { a.re - b.re, a.im - b.im }; return r; }
static int keyc(fxc a)
{
    const int a1 = bitlen(mag(a.re)), a2 = bitlen(mag(a.im));
    return a1 > a2 ? a1 : a2;
}
static int maxi(int a, int b) { return a > b ? a : b; }

/* shift of a block whose largest mantissa has `bl` bits, exponent E; returns
 * the new exponent (EZERO for zeros) */
static int norm_shift(int bl, int E, int *s)
{
    if (bl == 0) { *s = 0; return FX_EZERO; }
    *s = bl - FX_BITS;
    return E + *s;
}

/* NORM of the block v[first], v[first + step], ..., v[last] of exponent E */
static int fx_norm(fxc *v, long first, long last, long step, int E)
{
    int bl = 0, s;
    for (long i = first; i <= last; i += step) bl = maxi(bl, keyc(v[i]));
    const int En = norm_shift(bl, E, &s);
    for (long i = first; i <= last; i += step) v[i] = rsc(v[i], s);
    return En;
}

/* exponent of the aligned block: the larger of the two */
static int align_to(int Ea, int Eb) { return Ea > Eb ? Ea : Eb; }

/* The constant 1/(2 cos(2 pi n / N)) as c * 2^x, c in [2^30, 2^31): the
 * cosine (the sine of the complementary angle near n = N/4, which keeps the
 * relative accuracy) in long double, the secant rounded once to 31 bits.
 * N = 8, n = 1 is cos(pi/4), the base case of dct_oo / dst_oo (the same
 * value). */
static void fx_const(long N, long n, int64_t *c, int *x)
{
    long double v;
    if (N == 8) v = cosl(FX_PI / 4);
    else {
        long double cs = (8 * n <= N) ? cosl(2 * FX_PI * (long double)n / (long double)N)
                                      : sinl(2 * FX_PI * (long double)(N / 4 - n) / (long double)N);
        v = 1.0L / (2.0L * cs);
    }
    int e;
    long double f = frexpl(v, &e);                 /* v = f 2^e, f in [0.5, 1) */
    int64_t m = (int64_t)floorl(f * 2147483648.0L + 0.5L);
    if (m == ((int64_t)1 << 31)) { m >>= 1; ++e; }
    *c = m;
    *x = e - 31;
}

/* Secant products t(n) = o(n) sec_N(n) for odd n in [1, N/4-1] (eq qft_38A),
 * normalized as one block; o has exponent Eo.  Returns the block exponent. */
static int secant_block(long N, const fxc *o, int Eo, fxc *t)
{
    int kmax = 0;                                  /* max over n of x_n + bits(p_n) + 64 */
    for (long n = 1; n < N / 4; n += 2) {
        int64_t c; int x;
        fx_const(N, n, &c, &x);
        fxc p = { o[n].re * c, o[n].im * c };
        const int bl = keyc(p);
        if (bl) kmax = maxi(kmax, x + bl + 64);
    }
    if (kmax == 0) {
        for (long n = 1; n < N / 4; n += 2) { t[n].re = 0; t[n].im = 0; }
        return FX_EZERO;
    }
    const int top = kmax - 64 - FX_BITS;           /* block exponent - Eo */
    for (long n = 1; n < N / 4; n += 2) {
        int64_t c; int x;
        fx_const(N, n, &c, &x);
        fxc p = { o[n].re * c, o[n].im * c };
        t[n] = rsc(p, top - x);
    }
    return Eo + top;
}

static int dct_fx(long N, const fxc *c, int Ec, fxc *C);
static int dct_ot_fx(long N, const fxc *s, int Es, fxc *X);
static int dct_oo_fx(long N, const fxc *s, int Es, fxc *X);
static int dst_fx(long N, const fxc *d, int Ed, fxc *S);
static int dst_ot_fx(long N, const fxc *s, int Es, fxc *X);
static int dst_oo_fx(long N, const fxc *s, int Es, fxc *X);

/* dct (Sec. 5.2.1): c[n], n in [0, N/2] -> C[k], k in [0, N/2] */
static int dct_fx(long N, const fxc *c, int Ec, fxc *C)
{
    if (N == 2) {                                  /* eq qft_0B */
        C[0] = fadd(c[0], c[1]);
        C[1] = fsub(c[0], c[1]);
        return fx_norm(C, 0, 1, 1, Ec);
    }
    fxc *e = fxalloc(N / 4 + 1), *so = fxalloc(N / 2);
    for (long m = 0; m <= N / 4; ++m) e[m] = c[2 * m];
    for (long n = 1; n < N / 2; n += 2) so[n] = c[n];
    const int Ee = fx_norm(e, 0, N / 4, 1, Ec);
    const int Eso = fx_norm(so, 1, N / 2 - 1, 2, Ec);
    fxc *E = fxalloc(N / 4 + 1), *O = fxalloc(N / 4);
    const int EE = dct_fx(N / 2, e, Ee, E);
    const int EO = dct_ot_fx(N, so, Eso, O);
    const int Ex = align_to(EE, EO);
    for (long k = 0; k < N / 4; ++k) {
        const fxc a = rsc(E[k], Ex - EE), b = rsc(O[k], Ex - EO);
        C[k] = fadd(a, b);                         /* eq qft_5C */
        C[N / 2 - k] = fsub(a, b);                 /* eq qft_5D */
    }
    C[N / 4] = rsc(E[N / 4], Ex - EE);             /* eq qft_6 */
    free(e); free(so); free(E); free(O);
    return fx_norm(C, 0, N / 2, 1, Ex);
}

/* dct_ot (Sec. 5.2.2): s[n], odd n in [1, N/2-1] -> X[k], k in [0, N/4-1] */
static int dct_ot_fx(long N, const fxc *s, int Es, fxc *X)
{
    if (N == 4) { X[0] = s[1]; return Es; }
    fxc *e = fxalloc(N / 4), *o = fxalloc(N / 4);
    for (long n = 1; n < N / 4; n += 2) {
        e[n] = fadd(s[n], s[N / 2 - n]);           /* eq qft_1 */
        o[n] = fsub(s[n], s[N / 2 - n]);           /* eq qft_2 */
    }
    const int Ee = fx_norm(e, 1, N / 4 - 1, 2, Es);
    fxc *Xe = fxalloc(N / 8), *Xo = fxalloc(N / 4);
    const int EXe = dct_ot_fx(N / 2, e, Ee, Xe);
    const int EXo = dct_oo_fx(N, o, Es, Xo);
    const int Ex = align_to(EXe, EXo);
    for (long j = 0; j < N / 8; ++j) X[2 * j] = rsc(Xe[j], Ex - EXe);     /* eqs qft_4B, qft_10 */
    for (long k = 1; k < N / 4; k += 2) X[k] = rsc(Xo[k], Ex - EXo);      /* eq qft_4B */
    free(e); free(o); free(Xe); free(Xo);
    return fx_norm(X, 0, N / 4 - 1, 1, Ex);
}

/* dct_oo (Sec. 5.2.3): o[n], odd n in [1, N/4-1] -> X[k], odd k; returns the
 * neighbour sums unnormalized, with the exponent of Y */
static int dct_oo_fx(long N, const fxc *s, int Es, fxc *X)
{
    fxc *t = fxalloc(N / 4);
    const int Et = secant_block(N, s, Es, t);      /* eq qft_38A */
    if (N == 8) {                                  /* definition: X(1) = s(1) cos(pi/4) */
        X[1] = t[1];
        free(t);
        return Et;
    }
    fxc *Y = fxalloc(N / 8);
    const int EY = dct_ot_fx(N / 2, t, Et, Y);
    for (long j = 0; j + 1 < N / 8; ++j) X[2 * j + 1] = fadd(Y[j], Y[j + 1]);   /* eq qft_38C */
    X[N / 4 - 1] = Y[N / 8 - 1];                   /* eq qft_38B */
    free(t); free(Y);
    return EY;
}

/* dst (Sec. 5.2.4): d[n], n in [1, N/2-1] -> S[k], k in [1, N/2-1] */
static int dst_fx(long N, const fxc *d, int Ed, fxc *S)
{
    if (N == 4) { S[1] = d[1]; return Ed; }        /* eq qft_0C */
    fxc *e = fxalloc(N / 4), *so = fxalloc(N / 2);
    for (long m = 1; m < N / 4; ++m) e[m] = d[2 * m];
    for (long n = 1; n < N / 2; n += 2) so[n] = d[n];
    const int Ee = fx_norm(e, 1, N / 4 - 1, 1, Ed);
    const int Eso = fx_norm(so, 1, N / 2 - 1, 2, Ed);
    fxc *E = fxalloc(N / 4), *O = fxalloc(N / 4 + 1);
    const int EE = dst_fx(N / 2, e, Ee, E);
    const int EO = dst_ot_fx(N, so, Eso, O);
    const int Ex = align_to(EE, EO);
    for (long k = 1; k < N / 4; ++k) {
        const fxc a = rsc(E[k], Ex - EE), b = rsc(O[k], Ex - EO);
        S[k] = fadd(a, b);                         /* eq qft_5C, DST form */
        S[N / 2 - k] = fsub(b, a);                 /* eq qft_5D, DST form */
    }
    S[N / 4] = rsc(O[N / 4], Ex - EO);             /* eq qft_6, DST form */
    free(e); free(so); free(E); free(O);
    return fx_norm(S, 1, N / 2 - 1, 1, Ex);
}

/* dst_ot: s[n], odd n in [1, N/2-1] -> X[k], k in [1, N/4] */
static int dst_ot_fx(long N, const fxc *s, int Es, fxc *X)
{
    if (N == 4) { X[1] = s[1]; return Es; }
    fxc *e = fxalloc(N / 4), *o = fxalloc(N / 4);
    for (long n = 1; n < N / 4; n += 2) {
        e[n] = fsub(s[n], s[N / 2 - n]);           /* eq qft_2, DST roles */
        o[n] = fadd(s[n], s[N / 2 - n]);           /* eq qft_1, DST roles */
    }
    const int Ee = fx_norm(e, 1, N / 4 - 1, 2, Es);
    fxc *Xe = fxalloc(N / 8 + 1), *Xo = fxalloc(N / 4);
    const int EXe = dst_ot_fx(N / 2, e, Ee, Xe);
    const int EXo = dst_oo_fx(N, o, Es, Xo);
    const int Ex = align_to(EXe, EXo);
    for (long j = 1; j <= N / 8; ++j) X[2 * j] = rsc(Xe[j], Ex - EXe);
    for (long k = 1; k < N / 4; k += 2) X[k] = rsc(Xo[k], Ex - EXo);
    free(e); free(o); free(Xe); free(Xo);
    return fx_norm(X, 1, N / 4, 1, Ex);
}

/* dst_oo: o[n], odd n in [1, N/4-1] -> X[k], odd k (unnormalized, exponent of Z) */
static int dst_oo_fx(long N, const fxc *s, int Es, fxc *X)
{
    fxc *t = fxalloc(N / 4);
    const int Et = secant_block(N, s, Es, t);      /* eq qft_38A, DST context */
    if (N == 8) {                                  /* definition: X(1) = s(1) cos(pi/4) */
        X[1] = t[1];
        free(t);
        return Et;
    }
    fxc *Z = fxalloc(N / 8 + 1);
    const int EZ = dst_ot_fx(N / 2, t, Et, Z);
    X[1] = Z[1];                                   /* the DST at k = 0 is zero */
    for (long j = 1; j < N / 8; ++j) X[2 * j + 1] = fadd(Z[j], Z[j + 1]);       /* eq qft_38C */
    free(t); free(Z);
    return EZ;
}

/* cdft (Sec. 4.1 / 4.2 on complex data): z int16 pairs -> X mantissas, E */
static int cdft_fx(long N, const int16_t *z, fxc *X)
{
    if (N == 2) {
        fxc a = { z[0], z[1] }, b = { z[2], z[3] };
        X[0] = fadd(a, b);
        X[1] = fsub(a, b);
        const int E = fx_norm(X, 0, 1, 1, -15);
        return E == FX_EZERO ? 0 : E;
    }
    fxc *zz = fxalloc(N);
    for (long n = 0; n < N; ++n) { zz[n].re = z[2 * n]; zz[n].im = z[2 * n + 1]; }
    fxc *c = fxalloc(N / 2 + 1), *d = fxalloc(N / 2);
    c[0] = zz[0];
    c[N / 2] = zz[N / 2];
    for (long n = 1; n < N / 2; ++n) {
        c[n] = fadd(zz[n], zz[N - n]);             /* s_dc_tt */
        d[n] = fsub(zz[n], zz[N - n]);             /* s_ds_tt */
    }
    const int Ec = fx_norm(c, 0, N / 2, 1, -15);
    const int Ed = fx_norm(d, 1, N / 2 - 1, 1, -15);
    fxc *C = fxalloc(N / 2 + 1), *S = fxalloc(N / 2);
    const int EC = dct_fx(N, c, Ec, C);
    const int ES = dst_fx(N, d, Ed, S);
    const int Ex = align_to(EC, ES);
    X[0] = rsc(C[0], Ex - EC);
    X[N / 2] = rsc(C[N / 2], Ex - EC);
    for (long k = 1; k < N / 2; ++k) {
        const fxc a = rsc(C[k], Ex - EC), b = rsc(S[k], Ex - ES);
        X[k].re = a.re + b.im;                     /* X(k) = C(k) - i S(k) */
        X[k].im = a.im - b.re;
        X[N - k].re = a.re - b.im;                 /* X(N-k) = C(k) + i S(k) */
        X[N - k].im = a.im + b.re;
    }
    const int E = fx_norm(X, 0, N - 1, 1, Ex);
    free(zz); free(c); free(d); free(C); free(S);
    return E == FX_EZERO ? 0 : E;
}

/* ============================================================ public API */

/* Fixed-point forward CDFT of each row: z int16 [batch][N][2] (Q15) ->
 * X int32 mantissas [batch][N][2] and E[batch]; value X * 2^E.  N = 2^r,
 * 2 <= N <= 2^20.  Returns 0, or -1 for bad arguments. */
int oracle_cdft_fx(long N, long batch, const int16_t *z, int32_t *X, int32_t *E, int threads)
{
    if (N < 2 || (N & (N - 1)) || N > (1L << 20) || batch < 0) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    #pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < batch; ++b) {
        fxc *out = fxalloc(N);
        E[b] = cdft_fx(N, z + 2 * N * b, out);
        for (long k = 0; k < N; ++k) {
            X[2 * (N * b + k)] = (int32_t)out[k].re;
            X[2 * (N * b + k) + 1] = (int32_t)out[k].im;
        }
        free(out);
    }
    return 0;
}

/* The fixed-point secant constant of (N, n): *c * 2^*x. */
int oracle_fx_const(long N, long n, int64_t *c, int *x)
{
    if (N < 8 || (N & (N - 1)) || n < 1 || n >= N / 4 || !(n & 1)) return -1;
    fx_const(N, n, c, x);
    return 0;
}

/* One rounding right shift (for tests of the rounding rule). */
int64_t oracle_fx_rs(int64_t v, int s) { return rs(v, s); }
