/*
 * qft_oracle.c -- plain, slow CPU oracle of the improved QFT
 * (Pasquini, "Improved QFT algorithm for power-of-two FFT").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared
 * library that only the test-suite, the smoke check and the benchmark's CPU
 * baseline load.  The GPU library never links, includes or calls it, and it
 * shares no code, header, table or constant generator with the GPU library.
 *
 * What it computes.  The length-N = 2^r DFT (eq qft_0A) by the eight
 * recursive functions of Sec. 5 (cdft, rdft, dct, dct_ot, dct_oo, dst,
 * dst_ot, dst_oo), in FP64, in the paper's order and notation.  A second
 * section holds the paper's comparison algorithm, the classical QFT of Sec. 4
 * (cdft_cla, rdft_cla, dct_cla, dct_to_cla, dst_cla, dst_to_cla), and a
 * long-double reference DFT for the error measure of eq qft_44.  Every
 * function works on arrays indexed by the paper's own time index n or
 * frequency index k (so s[n] is s(n) of the text; unused cells stay zero),
 * which keeps each line checkable against the equations by eye.
 *
 * Counting.  Every real addition/subtraction and every real multiplication
 * of the algorithm goes through ADD/SUB/MUL, which count them (per thread),
 * so that the computational-cost tables (Tab. 2-5) can be reproduced.
 * Copies and sign changes are free, as in the paper's cost model.
 *
 * Constants.  As in Sec. 6.3, every trigonometric constant is evaluated in
 * extended precision (long double) and rounded once to double.  Which
 * constants a transform touched is recorded, for the constant-count claim
 * of Sec. 6.1.
 *
 * Readings of the paper used here (it is silent or garbled at these points):
 *  - Sec. 5, dct function: the even-time child is a DCT-context signal
 *    (s_dc_et); the text prints "s_ds_et".
 *  - eq qft_38A: only the odd n of s_dc_oo exist, so the secant multiply runs
 *    over odd n in [1, N/4-1].
 *  - eq qft_38B: DCT[s_dc_oe](N/4) is zero for odd-n signals; the last odd
 *    output is X(N/4-1) = Y(N/8-1), i.e. the k+1 term of eq qft_38C vanishes.
 *  - dst_oo (Sec. 5.2.4): the special case is X(1) = Z(1), since the
 *    even-harmonic DST at k = 0 is zero.
 *  - DST form of the even/odd time separation (Sec. 3.1, "swapping s_en and
 *    s_on"): S(k) = E(k) + O(k), S(N/2-k) = O(k) - E(k), S(N/4) = O(N/4).
 *  - DST form of the even/odd harmonic separation (Sec. 3.2): the even-k
 *    child takes the difference s(n) - s(N/2-n), the odd-k child the sum.
 *  - "log" in Tab. 2 is log2.
 *  - Inverse (the paper is silent): IDFT(X) = swap(DFT(swap(X)))/N where swap
 *    exchanges real and imaginary parts.  Forward is unscaled (eq qft_0A).
 *  - Real inverse: x(n) = (A(n) - B(n))/N, x(N-n) = (A(n) + B(n))/N, with
 *    A = DCT-0 of a(k) = w_k Re Y(k) and B = DST-0 of b(k) = 2 Im Y(k),
 *    w_k = 1 at k = 0, N/2 and 2 elsewhere (eqs qft_0B, qft_0C applied to
 *    the Hermitian extension of Y).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

static const long double PI_L = 3.141592653589793238462643383279502884197L;

/* ---------------------------------------------------------------- counters */
static _Thread_local long long t_adds, t_muls;

static inline real ADD(real a, real b) { t_adds++; return a + b; }
static inline real SUB(real a, real b) { t_adds++; return a - b; }
static inline real MUL(real a, real b) { t_muls++; return a * b; }

/* -------------------------------------------------------------- constants */
/* Per root transform: the secant table 1/(2 cos(2 pi m / Nroot)), m in
 * [1, Nroot/4), computed in long double and rounded once (Sec. 6.3), and the
 * base-case constant cos(pi/4) = sin(pi/4) used by dct_oo/dst_oo at N = 8. */
typedef struct {
    long Nroot;
    real *sec;                 /* sec[m], m in [0, Nroot/4]; sec[0] unused */
    real cos_pi_4;
    unsigned char *used;       /* used[m] = 1 if secant angle m was used     */
    int cos_pi_4_used;
} consts_t;

static _Thread_local consts_t *t_c;

static consts_t *consts_make(long Nroot)
{
    consts_t *c = (consts_t *)calloc(1, sizeof(consts_t));
    c->Nroot = Nroot;
    long q = Nroot / 4 + 1;
    c->sec = (real *)calloc((size_t)q, sizeof(real));
    c->used = (unsigned char *)calloc((size_t)q, 1);
    for (long m = 1; m < Nroot / 4; ++m) {
        long double a = 2.0L * PI_L * (long double)m / (long double)Nroot;
        c->sec[m] = (real)(1.0L / (2.0L * cosl(a)));
    }
    c->cos_pi_4 = (real)cosl(PI_L / 4.0L);
    return c;
}

static void consts_free(consts_t *c)
{
    if (!c) return;
    free(c->sec);
    free(c->used);
    free(c);
}

/* 1/(2 cos(theta n)) with theta = 2 pi / N (eq qft_38A), looked up in the
 * root table: angle 2 pi n / N = 2 pi (n Nroot/N) / Nroot. */
static real secant(long N, long n)
{
    long m = n * (t_c->Nroot / N);
    t_c->used[m] = 1;
    return t_c->sec[m];
}

static real cos_pi_4(void)
{
    t_c->cos_pi_4_used = 1;
    return t_c->cos_pi_4;
}

static real *zalloc(long n) { return (real *)calloc((size_t)(n > 0 ? n : 1), sizeof(real)); }

/* ------------------------------------------------- the eight functions */
static void dct(long N, const real *c, real *C);
static void dct_ot(long N, const real *s, real *X);
static void dct_oo(long N, const real *s, real *X);
static void dst(long N, const real *d, real *S);
static void dst_ot(long N, const real *s, real *X);
static void dst_oo(long N, const real *s, real *X);
#ifdef ORACLE_COMPENSATED
static int class_compensated(long M);
static void dct_ot_comp(long N, const real *s, real *X);
static void dst_ot_comp(long N, const real *s, real *X);
#endif

/* dct: input s_dc_tt, c[n] for n in [0, N/2]; output C[k], k in [0, N/2].
 * Sec. 5.2.1: even/odd time separation (Sec. 3.1, eqs qft_5A/5B), then the
 * even child is halved in time (Sec. 3.4, eq qft_12) into a DCT of
 * periodization N/2; the odd child is an s_dc_ot handled by dct_ot.
 * Backward: eqs qft_5C, qft_5D, qft_6 (with eq qft_13 for the halved child). */
static void dct(long N, const real *c, real *C)
{
    if (N == 2) {                          /* DCT-0 definition, eq qft_0B */
        C[0] = ADD(c[0], c[1]);
        C[1] = SUB(c[0], c[1]);
        return;
    }
    real *e = zalloc(N / 4 + 1);           /* s_A_dc_tt(m) = c(2m), m in [0,N/4] */
    real *so = zalloc(N / 2);              /* s_dc_ot(n) = c(n), odd n          */
    for (long m = 0; m <= N / 4; ++m) e[m] = c[2 * m];
    for (long n = 1; n < N / 2; n += 2) so[n] = c[n];
    real *E = zalloc(N / 4 + 1);           /* DCT[s_A_dc_tt](k), k in [0,N/4]   */
    real *O = zalloc(N / 4);               /* DCT[s_dc_ot](k),   k in [0,N/4-1] */
    dct(N / 2, e, E);
#ifdef ORACLE_COMPENSATED
    if (class_compensated(N)) dct_ot_comp(N, so, O); else
#endif
    dct_ot(N, so, O);
    for (long k = 0; k < N / 4; ++k) {
        C[k] = ADD(E[k], O[k]);            /* eq qft_5C */
        C[N / 2 - k] = SUB(E[k], O[k]);    /* eq qft_5D */
    }
    C[N / 4] = E[N / 4];                   /* eq qft_6 */
    free(e); free(so); free(E); free(O);
}

/* dct_ot: input s_dc_ot, s[n] for odd n in [1, N/2-1]; output X[k], k in
 * [0, N/4-1].  Sec. 5.2.2: even/odd harmonic separation (Sec. 3.2, eqs
 * qft_1, qft_2) into s_dc_oe and s_dc_oo; s_dc_oe is halved in frequency
 * (Sec. 3.3, eqs qft_9/qft_10) into a dct_ot of periodization N/2.
 * Backward: eq qft_4B. */
static void dct_ot(long N, const real *s, real *X)
{
    if (N == 4) {                          /* definition: only n = 1, k = 0 */
        X[0] = s[1];
        return;
    }
    real *e = zalloc(N / 4);               /* s_dc_oe(n), odd n in [1,N/4-1] */
    real *o = zalloc(N / 4);               /* s_dc_oo(n), odd n in [1,N/4-1] */
    for (long n = 1; n < N / 4; n += 2) {
        e[n] = ADD(s[n], s[N / 2 - n]);    /* eq qft_1 */
        o[n] = SUB(s[n], s[N / 2 - n]);    /* eq qft_2 */
    }
    real *Xe = zalloc(N / 8);              /* DCT[s_A_dc_ot](j), j in [0,N/8-1] */
    real *Xo = zalloc(N / 4);              /* DCT[s_dc_oo](k),  odd k          */
    dct_ot(N / 2, e, Xe);
    dct_oo(N, o, Xo);
    for (long j = 0; j < N / 8; ++j) X[2 * j] = Xe[j];      /* eqs qft_4B, qft_10 */
    for (long k = 1; k < N / 4; k += 2) X[k] = Xo[k];       /* eq qft_4B */
    free(e); free(o); free(Xe); free(Xo);
}

/* dct_oo: input s_dc_oo, s[n] for odd n in [1, N/4-1]; output X[k] for odd
 * k in [1, N/4-1].  Sec. 5.2.3: multiply by the secant (eq qft_38A), which
 * turns the wanted odd harmonics into even ones of s_dc_oe; halve those
 * (Sec. 3.3) into a dct_ot of periodization N/2; backward eqs qft_38B/38C. */
static void dct_oo(long N, const real *s, real *X)
{
    if (N == 8) {                          /* definition: n = 1, k = 1 */
        X[1] = MUL(s[1], cos_pi_4());
        return;
    }
    real *t = zalloc(N / 4);               /* s_dc_oe(n), odd n */
    for (long n = 1; n < N / 4; n += 2)
        t[n] = MUL(s[n], secant(N, n));    /* eq qft_38A */
    real *Y = zalloc(N / 8);               /* Y(j) = DCT[s_dc_oe](2j), j in [0,N/8-1] */
    dct_ot(N / 2, t, Y);
    for (long j = 0; j + 1 < N / 8; ++j)
        X[2 * j + 1] = ADD(Y[j], Y[j + 1]);/* eq qft_38C */
    X[N / 4 - 1] = Y[N / 8 - 1];           /* eq qft_38B (k+1 term is zero) */
    free(t); free(Y);
}

/* dst: input s_ds_tt, d[n] for n in [1, N/2-1]; output S[k], k in
 * [1, N/2-1].  Same chain as dct (Sec. 5.2.4) with base case N = 4. */
static void dst(long N, const real *d, real *S)
{
    if (N == 4) {                          /* DST-0 definition, eq qft_0C */
        S[1] = d[1];
        return;
    }
    real *e = zalloc(N / 4);               /* s_A_ds_tt(m) = d(2m), m in [1,N/4-1] */
    real *so = zalloc(N / 2);              /* s_ds_ot(n), odd n */
    for (long m = 1; m < N / 4; ++m) e[m] = d[2 * m];
    for (long n = 1; n < N / 2; n += 2) so[n] = d[n];
    real *E = zalloc(N / 4);               /* DST[s_A_ds_tt](k), k in [1,N/4-1] */
    real *O = zalloc(N / 4 + 1);           /* DST[s_ds_ot](k),   k in [1,N/4]   */
    dst(N / 2, e, E);
#ifdef ORACLE_COMPENSATED
    if (class_compensated(N)) dst_ot_comp(N, so, O); else
#endif
    dst_ot(N, so, O);
    for (long k = 1; k < N / 4; ++k) {
        S[k] = ADD(E[k], O[k]);            /* eq qft_5C, DST form */
        S[N / 2 - k] = SUB(O[k], E[k]);    /* eq qft_5D, DST form */
    }
    S[N / 4] = O[N / 4];                   /* eq qft_6,  DST form */
    free(e); free(so); free(E); free(O);
}

/* dst_ot: input s_ds_ot, s[n] for odd n in [1, N/2-1]; output X[k], k in
 * [1, N/4]. */
static void dst_ot(long N, const real *s, real *X)
{
    if (N == 4) {                          /* definition: n = 1, k = 1 */
        X[1] = s[1];
        return;
    }
    real *e = zalloc(N / 4);               /* s_ds_oe(n) */
    real *o = zalloc(N / 4);               /* s_ds_oo(n) */
    for (long n = 1; n < N / 4; n += 2) {
        e[n] = SUB(s[n], s[N / 2 - n]);    /* eq qft_2 (DST: roles swapped) */
        o[n] = ADD(s[n], s[N / 2 - n]);    /* eq qft_1 (DST: roles swapped) */
    }
    real *Xe = zalloc(N / 8 + 1);          /* DST[s_A_ds_ot](j), j in [1,N/8] */
    real *Xo = zalloc(N / 4);              /* DST[s_ds_oo](k),  odd k        */
    dst_ot(N / 2, e, Xe);
    dst_oo(N, o, Xo);
    for (long j = 1; j <= N / 8; ++j) X[2 * j] = Xe[j];     /* eqs qft_4B, qft_10 */
    for (long k = 1; k < N / 4; k += 2) X[k] = Xo[k];
    free(e); free(o); free(Xe); free(Xo);
}

/* dst_oo: input s_ds_oo, odd n in [1, N/4-1]; output odd k in [1, N/4-1]. */
static void dst_oo(long N, const real *s, real *X)
{
    if (N == 8) {                          /* definition: n = 1, k = 1 */
        X[1] = MUL(s[1], cos_pi_4());      /* sin(pi/4) = cos(pi/4) */
        return;
    }
    real *t = zalloc(N / 4);
    for (long n = 1; n < N / 4; n += 2)
        t[n] = MUL(s[n], secant(N, n));    /* eq qft_38A, DST context */
    real *Z = zalloc(N / 8 + 1);           /* Z(j) = DST[s_ds_oe](2j), j in [1,N/8] */
    dst_ot(N / 2, t, Z);
    X[1] = Z[1];                           /* special case k = 1: DST at k = 0 is 0 */
    for (long j = 1; j < N / 8; ++j)
        X[2 * j + 1] = ADD(Z[j], Z[j + 1]);/* eq qft_38C, DST context */
    free(t); free(Z);
}

/* ====================================== compensated FP32 evaluation
 * With -DORACLE_COMPENSATED (and ORACLE_REAL=float) this oracle evaluates the
 * class trees whose periodization is large the way the library does by
 * default.  The FP32 error of the improved QFT comes from the secant
 * conversion (eq qft_38A): near n = N/4 the factor 1/(2 cos(2 pi n/N)) grows
 * like N/(4 pi), every value below it in the tree is that much larger, and
 * the neighbour adds of eqs qft_38B/C cancel the excess, leaving the rounding
 * errors.  So the dct_ot (dst_ot) tree of each of the J largest classes --
 * the odd-time child of dct(M) (dst(M)) for M >= Nroot / 2^(J-1), with
 * J = max(0, floor((log2 Nroot - 14) / 2)) -- runs on unevaluated pairs
 * v = h + l of FP32 numbers, h being exactly the plain FP32 value:
 *   add:  s = ah + bh; z = s - ah; e = (ah - (s - z)) + (bh - z)   (TwoSum,
 *         Knuth, TAOCP vol. 2: s + e = ah + bh exactly); l = (al + bl) + e
 *   sub:  add of (-bh, -bl)
 *   mul by a constant c:  p = ah c; e = fma(ah, c, -p) (the exact product
 *         error, Ogita, Rump and Oishi 2005); l = fma(al, c, e)
 * and each class output is rounded once, h + l, before the combines of
 * eqs qft_5C-6.  The constants are the plain FP32 ones; the operations and
 * their order are the recursion's, so the counters are unchanged. */
#ifdef ORACLE_COMPENSATED
typedef struct { real h, l; } pair;

static inline real fma_r(real a, real b, real c)
{
    return sizeof(real) == sizeof(float) ? (real)fmaf((float)a, (float)b, (float)c) : (real)fma(a, b, c);
}
static inline pair PADD(pair a, pair b)
{
    t_adds++;
    const real s = a.h + b.h;
    const real z = s - a.h;
    const real e = (a.h - (s - z)) + (b.h - z);
    pair r = {s, (a.l + b.l) + e};
    return r;
}
static inline pair PSUB(pair a, pair b)
{
    pair nb = {-b.h, -b.l};
    return PADD(a, nb);
}
static inline pair PMUL(pair a, real c)
{
    t_muls++;
    const real p = a.h * c;
    const real e = fma_r(a.h, c, -p);
    pair r = {p, fma_r(a.l, c, e)};
    return r;
}
static pair *palloc(long n) { return (pair *)calloc((size_t)(n > 0 ? n : 1), sizeof(pair)); }

/* number of compensated classes of a root transform of length Nroot (a test
 * may set another count with oracle_set_comp_classes) */
static int g_comp_override = -1;
static int comp_classes(long Nroot)
{
    if (g_comp_override >= 0) return g_comp_override;
    int r = 0;
    while ((1L << r) < Nroot) ++r;
    return r >= 16 ? (r - 14) / 2 : 0;
}
static int class_compensated(long M)
{
    const int J = comp_classes(t_c->Nroot);
    return J > 0 && M >= (t_c->Nroot >> (J - 1));
}

static void dct_ot_p(long N, const pair *s, pair *X);
static void dct_oo_p(long N, const pair *s, pair *X);
static void dst_ot_p(long N, const pair *s, pair *X);
static void dst_oo_p(long N, const pair *s, pair *X);

/* dct_ot / dct_oo / dst_ot / dst_oo of Sec. 5 on pairs (same steps) */
static void dct_ot_p(long N, const pair *s, pair *X)
{
    if (N == 4) { X[0] = s[1]; return; }
    pair *e = palloc(N / 4), *o = palloc(N / 4), *Xe = palloc(N / 8), *Xo = palloc(N / 4);
    for (long n = 1; n < N / 4; n += 2) {
        e[n] = PADD(s[n], s[N / 2 - n]);   /* eq qft_1 */
        o[n] = PSUB(s[n], s[N / 2 - n]);   /* eq qft_2 */
    }
    dct_ot_p(N / 2, e, Xe);
    dct_oo_p(N, o, Xo);
    for (long j = 0; j < N / 8; ++j) X[2 * j] = Xe[j];
    for (long k = 1; k < N / 4; k += 2) X[k] = Xo[k];
    free(e); free(o); free(Xe); free(Xo);
}
static void dct_oo_p(long N, const pair *s, pair *X)
{
    if (N == 8) { X[1] = PMUL(s[1], cos_pi_4()); return; }
    pair *t = palloc(N / 4), *Y = palloc(N / 8);
    for (long n = 1; n < N / 4; n += 2) t[n] = PMUL(s[n], secant(N, n));   /* eq qft_38A */
    dct_ot_p(N / 2, t, Y);
    for (long j = 0; j + 1 < N / 8; ++j) X[2 * j + 1] = PADD(Y[j], Y[j + 1]);   /* eq qft_38C */
    X[N / 4 - 1] = Y[N / 8 - 1];                                               /* eq qft_38B */
    free(t); free(Y);
}
static void dst_ot_p(long N, const pair *s, pair *X)
{
    if (N == 4) { X[1] = s[1]; return; }
    pair *e = palloc(N / 4), *o = palloc(N / 4), *Xe = palloc(N / 8 + 1), *Xo = palloc(N / 4);
    for (long n = 1; n < N / 4; n += 2) {
        e[n] = PSUB(s[n], s[N / 2 - n]);
        o[n] = PADD(s[n], s[N / 2 - n]);
    }
    dst_ot_p(N / 2, e, Xe);
    dst_oo_p(N, o, Xo);
    for (long j = 1; j <= N / 8; ++j) X[2 * j] = Xe[j];
    for (long k = 1; k < N / 4; k += 2) X[k] = Xo[k];
    free(e); free(o); free(Xe); free(Xo);
}
static void dst_oo_p(long N, const pair *s, pair *X)
{
    if (N == 8) { X[1] = PMUL(s[1], cos_pi_4()); return; }
    pair *t = palloc(N / 4), *Z = palloc(N / 8 + 1);
    for (long n = 1; n < N / 4; n += 2) t[n] = PMUL(s[n], secant(N, n));
    dst_ot_p(N / 2, t, Z);
    X[1] = Z[1];
    for (long j = 1; j < N / 8; ++j) X[2 * j + 1] = PADD(Z[j], Z[j + 1]);
    free(t); free(Z);
}

/* a class tree on pairs: plain input (l = 0), each output rounded once */
static void dct_ot_comp(long N, const real *s, real *X)
{
    pair *sp = palloc(N / 2), *Xp = palloc(N / 4);
    for (long n = 1; n < N / 2; n += 2) sp[n].h = s[n];
    dct_ot_p(N, sp, Xp);
    for (long k = 0; k < N / 4; ++k) X[k] = Xp[k].h + Xp[k].l;
    free(sp); free(Xp);
}
static void dst_ot_comp(long N, const real *s, real *X)
{
    pair *sp = palloc(N / 2), *Xp = palloc(N / 4 + 1);
    for (long n = 1; n < N / 2; n += 2) sp[n].h = s[n];
    dst_ot_p(N, sp, Xp);
    for (long k = 1; k <= N / 4; ++k) X[k] = Xp[k].h + Xp[k].l;
    free(sp); free(Xp);
}
#endif

/* rdft (= rdft_cla, Sec. 4.2): input s_re_tt x[n], n in [0, N-1]; output
 * X[k], k in [0, N/2] as real and imaginary parts. */
static void rdft(long N, const real *x, real *Xre, real *Xim)
{
    if (N == 2) {                          /* RDFT definition */
        Xre[0] = ADD(x[0], x[1]);
        Xre[1] = SUB(x[0], x[1]);
        Xim[0] = 0; Xim[1] = 0;
        return;
    }
    real *c = zalloc(N / 2 + 1);           /* s_dc_tt */
    real *d = zalloc(N / 2);               /* s_ds_tt */
    c[0] = x[0];
    c[N / 2] = x[N / 2];
    for (long n = 1; n < N / 2; ++n) {
        c[n] = ADD(x[n], x[N - n]);
        d[n] = SUB(x[n], x[N - n]);
    }
    real *C = zalloc(N / 2 + 1);
    real *S = zalloc(N / 2);
    dct(N, c, C);
    dst(N, d, S);
    for (long k = 0; k <= N / 2; ++k) Xre[k] = C[k];
    Xim[0] = 0; Xim[N / 2] = 0;
    for (long k = 1; k < N / 2; ++k) Xim[k] = -S[k];
    free(c); free(d); free(C); free(S);
}

/* cdft (= cdft_cla, Sec. 4.1): input s_cx_tt z[n]; output Z[k], k in [0,N-1].
 * Splits into the RDFTs of the real and imaginary parts and recombines with
 * the six frequency-domain relations of Sec. 4.1. */
static void cdft(long N, const real *zre, const real *zim, real *Zre, real *Zim)
{
    if (N == 2) {                          /* CDFT definition */
        Zre[0] = ADD(zre[0], zre[1]); Zim[0] = ADD(zim[0], zim[1]);
        Zre[1] = SUB(zre[0], zre[1]); Zim[1] = SUB(zim[0], zim[1]);
        return;
    }
    real *Ar = zalloc(N / 2 + 1), *Ai = zalloc(N / 2 + 1);
    real *Br = zalloc(N / 2 + 1), *Bi = zalloc(N / 2 + 1);
    rdft(N, zre, Ar, Ai);
    rdft(N, zim, Br, Bi);
    for (long k = 1; k < N / 2; ++k) {
        Zre[k]     = SUB(Ar[k], Bi[k]);
        Zre[N - k] = ADD(Ar[k], Bi[k]);
        Zim[k]     = ADD(Ai[k], Br[k]);
        Zim[N - k] = SUB(Br[k], Ai[k]);
    }
    Zre[0] = Ar[0];         Zim[0] = Br[0];
    Zre[N / 2] = Ar[N / 2]; Zim[N / 2] = Br[N / 2];
    free(Ar); free(Ai); free(Br); free(Bi);
}

/* ============================================ classical QFT (Sec. 4)
 * The comparison algorithm of the paper: the same cdft / rdft, but dct_cla,
 * dct_to_cla, dst_cla and dst_to_cla below the fold (Sec. 4.3-4.6), which
 * separate even from odd HARMONICS first (eqs qft_1/qft_2, qft_9/qft_10) and
 * convert odd harmonics into even ones by the secant (eqs qft_26/qft_28) on
 * signals that still hold even time indices.  Arrays are indexed by the
 * paper's n and k, as above; counters and constants are shared.
 * Readings (the paper describes the functions in words; the printed
 * clas_QFT columns of Tab. 3-5 and the cost formulas of Sec. 4 fix them):
 *  - dct_to_cla: the n = 0 secant 1/(2 cos 0) = 1/2 is applied as a
 *    multiplication by 1/2 (exact; counted, as in the cost formulas), and the
 *    even/odd harmonic separation of s_dc_t1t runs over n in [0, N/4-1] like
 *    the one of dct_cla, with the partner of n = 0 a stored zero (exact;
 *    counted).
 *  - dct_to_cla at N = 8 applies the DCT definition:
 *    X(1) = s(0) + s(1) cos(pi/4), X(3) = s(0) - s(1) cos(pi/4).
 *  - dst_to_cla: DST[s_ds_te](0) = DST[s_ds_te](N/2) = 0 in eq qft_28 (DST
 *    form), so X(1) and X(N/2-1) take one term.
 * With these readings the counted operations equal Tab. 3-5 (N = 4..2048)
 * and the Sec. 4 formulas (N >= 8). */
static void dct_cla(long N, const real *c, real *C);
static void dct_to_cla(long N, const real *s, real *X);
static void dst_cla(long N, const real *d, real *S);
static void dst_to_cla(long N, const real *s, real *X);

/* dct_cla: s_dc_tt c[n], n in [0, N/2] -> C[k], k in [0, N/2].  Separation
 * of even from odd harmonics (eqs qft_1, qft_2), even-harmonic halving of
 * s_dc_te (eqs qft_9, qft_10), backward eq qft_4B. */
static void dct_cla(long N, const real *c, real *C)
{
    if (N == 2) {                          /* DCT-0 definition */
        C[0] = ADD(c[0], c[1]);
        C[1] = SUB(c[0], c[1]);
        return;
    }
    real *te = zalloc(N / 4 + 1);          /* s_dc_te(n), n in [0, N/4] -> s_A_dc_tt */
    real *to = zalloc(N / 4);              /* s_dc_to(n), n in [0, N/4-1] */
    for (long n = 0; n < N / 4; ++n) {
        te[n] = ADD(c[n], c[N / 2 - n]);   /* eq qft_1 */
        to[n] = SUB(c[n], c[N / 2 - n]);   /* eq qft_2 */
    }
    te[N / 4] = c[N / 4];                  /* eq qft_1, n = N/4 */
    real *CA = zalloc(N / 4 + 1);          /* DCT[s_A_dc_tt](kA), kA in [0, N/4] */
    real *Xo = zalloc(N / 2);              /* DCT[s_dc_to](k), odd k */
    dct_cla(N / 2, te, CA);
    dct_to_cla(N, to, Xo);
    for (long kA = 0; kA <= N / 4; ++kA) C[2 * kA] = CA[kA];   /* eqs qft_10, qft_4B */
    for (long k = 1; k < N / 2; k += 2) C[k] = Xo[k];         /* eq qft_4B */
    free(te); free(to); free(CA); free(Xo);
}

/* dct_to_cla: s_dc_to s[n], n in [0, N/4-1] -> X[k], odd k in [1, N/2-1].
 * Secant conversion into s_dc_t1e (eq qft_26, backward eq qft_28), even
 * harmonic halving into s_A_dc_t1t of periodization N/2, then that signal is
 * split like s_dc_tt in dct_cla into s_B_dc_tt (periodization N/4) and
 * s_A_dc_to (periodization N/2). */
static void dct_to_cla(long N, const real *s, real *X)
{
    if (N == 4) {                          /* DCT definition: n = 0, k = 1 */
        X[1] = s[0];
        return;
    }
    if (N == 8) {                          /* DCT definition: n in {0, 1}, k in {1, 3} */
        const real p = MUL(s[1], cos_pi_4());
        X[1] = ADD(s[0], p);
        X[3] = SUB(s[0], p);
        return;
    }
    const long NA = N / 2;
    real *t = zalloc(NA / 2 + 1);          /* s_dc_t1e(n) = s_A_dc_t1t(n), n in [0, N/4-1]; t[N/4] = 0 */
    t[0] = MUL(s[0], (real)0.5);           /* eq qft_26, n = 0: 1/(2 cos 0) */
    for (long n = 1; n < N / 4; ++n)
        t[n] = MUL(s[n], secant(N, n));    /* eq qft_26 */
    real *B = zalloc(NA / 4 + 1);          /* s_B_dc_tt(n), n in [0, NA/4] (periodization N/4) */
    real *Ao = zalloc(NA / 4);             /* s_A_dc_to(n), n in [0, NA/4-1] (periodization N/2) */
    for (long n = 0; n < NA / 4; ++n) {
        B[n] = ADD(t[n], t[NA / 2 - n]);   /* eq qft_1 at periodization NA */
        Ao[n] = SUB(t[n], t[NA / 2 - n]);  /* eq qft_2 at periodization NA */
    }
    B[NA / 4] = t[NA / 4];
    real *YB = zalloc(NA / 4 + 1);         /* DCT[s_B_dc_tt](kB), kB in [0, N/8] */
    real *YA = zalloc(NA / 2);             /* DCT[s_A_dc_to](kA), odd kA in [1, N/4-1] */
    dct_cla(NA / 2, B, YB);
    dct_to_cla(NA, Ao, YA);
    real *T = zalloc(NA / 2 + 1);          /* DCT[s_A_dc_t1t](kA) = DCT[s_dc_t1e](2 kA), kA in [0, N/4] */
    for (long kA = 0; kA <= NA / 2; ++kA) T[kA] = (kA & 1) ? YA[kA] : YB[kA / 2];   /* eq qft_4B */
    for (long k = 1; k < N / 2; k += 2)
        X[k] = ADD(T[(k - 1) / 2], T[(k + 1) / 2]);   /* eq qft_28 */
    free(t); free(B); free(Ao); free(YB); free(YA); free(T);
}

/* dst_cla: s_ds_tt d[n], n in [1, N/2-1] -> S[k], k in [1, N/2-1].  DST form
 * of the harmonic separation (the even-k child takes the difference). */
static void dst_cla(long N, const real *d, real *S)
{
    if (N == 4) {                          /* DST-0 definition: n = 1, k = 1 */
        S[1] = d[1];
        return;
    }
    real *te = zalloc(N / 4);              /* s_ds_te(n), n in [1, N/4-1] -> s_A_ds_tt */
    real *to = zalloc(N / 4 + 1);          /* s_ds_to(n), n in [1, N/4] */
    for (long n = 1; n < N / 4; ++n) {
        te[n] = SUB(d[n], d[N / 2 - n]);
        to[n] = ADD(d[n], d[N / 2 - n]);
    }
    to[N / 4] = d[N / 4];
    real *SA = zalloc(N / 4);              /* DST[s_A_ds_tt](kA), kA in [1, N/4-1] */
    real *Xo = zalloc(N / 2);              /* DST[s_ds_to](k), odd k */
    dst_cla(N / 2, te, SA);
    dst_to_cla(N, to, Xo);
    for (long kA = 1; kA < N / 4; ++kA) S[2 * kA] = SA[kA];
    for (long k = 1; k < N / 2; k += 2) S[k] = Xo[k];
    free(te); free(to); free(SA); free(Xo);
}

/* dst_to_cla: s_ds_to s[n], n in [1, N/4] -> X[k], odd k in [1, N/2-1].
 * The index n = N/4 is split off (eqs qft_29, qft_29b) and its contribution
 * added by the definition (eqs qft_29c, qft_29d); the rest (s_ds_t1o) is
 * converted by the secant into s_ds_te (eqs qft_26, qft_28, DST form) and
 * halved into s_A_ds_tt of periodization N/2. */
static void dst_to_cla(long N, const real *s, real *X)
{
    if (N == 4) {                          /* DST definition: n = 1, k = 1 */
        X[1] = s[1];
        return;
    }
    real *t = zalloc(N / 4);               /* s_ds_te(n) = s_A_ds_tt(n), n in [1, N/4-1] */
    for (long n = 1; n < N / 4; ++n)
        t[n] = MUL(s[n], secant(N, n));    /* eq qft_26, DST context */
    real *SA = zalloc(N / 4);              /* DST[s_A_ds_tt](kA) = DST[s_ds_te](2 kA), kA in [1, N/4-1] */
    dst_cla(N / 2, t, SA);
    const real e1 = s[N / 4];              /* DST[s_ds_e1o](1), eq qft_29d */
    for (long k = 1; k < N / 2; k += 2) {
        real v;                            /* DST[s_ds_t1o](k), eq qft_28 (DST form) */
        if (k == 1) v = SA[1];
        else if (k == N / 2 - 1) v = SA[N / 4 - 1];
        else v = ADD(SA[(k - 1) / 2], SA[(k + 1) / 2]);
        X[k] = (((k - 1) / 2) & 1) ? SUB(v, e1) : ADD(v, e1);   /* eq qft_29c */
    }
    free(t); free(SA);
}

static void rdft_cla(long N, const real *x, real *Xre, real *Xim)
{
    if (N == 2) {
        Xre[0] = ADD(x[0], x[1]);
        Xre[1] = SUB(x[0], x[1]);
        Xim[0] = 0; Xim[1] = 0;
        return;
    }
    real *c = zalloc(N / 2 + 1);
    real *d = zalloc(N / 2);
    c[0] = x[0];
    c[N / 2] = x[N / 2];
    for (long n = 1; n < N / 2; ++n) {
        c[n] = ADD(x[n], x[N - n]);
        d[n] = SUB(x[n], x[N - n]);
    }
    real *C = zalloc(N / 2 + 1);
    real *S = zalloc(N / 2);
    dct_cla(N, c, C);
    dst_cla(N, d, S);
    for (long k = 0; k <= N / 2; ++k) Xre[k] = C[k];
    Xim[0] = 0; Xim[N / 2] = 0;
    for (long k = 1; k < N / 2; ++k) Xim[k] = -S[k];
    free(c); free(d); free(C); free(S);
}

static void cdft_cla(long N, const real *zre, const real *zim, real *Zre, real *Zim)
{
    if (N == 2) {
        Zre[0] = ADD(zre[0], zre[1]); Zim[0] = ADD(zim[0], zim[1]);
        Zre[1] = SUB(zre[0], zre[1]); Zim[1] = SUB(zim[0], zim[1]);
        return;
    }
    real *Ar = zalloc(N / 2 + 1), *Ai = zalloc(N / 2 + 1);
    real *Br = zalloc(N / 2 + 1), *Bi = zalloc(N / 2 + 1);
    rdft_cla(N, zre, Ar, Ai);
    rdft_cla(N, zim, Br, Bi);
    for (long k = 1; k < N / 2; ++k) {
        Zre[k]     = SUB(Ar[k], Bi[k]);
        Zre[N - k] = ADD(Ar[k], Bi[k]);
        Zim[k]     = ADD(Ai[k], Br[k]);
        Zim[N - k] = SUB(Br[k], Ai[k]);
    }
    Zre[0] = Ar[0];         Zim[0] = Br[0];
    Zre[N / 2] = Ar[N / 2]; Zim[N / 2] = Br[N / 2];
    free(Ar); free(Ai); free(Br); free(Bi);
}

/* ------------------------------------------------------------- helpers */
static int is_pow2(long n) { return n >= 2 && (n & (n - 1)) == 0; }

static void set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

/* ============================================================ public API
 * All arrays are row-major [batch][...] with complex values interleaved
 * (re, im) as doubles.  Return 0 on success, -1 on a bad argument. */

int oracle_is_float(void) { return sizeof(real) == sizeof(float); }

int oracle_is_compensated(void)
{
#ifdef ORACLE_COMPENSATED
    return 1;
#else
    return 0;
#endif
}

/* Sets the number of compensated classes for every transform (J >= 0), or
 * restores the default rule (J < 0).  No effect without ORACLE_COMPENSATED. */
void oracle_set_comp_classes(int J)
{
#ifdef ORACLE_COMPENSATED
    g_comp_override = J;
#else
    (void)J;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Forward CDFT (eq qft_0A) of each row; z, Z: [batch][N][2]. */
int oracle_cdft(long N, long batch, const double *z, double *Z, int threads)
{
    if (!is_pow2(N) || batch < 0) return -1;
    set_threads(threads);
    #pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < batch; ++b) {
        consts_t *c = consts_make(N);
        t_c = c;
        real *zr = zalloc(N), *zi = zalloc(N), *Zr = zalloc(N), *Zi = zalloc(N);
        for (long n = 0; n < N; ++n) { zr[n] = (real)z[(b * N + n) * 2]; zi[n] = (real)z[(b * N + n) * 2 + 1]; }
        cdft(N, zr, zi, Zr, Zi);
        for (long k = 0; k < N; ++k) { Z[(b * N + k) * 2] = (double)Zr[k]; Z[(b * N + k) * 2 + 1] = (double)Zi[k]; }
        free(zr); free(zi); free(Zr); free(Zi);
        t_c = NULL;
        consts_free(c);
    }
    return 0;
}

/* Inverse CDFT: x = swap(cdft(swap(X))) / N (reading of the paper's silence). */
int oracle_icdft(long N, long batch, const double *X, double *x, int threads)
{
    if (!is_pow2(N) || batch < 0) return -1;
    double *sw = (double *)malloc(sizeof(double) * 2 * (size_t)(N * (batch > 0 ? batch : 1)));
    for (long i = 0; i < N * batch; ++i) { sw[2 * i] = X[2 * i + 1]; sw[2 * i + 1] = X[2 * i]; }
    int rc = oracle_cdft(N, batch, sw, x, threads);
    for (long i = 0; i < N * batch; ++i) {
        double re = x[2 * i + 1], im = x[2 * i];
        x[2 * i] = re / (double)N;
        x[2 * i + 1] = im / (double)N;
    }
    free(sw);
    return rc;
}

/* Forward RDFT of real rows: x [batch][N] -> X [batch][N/2+1][2]. */
int oracle_rdft(long N, long batch, const double *x, double *X, int threads)
{
    if (!is_pow2(N) || batch < 0) return -1;
    set_threads(threads);
    long H = N / 2 + 1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < batch; ++b) {
        consts_t *c = consts_make(N);
        t_c = c;
        real *xr = zalloc(N), *Xr = zalloc(H), *Xi = zalloc(H);
        for (long n = 0; n < N; ++n) xr[n] = (real)x[b * N + n];
        rdft(N, xr, Xr, Xi);
        for (long k = 0; k < H; ++k) { X[(b * H + k) * 2] = (double)Xr[k]; X[(b * H + k) * 2 + 1] = (double)Xi[k]; }
        free(xr); free(Xr); free(Xi);
        t_c = NULL;
        consts_free(c);
    }
    return 0;
}

/* Shared body of the real inverse and of the rfft adjoint:
 * a(k) = wa_k Re Y(k), k in [0, N/2]; b(k) = wb Im Y(k), k in [1, N/2-1];
 * A = DCT-0[a], B = DST-0[b] (eqs qft_0B, qft_0C, by dct and dst);
 * x(n) = s (A(n) - B(n)), x(N-n) = s (A(n) + B(n)).  N >= 4. */
static void real_synthesis(long N, const double *Y, double *x, double w_mid, double scale)
{
    long H = N / 2 + 1;
    real *a = zalloc(H), *bb = zalloc(N / 2), *A = zalloc(H), *B = zalloc(N / 2);
    a[0] = (real)Y[0];
    a[N / 2] = (real)Y[2 * (N / 2)];
    for (long k = 1; k < N / 2; ++k) {
        a[k] = (real)(w_mid * Y[2 * k]);
        bb[k] = (real)(w_mid * Y[2 * k + 1]);
    }
    dct(N, a, A);
    dst(N, bb, B);
    x[0] = (double)A[0] * scale;
    x[N / 2] = (double)A[N / 2] * scale;
    for (long n = 1; n < N / 2; ++n) {
        x[n] = (double)SUB(A[n], B[n]) * scale;
        x[N - n] = (double)ADD(A[n], B[n]) * scale;
    }
    free(a); free(bb); free(A); free(B);
}

/* Inverse real DFT (C2R): Y [batch][N/2+1][2] -> x [batch][N], scaled 1/N.
 * The imaginary parts of Y(0) and Y(N/2) are ignored. */
int oracle_irdft(long N, long batch, const double *Y, double *x, int threads)
{
    if (!is_pow2(N) || N < 4 || batch < 0) return -1;
    set_threads(threads);
    long H = N / 2 + 1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < batch; ++b) {
        consts_t *c = consts_make(N);
        t_c = c;
        real_synthesis(N, Y + b * H * 2, x + b * N, 2.0, 1.0 / (double)N);
        t_c = NULL;
        consts_free(c);
    }
    return 0;
}

/* Adjoint of the forward RDFT with respect to the real inner product on
 * (Re, Im) pairs: g_x(n) = sum_k g_re(k) cos(theta n k) - g_im(k) sin(theta n k),
 * k in [0, N/2], i.e. real_synthesis with unit weights and no scaling. */
int oracle_rdft_adjoint(long N, long batch, const double *G, double *gx, int threads)
{
    if (!is_pow2(N) || N < 4 || batch < 0) return -1;
    set_threads(threads);
    long H = N / 2 + 1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < batch; ++b) {
        consts_t *c = consts_make(N);
        t_c = c;
        real_synthesis(N, G + b * H * 2, gx + b * N, 1.0, 1.0);
        t_c = NULL;
        consts_free(c);
    }
    return 0;
}

/* Standalone DCT-0 / DST-0 of periodization N (eqs qft_0B/qft_0C) by the
 * improved QFT functions dct and dst (single row).
 * dct: c[0..N/2] -> C[0..N/2];  dst: d[0..N/2] (d[0], d[N/2] ignored) ->
 * S[0..N/2] (S[0] = S[N/2] = 0). */
int oracle_dct0(long N, const double *c, double *C)
{
    if (!is_pow2(N)) return -1;
    consts_t *k = consts_make(N < 8 ? 8 : N);
    t_c = k;
    real *ci = zalloc(N / 2 + 1), *Co = zalloc(N / 2 + 1);
    for (long n = 0; n <= N / 2; ++n) ci[n] = (real)c[n];
    dct(N, ci, Co);
    for (long n = 0; n <= N / 2; ++n) C[n] = (double)Co[n];
    free(ci); free(Co);
    t_c = NULL;
    consts_free(k);
    return 0;
}

int oracle_dst0(long N, const double *d, double *S)
{
    if (!is_pow2(N) || N < 4) return -1;
    consts_t *k = consts_make(N < 8 ? 8 : N);
    t_c = k;
    real *di = zalloc(N / 2 + 1), *So = zalloc(N / 2 + 1);
    for (long n = 1; n < N / 2; ++n) di[n] = (real)d[n];
    dst(N, di, So);
    S[0] = 0; S[N / 2] = 0;
    for (long n = 1; n < N / 2; ++n) S[n] = (double)So[n];
    free(di); free(So);
    t_c = NULL;
    consts_free(k);
    return 0;
}

/* One of the eight functions on its own signal type (Tab. 1), for the
 * per-function checks.  which: 0 dct, 1 dct_ot, 2 dct_oo, 3 dst, 4 dst_ot,
 * 5 dst_oo.  in[] is indexed by n (length N/2+1, unused cells ignored);
 * out[] is indexed by k (length N/2+1, cells outside sto_k left 0). */
int oracle_function(int which, long N, const double *in, double *out)
{
    long L = N / 2 + 1;
    if (!is_pow2(N)) return -1;
    consts_t *k = consts_make(N < 8 ? 8 : N);
    t_c = k;
    real *s = zalloc(L), *X = zalloc(L);
    for (long i = 0; i < L; ++i) s[i] = (real)in[i];
    int rc = 0;
    switch (which) {
    case 0: if (N < 2) rc = -1; else dct(N, s, X); break;
    case 1: if (N < 4) rc = -1; else dct_ot(N, s, X); break;
    case 2: if (N < 8) rc = -1; else dct_oo(N, s, X); break;
    case 3: if (N < 4) rc = -1; else dst(N, s, X); break;
    case 4: if (N < 4) rc = -1; else dst_ot(N, s, X); break;
    case 5: if (N < 8) rc = -1; else dst_oo(N, s, X); break;
    default: rc = -1;
    }
    for (long i = 0; i < L; ++i) out[i] = (double)X[i];
    free(s); free(X);
    t_c = NULL;
    consts_free(k);
    return rc;
}

/* Operation counts of one transform (kind 0 CDFT, 1 RDFT, 2 DCT-0, 3 DST-0)
 * of size N, as counted by ADD/SUB/MUL while computing it on a zero input. */
int oracle_counts(int kind, long N, long long *adds, long long *muls)
{
    if (!is_pow2(N)) return -1;
    consts_t *k = consts_make(N < 8 ? 8 : N);
    t_c = k;
    t_adds = 0; t_muls = 0;
    real *a = zalloc(N), *b = zalloc(N), *c = zalloc(N), *d = zalloc(N);
    int rc = 0;
    switch (kind) {
    case 0: cdft(N, a, b, c, d); break;
    case 1: rdft(N, a, c, d); break;
    case 2: dct(N, a, c); break;
    case 3: if (N < 4) rc = -1; else dst(N, a, c); break;
    default: rc = -1;
    }
    *adds = t_adds; *muls = t_muls;
    free(a); free(b); free(c); free(d);
    t_c = NULL;
    consts_free(k);
    return rc;
}

/* Which trigonometric constants a CDFT of size N uses (Sec. 6.1):
 * used[m] = 1 for every secant angle 2 pi m / N used, m in [1, N/4);
 * *cos_pi_4 = 1 if the base-case constant cos(pi/4) was used.
 * Returns the number of secant angles used. */
long oracle_constants_used(long N, unsigned char *used, int *cos_pi_4_used)
{
    if (!is_pow2(N) || N < 8) return -1;
    consts_t *k = consts_make(N);
    t_c = k;
    real *a = zalloc(N), *b = zalloc(N), *c = zalloc(N), *d = zalloc(N);
    cdft(N, a, b, c, d);
    long cnt = 0;
    for (long m = 0; m <= N / 4; ++m) { used[m] = k->used[m]; cnt += k->used[m]; }
    *cos_pi_4_used = k->cos_pi_4_used;
    free(a); free(b); free(c); free(d);
    t_c = NULL;
    consts_free(k);
    return cnt;
}

/* The secant constants as the oracle rounds them (for the test that pins
 * their rounding to the long-double value). */
int oracle_secant_table(long N, double *sec)
{
    if (!is_pow2(N) || N < 8) return -1;
    consts_t *k = consts_make(N);
    for (long m = 0; m <= N / 4; ++m) sec[m] = (double)k->sec[m];
    consts_free(k);
    return 0;
}

/* O(N^2) DFT straight from eq qft_0A, accumulated in long double with the
 * angle reduced exactly (n k mod N).  One row. */
int oracle_brute_dft(long N, const double *z, double *Z)
{
    if (N < 1) return -1;
    long double *cs = (long double *)malloc(sizeof(long double) * (size_t)N);
    long double *sn = (long double *)malloc(sizeof(long double) * (size_t)N);
    for (long r = 0; r < N; ++r) {
        long double a = 2.0L * PI_L * (long double)r / (long double)N;
        cs[r] = cosl(a);
        sn[r] = sinl(a);
    }
    for (long k = 0; k < N; ++k) {
        long double ar = 0, ai = 0;
        for (long n = 0; n < N; ++n) {
            long r = (long)(((long long)n * (long long)k) % N);
            long double xr = z[2 * n], xi = z[2 * n + 1];
            /* (xr + i xi)(cos - i sin) */
            ar += xr * cs[r] + xi * sn[r];
            ai += xi * cs[r] - xr * sn[r];
        }
        Z[2 * k] = (double)ar;
        Z[2 * k + 1] = (double)ai;
    }
    free(cs); free(sn);
    return 0;
}

/* ------------------------------------------------ classical QFT public API */
/* Forward CDFT (eq qft_0A) of each row by the classical QFT of Sec. 4. */
int oracle_cdft_cla(long N, long batch, const double *z, double *Z, int threads)
{
    if (!is_pow2(N) || batch < 0) return -1;
    set_threads(threads);
    #pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < batch; ++b) {
        consts_t *c = consts_make(N < 8 ? 8 : N);
        t_c = c;
        real *zr = zalloc(N), *zi = zalloc(N), *Zr = zalloc(N), *Zi = zalloc(N);
        for (long n = 0; n < N; ++n) { zr[n] = (real)z[(b * N + n) * 2]; zi[n] = (real)z[(b * N + n) * 2 + 1]; }
        cdft_cla(N, zr, zi, Zr, Zi);
        for (long k = 0; k < N; ++k) { Z[(b * N + k) * 2] = (double)Zr[k]; Z[(b * N + k) * 2 + 1] = (double)Zi[k]; }
        free(zr); free(zi); free(Zr); free(Zi);
        t_c = NULL;
        consts_free(c);
    }
    return 0;
}

/* One classical function on its own signal type (Tab. 1): which 0 dct_cla,
 * 1 dct_to_cla, 2 dst_cla, 3 dst_to_cla; in[] indexed by n, out[] by k
 * (length N/2+1 each, cells outside sto_k left 0). */
int oracle_function_cla(int which, long N, const double *in, double *out)
{
    long L = N / 2 + 1;
    if (!is_pow2(N)) return -1;
    consts_t *k = consts_make(N < 8 ? 8 : N);
    t_c = k;
    real *s = zalloc(L), *X = zalloc(L);
    for (long i = 0; i < L; ++i) s[i] = (real)in[i];
    int rc = 0;
    switch (which) {
    case 0: if (N < 2) rc = -1; else dct_cla(N, s, X); break;
    case 1: if (N < 4) rc = -1; else dct_to_cla(N, s, X); break;
    case 2: if (N < 4) rc = -1; else dst_cla(N, s, X); break;
    case 3: if (N < 4) rc = -1; else dst_to_cla(N, s, X); break;
    default: rc = -1;
    }
    for (long i = 0; i < L; ++i) out[i] = (double)X[i];
    free(s); free(X);
    t_c = NULL;
    consts_free(k);
    return rc;
}

/* Operation counts of one classical transform (kind 0 CDFT, 1 RDFT). */
int oracle_counts_cla(int kind, long N, long long *adds, long long *muls)
{
    if (!is_pow2(N)) return -1;
    consts_t *k = consts_make(N < 8 ? 8 : N);
    t_c = k;
    t_adds = 0; t_muls = 0;
    real *a = zalloc(N), *b = zalloc(N), *c = zalloc(N), *d = zalloc(N);
    int rc = 0;
    switch (kind) {
    case 0: cdft_cla(N, a, b, c, d); break;
    case 1: rdft_cla(N, a, c, d); break;
    default: rc = -1;
    }
    *adds = t_adds; *muls = t_muls;
    free(a); free(b); free(c); free(d);
    t_c = NULL;
    consts_free(k);
    return rc;
}

/* Constants a classical CDFT of size N uses (as oracle_constants_used). */
long oracle_constants_used_cla(long N, unsigned char *used, int *cos_pi_4_used)
{
    if (!is_pow2(N) || N < 8) return -1;
    consts_t *k = consts_make(N);
    t_c = k;
    real *a = zalloc(N), *b = zalloc(N), *c = zalloc(N), *d = zalloc(N);
    cdft_cla(N, a, b, c, d);
    long cnt = 0;
    for (long m = 0; m <= N / 4; ++m) { used[m] = k->used[m]; cnt += k->used[m]; }
    *cos_pi_4_used = k->cos_pi_4_used;
    free(a); free(b); free(c); free(d);
    t_c = NULL;
    consts_free(k);
    return cnt;
}

/* Reference DFT for error measurements (eq qft_44 needs a result more exact
 * than FP64): iterative radix-2 decimation in time, every value and every
 * twiddle factor e^{-2 pi i j / len} in long double (cosl/sinl of the exact
 * angle).  Not part of either QFT algorithm.  One row, N a power of two. */
int oracle_fft_ld(long N, const double *z, double *Z)
{
    if (!is_pow2(N) && N != 1) return -1;
    long double *re = (long double *)malloc(sizeof(long double) * (size_t)N);
    long double *im = (long double *)malloc(sizeof(long double) * (size_t)N);
    for (long n = 0; n < N; ++n) { re[n] = z[2 * n]; im[n] = z[2 * n + 1]; }
    for (long i = 1, j = 0; i < N; ++i) {      /* bit-reversal permutation */
        long bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            long double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (long len = 2; len <= N; len <<= 1) {
        for (long j = 0; j < len / 2; ++j) {
            const long double a = -2.0L * PI_L * (long double)j / (long double)len;
            const long double wr = cosl(a), wi = sinl(a);
            for (long i = 0; i < N; i += len) {
                long double *ur = &re[i + j], *ui = &im[i + j];
                long double *vr = &re[i + j + len / 2], *vi = &im[i + j + len / 2];
                const long double tr = *vr * wr - *vi * wi, ti = *vr * wi + *vi * wr;
                *vr = *ur - tr; *vi = *ui - ti;
                *ur = *ur + tr; *ui = *ui + ti;
            }
        }
    }
    for (long k = 0; k < N; ++k) { Z[2 * k] = (double)re[k]; Z[2 * k + 1] = (double)im[k]; }
    free(re); free(im);
    return 0;
}
