/*
 * hz_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, single-threaded CPU implementation of the one-sided implicit
 * Hari-Zimmermann GSVD of a full-column-rank pair (F, G), written from
 * Novakovic & Singer, "Implicit Hari-Zimmermann algorithm for the generalized
 * SVD on the GPUs" (arXiv 1909.00101):
 *
 *   - pointwise (non-blocked), sequential row-cyclic pivot order
 *     (i = 0..n-2, j = i+1..n-1), the sequential strategy of Sec. 2.1;
 *   - the variants of Table "Variants" (Sec. 2.6), one bit each:
 *     variant 0: prescaling of F, G by Z0 = diag(1/||g_j||) (Sec. 2, the
 *     diagonal of B assumed unit), pivot B-hat taken with unit diagonal,
 *     ordinary dot products; +1: the enhanced dot products of App. A;
 *     +2: no prescaling, each pivot pair rescaled by D-hat (Sec. 2.1) and
 *     Z-hat = D-hat Z-hat'; +4: criterion C2;
 *   - per-step column sorting (Sec. 2.1, the P-hat permutation);
 *   - relative-orthogonality skip test (Sec. 2.1);
 *   - transformation Z-hat' by Sec. 2.1.1 (complex) or Sec. 2.1.2 (real),
 *     with their exceptions;
 *   - small/big classification by criterion C1 or C2 (Sec. 2.5);
 *   - stop after a sweep with no transformation at all (Sec. 2.5, the
 *     pointwise stopping rule);
 *   - final rescaling (Sec. 2.4) and the sort by descending Sigma (Sec. 1).
 *
 * The same source is compiled twice: with real_t = double (names *_d) and
 * with real_t = long double (names *_ld, HZO_EXTENDED), the latter giving
 * reference generalized singular values of the rounded inputs.
 *
 * Every sum is a plain sequential loop; compiled with -ffp-contract=off, so
 * no multiply-add is fused unless written as fma().  No blocking, fusion or
 * reordering beyond what the paper's sequential method states.
 *
 * This file shares no code, header, table or helper with the CUDA library;
 * only tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Readings of the paper (where it is silent, garbled or at odds with itself):
 *   R1  cos(theta) = 1/sqrt(1 + tan^2(theta)) (Sec. 2.1.1 prints the root
 *       without the square root; without it Z^T B Z != I).
 *   R2  real exception (Sec. 2.1.2): the signed form of the complex
 *       exception (Sec. 2.1.1) with e^{i zeta} = sign(x); the printed |x| in
 *       both columns does not diagonalise B for x < 0.
 *   R3  tan(gamma) = 2v/h at h = +-0 follows IEEE signed division:
 *       cos = 0, sin = copysign(1, tan).
 *   R4  sign(1, y) is copysign(1, y) (so -0 gives -1).
 *   R5  epsilon is the unit roundoff 2^-53 (double) / LDBL_EPSILON/2.
 *   R6  sqrt(n) in the skip test: n = number of columns at this level.
 *   R7  prescaling uses 1/||g_j|| = 1/sqrt(sum |g_rj|^2) (Sec. 3.3); the
 *       1/sqrt(||g_j||) printed in Sec. 2 does not make diag(B) = I.
 *   R8  Sigma_j = ||f_j|| / ||g_j||; the final sort is stable (ties keep
 *       the lower original column index first).
 *   R9  D-hat variants: the sort after a transformation compares the
 *       diagonal of Z-hat'^* A-hat' Z-hat' (= that of Z-hat^* A-hat Z-hat);
 *       the printed formula pairs the D-scaled Z-hat with A-hat', which is
 *       the same only when D-hat = I.  Without a transformation the sort
 *       compares a'_ii = a_ii / b_ii and a'_jj.
 *   R10 App. A: the product rounded toward -infinity is the largest value
 *       not above a b; it is taken from the round-to-nearest product p and
 *       its exact error a b - p (one fma), so no rounding-mode switch is
 *       needed.  Complex data: the norms use the simpler of the two
 *       enhanced procedures (the one the paper's variants use); the
 *       off-diagonal complex dot products stay ordinary (App. A defines no
 *       enhanced complex dot product).
 */
#include <complex.h>
#include <float.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

#ifdef HZO_EXTENDED
typedef long double real_t;
typedef long double _Complex cplx_t;
#define HZO(name) name##_ld
#define HZO_EPS (LDBL_EPSILON / 2.0L)
#else
typedef double real_t;
typedef double _Complex cplx_t;
#define HZO(name) name##_d
#define HZO_EPS (DBL_EPSILON / 2.0)
#endif

/* status codes of the oracle (its own definitions) */
#define HZO_OK 0
#define HZO_EINVAL (-1)
#define HZO_ENOCONV (-3)
#define HZO_ENOTPD (-4)

typedef struct {
    int32_t max_sweeps; /* sweep cap; exceeding it gives HZO_ENOCONV       */
    int32_t sort;       /* 1: per-step column sorting (Sec. 2.1)           */
    int32_t criterion;  /* 1: C1, 2: C2 (Sec. 2.5)                          */
    int32_t max_pivots; /* > 0: stop after this many pivot pairs (a bounded
                           timing sample; the result is then HZO_ENOCONV)  */
    int32_t enhanced;   /* 1: enhanced dot products (App. A; variant bit 1) */
    int32_t dscale;     /* 1: D-hat rescaling, no prescaling (bit 2)        */
} hzo_opts;

typedef struct {
    int32_t status;
    int32_t sweeps;     /* sweeps run, the last one without transformations */
    int64_t transf_all;
    int64_t transf_big;
    int32_t presorted;  /* 1: the final sort found the columns in order      */
    int32_t pad;
} hzo_stats;

/* sign(1, y) of the paper, reading R4 */
static real_t sgn1(real_t y) { return copysign((real_t)1, y); }

/* cos and sin from tan of an angle in (-pi/2, pi/2], readings R1 and R3 */
static void trig_from_tan(real_t tn, real_t *c, real_t *s)
{
    if (isinf(tn)) {
        *c = 0;
        *s = sgn1(tn);
    } else {
        *c = 1 / sqrt(1 + tn * tn);
        *s = tn * *c;
    }
}

/*
 * Real 2x2 transformation of Sec. 2.1.2.  Input: a11 = a_ii, a22 = a_jj,
 * a12 = a_ij, x = b_ij (B-hat has unit diagonal).  Output z[4] in row-major
 * order: z[0]=Z11, z[1]=Z12, z[2]=Z21, z[3]=Z22, and *small per criterion.
 * Returns HZO_ENOTPD if t^2 = 1 - x^2 is not positive.
 */
static int pivot_real(real_t a11, real_t a22, real_t a12, real_t x,
                      int criterion, real_t z[4], int *small)
{
    real_t t2 = 1 - x * x;
    if (!(t2 > 0)) return HZO_ENOTPD;
    real_t t = sqrt(t2);
    real_t num = t * (a22 - a11);
    real_t den = 2 * a12 - (a11 + a22) * x;
    if (num == 0 && den == 0) {
        /* exception: A-hat and B-hat proportional, reading R2 */
        real_t s = sgn1(x), ax = fabs(x), r2 = 1 / sqrt((real_t)2);
        real_t p = 1 / sqrt(1 + ax), q = 1 / sqrt(1 - ax);
        z[0] = r2 * p;
        z[1] = -r2 * s * q;
        z[2] = r2 * s * p;
        z[3] = r2 * q;
        /* C1 compares cos(phi)/t, C2 cos(phi); here no t appears */
        *small = (z[0] == 1 && z[3] == 1);
        return HZO_OK;
    }
    real_t xi = x / (sqrt(1 + x) + sqrt(1 - x));
    real_t eta = x / ((1 + sqrt(1 + x)) * (1 + sqrt(1 - x)));
    real_t cot2 = num / den; /* may be +-inf when den = +-0 */
    real_t tn;
    if (isinf(cot2))
        tn = sgn1(cot2) * (real_t)0; /* 1/inf, non-trapping */
    else
        tn = sgn1(cot2) / (fabs(cot2) + sqrt(1 + cot2 * cot2));
    real_t c, s;
    trig_from_tan(tn, &c, &s);
    real_t cphi = c + xi * (s - eta * c);
    real_t cpsi = c - xi * (s + eta * c);
    real_t sphi = s - xi * (c + eta * s);
    real_t spsi = s + xi * (c - eta * s);
    z[0] = cphi / t;
    z[1] = sphi / t;
    z[2] = -spsi / t;
    z[3] = cpsi / t;
    if (criterion == 2)
        *small = (cphi == 1 && cpsi == 1);
    else
        *small = (z[0] == 1 && z[3] == 1);
    return HZO_OK;
}

/*
 * Complex 2x2 transformation of Sec. 2.1.1.  Input: real a11, a22, complex
 * a12 = a_ij and b12 = b_ij.  Output z[4] row-major, as pivot_real.
 */
static int pivot_cplx(real_t a11, real_t a22, cplx_t a12, cplx_t b12,
                      int criterion, cplx_t z[4], int *small)
{
    real_t x = hypot(creal(b12), cimag(b12));
    real_t t2 = 1 - x * x;
    if (!(t2 > 0)) return HZO_ENOTPD;
    real_t t = sqrt(t2);
    /* e^{i zeta} = b12/|b12|, or 1 if b12 = 0 */
    cplx_t ez = (x == 0) ? (cplx_t)1 : b12 / x;
    cplx_t zz = conj(ez) * a12; /* z = e^{-i zeta} a_ij */
    real_t u = creal(zz), v = cimag(zz);
    real_t h = a22 - a11;
    if (v == 0 && h == 0) {
        /* exception of Sec. 2.1.1 */
        real_t r2 = 1 / sqrt((real_t)2);
        real_t p = 1 / sqrt(1 + x), q = 1 / sqrt(1 - x);
        z[0] = r2 * p;
        z[1] = -r2 * ez * q;
        z[2] = r2 * conj(ez) * p;
        z[3] = r2 * q;
        *small = (creal(z[0]) == 1 && creal(z[3]) == 1);
        return HZO_OK;
    }
    real_t tau = sgn1(h);
    real_t tan2 = tau * (2 * u - (a11 + a22) * x) / (t * sqrt(h * h + 4 * v * v));
    real_t tang = 2 * v / h; /* +-inf at h = +-0, reading R3 */
    real_t c2, s2, cg, sg;
    trig_from_tan(tan2, &c2, &s2);
    trig_from_tan(tang, &cg, &sg);
    real_t r2 = 1 / sqrt((real_t)2);
    real_t cphi = r2 * sqrt(1 + x * s2 + t * cg * c2);
    real_t cpsi = r2 * sqrt(1 - x * s2 + t * cg * c2);
    cplx_t easphi = ez * ((s2 - x) + I * (t * sg * c2)) / (2 * cpsi);
    cplx_t ebspsi = conj(ez) * ((s2 + x) - I * (t * sg * c2)) / (2 * cphi);
    z[0] = cphi / t;
    z[1] = easphi / t;
    z[2] = -ebspsi / t;
    z[3] = cpsi / t;
    if (criterion == 2)
        *small = (cphi == 1 && cpsi == 1);
    else
        *small = (creal(z[0]) == 1 && creal(z[3]) == 1);
    return HZO_OK;
}

/* exported 2x2 routines (for the invariant tests of the transformations) */
int HZO(hzo_pivot_real)(double a11, double a22, double a12, double x,
                        int32_t criterion, double zout[4], int32_t *small)
{
    real_t z[4];
    int sm = 0;
    int st = pivot_real(a11, a22, a12, x, criterion, z, &sm);
    for (int k = 0; k < 4; ++k) zout[k] = (double)z[k];
    *small = sm;
    return st;
}

int HZO(hzo_pivot_cplx)(double a11, double a22, const double a12[2],
                        const double b12[2], int32_t criterion,
                        double zout[8], int32_t *small)
{
    cplx_t z[4];
    int sm = 0;
    cplx_t ca = (real_t)a12[0] + I * (real_t)a12[1];
    cplx_t cb = (real_t)b12[0] + I * (real_t)b12[1];
    int st = pivot_cplx(a11, a22, ca, cb, criterion, z, &sm);
    for (int k = 0; k < 4; ++k) {
        zout[2 * k] = (double)creal(z[k]);
        zout[2 * k + 1] = (double)cimag(z[k]);
    }
    *small = sm;
    return st;
}

/*
 * D-hat of Sec. 2.1 (variants 2, 3, 6, 7), as the pivot step forms it: where
 * b_kk != 1, a'_kk = a_kk / b_kk, D_kk = 1/sqrt(b_kk), and the off-diagonal
 * a_ij, b_ij are multiplied by D_kk (first k = i, then k = j); elsewhere
 * D_kk = 1.  Then A-hat' = D A-hat D, B-hat' = D B-hat D (up to rounding).
 */
static void dscale_r(real_t bii, real_t bjj, real_t *aii, real_t *ajj, real_t *aij, real_t *x,
                     real_t *d1, real_t *d2)
{
    *d1 = 1;
    *d2 = 1;
    if (bii != 1) {
        *aii = *aii / bii;
        *d1 = 1 / sqrt(bii);
        *aij *= *d1;
        *x *= *d1;
    }
    if (bjj != 1) {
        *ajj = *ajj / bjj;
        *d2 = 1 / sqrt(bjj);
        *aij *= *d2;
        *x *= *d2;
    }
}

static void dscale_c(real_t bii, real_t bjj, real_t *aii, real_t *ajj, cplx_t *aij, cplx_t *bij,
                     real_t *d1, real_t *d2)
{
    *d1 = 1;
    *d2 = 1;
    if (bii != 1) {
        *aii = *aii / bii;
        *d1 = 1 / sqrt(bii);
        *aij *= *d1;
        *bij *= *d1;
    }
    if (bjj != 1) {
        *ajj = *ajj / bjj;
        *d2 = 1 / sqrt(bjj);
        *aij *= *d2;
        *bij *= *d2;
    }
}

/* Z-hat = D-hat Z-hat': the first row of Z-hat' (row-major z[0], z[1]) times
   D11, the second (z[2], z[3]) times D22 */
static void drows_r(real_t z[4], real_t d1, real_t d2)
{
    z[0] *= d1;
    z[1] *= d1;
    z[2] *= d2;
    z[3] *= d2;
}

static void drows_c(cplx_t z[4], real_t d1, real_t d2)
{
    z[0] *= d1;
    z[1] *= d1;
    z[2] *= d2;
    z[3] *= d2;
}

/* exported D-hat pivots: Z-hat = D-hat Z-hat', for the invariant tests
   Z^* B Z = I with b_ii, b_jj != 1 */
int HZO(hzo_pivot_real_dscaled)(double a11, double a22, double a12, double b11, double b22,
                                double b12, int32_t criterion, double zout[4], int32_t *small)
{
    real_t aii = a11, ajj = a22, aij = a12, x = b12, d1, d2, z[4];
    int sm = 0;
    dscale_r(b11, b22, &aii, &ajj, &aij, &x, &d1, &d2);
    int st = pivot_real(aii, ajj, aij, x, criterion, z, &sm);
    drows_r(z, d1, d2);
    for (int k = 0; k < 4; ++k) zout[k] = (double)z[k];
    *small = sm;
    return st;
}

int HZO(hzo_pivot_cplx_dscaled)(double a11, double a22, const double a12[2], double b11,
                                double b22, const double b12[2], int32_t criterion,
                                double zout[8], int32_t *small)
{
    real_t aii = a11, ajj = a22, d1, d2;
    cplx_t ca = (real_t)a12[0] + I * (real_t)a12[1];
    cplx_t cb = (real_t)b12[0] + I * (real_t)b12[1];
    cplx_t z[4];
    int sm = 0;
    dscale_c(b11, b22, &aii, &ajj, &ca, &cb, &d1, &d2);
    int st = pivot_cplx(aii, ajj, ca, cb, criterion, z, &sm);
    drows_c(z, d1, d2);
    for (int k = 0; k < 4; ++k) {
        zout[2 * k] = (double)creal(z[k]);
        zout[2 * k + 1] = (double)cimag(z[k]);
    }
    *small = sm;
    return st;
}

/* ------------------------------------------------- dot products (App. A) -- */

/* the product a b rounded toward -infinity, reading R10 */
static real_t mul_rd(real_t a, real_t b)
{
    real_t p = a * b;
    real_t e = fma(a, b, -p);
    return e < 0 ? nextafter(p, -INFINITY) : p;
}

/* enhanced real dot product: c_r = RD(a_r b_r), d_r = a_r b_r - c_r >= 0
   (exact, by one fma); the sum of the c_r plus the sum of the d_r */
static real_t dot_enh_rr(const real_t *a, const real_t *b, int64_t m)
{
    real_t sc = 0, sd = 0;
    for (int64_t r = 0; r < m; ++r) {
        real_t c = mul_rd(a[r], b[r]);
        sc += c;
        sd += fma(a[r], b[r], -c);
    }
    return sc + sd;
}

/* enhanced ||a||^2 of a complex vector, the simpler procedure of App. A:
   per element e = d_re + d_im, then (e + the smaller c) + the larger c */
static real_t nrm2sq_enh_c(const cplx_t *a, int64_t m)
{
    real_t s = 0;
    for (int64_t r = 0; r < m; ++r) {
        real_t re = creal(a[r]), im = cimag(a[r]);
        real_t cr = mul_rd(re, re), ci = mul_rd(im, im);
        real_t e = fma(re, re, -cr) + fma(im, im, -ci);
        s += (cr <= ci) ? (e + cr) + ci : (e + ci) + cr;
    }
    return s;
}

/* ---------------------------------------------------------------- real -- */

static real_t dot_rr(const real_t *a, const real_t *b, int64_t m)
{
    real_t s = 0;
    for (int64_t r = 0; r < m; ++r) s += a[r] * b[r];
    return s;
}

/* a^T b, ordinary or enhanced (variants 1, 3, 5, 7) */
static real_t dot_r(const hzo_opts *opt, const real_t *a, const real_t *b, int64_t m)
{
    return opt->enhanced ? dot_enh_rr(a, b, m) : dot_rr(a, b, m);
}

static void swap_cols_r(real_t *Y, int64_t m, int64_t i, int64_t j)
{
    for (int64_t r = 0; r < m; ++r) {
        real_t t = Y[i * m + r];
        Y[i * m + r] = Y[j * m + r];
        Y[j * m + r] = t;
    }
}

/* [y_i y_j] <- [y_i y_j] * Z-hat, Z-hat row-major z[4] (Sec. 2.1) */
static void rot_cols_r(real_t *Y, int64_t m, int64_t i, int64_t j, const real_t z[4])
{
    for (int64_t r = 0; r < m; ++r) {
        real_t yi = Y[i * m + r], yj = Y[j * m + r];
        Y[i * m + r] = yi * z[0] + yj * z[2];
        Y[j * m + r] = yi * z[1] + yj * z[3];
    }
}

/*
 * Real GSVD.  F (mf x n, ld ldf), G (mg x n, ld ldg): column-major doubles,
 * overwritten by U and V.  Z (n x n, ld ldz) written.  sf, sg, sigma:
 * length n.  Returns the status, also stored in st->status.
 */
int HZO(hzo_gsvd_real)(int64_t mf, int64_t mg, int64_t n,
                       double *F, int64_t ldf, double *G, int64_t ldg,
                       double *Z, int64_t ldz,
                       double *sf, double *sg, double *sigma,
                       const hzo_opts *opt, hzo_stats *st)
{
    memset(st, 0, sizeof *st);
    if (n < 1 || mf < n || mg < n || ldf < mf || ldg < mg || ldz < n) {
        st->status = HZO_EINVAL;
        return st->status;
    }
    real_t *f = malloc(sizeof(real_t) * mf * n);
    real_t *g = malloc(sizeof(real_t) * mg * n);
    real_t *z = calloc((size_t)(n * n), sizeof(real_t));
    real_t *nf = malloc(sizeof(real_t) * n), *ng = malloc(sizeof(real_t) * n);
    int64_t *perm = malloc(sizeof(int64_t) * n);
    int status = HZO_OK;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t r = 0; r < mf; ++r) f[j * mf + r] = F[j * ldf + r];
        for (int64_t r = 0; r < mg; ++r) g[j * mg + r] = G[j * ldg + r];
    }
    for (int64_t k = 0; k < mf * n; ++k)
        if (!isfinite(f[k])) status = HZO_EINVAL;
    for (int64_t k = 0; k < mg * n; ++k)
        if (!isfinite(g[k])) status = HZO_EINVAL;
    if (status != HZO_OK) goto done;

    /* prescaling: Z0 = diag(1/||g_j||), F0 = F Z0, G0 = G Z0 (reading R7);
       the D-hat variants start from Z0 = I */
    for (int64_t j = 0; j < n; ++j) {
        real_t s = dot_r(opt, &g[j * mg], &g[j * mg], mg);
        if (!(s > 0)) { status = HZO_ENOTPD; goto done; }
        if (opt->dscale) {
            z[j * n + j] = 1;
            continue;
        }
        real_t zj = 1 / sqrt(s);
        for (int64_t r = 0; r < mf; ++r) f[j * mf + r] *= zj;
        for (int64_t r = 0; r < mg; ++r) g[j * mg + r] *= zj;
        z[j * n + j] = zj;
    }

    const real_t tol = HZO_EPS * sqrt((real_t)n); /* eps * sqrt(n), R5, R6 */
    int converged = (n == 1);
    int sweep = 0;
    int64_t pivots = 0;
    while (!converged && sweep < opt->max_sweeps) {
        ++sweep;
        int64_t nall = 0, nbig = 0;
        for (int64_t i = 0; i < n - 1; ++i) {
            for (int64_t j = i + 1; j < n; ++j) {
                if (opt->max_pivots > 0 && pivots++ >= opt->max_pivots) {
                    st->transf_all += nall;
                    st->transf_big += nbig;
                    st->sweeps = sweep;
                    status = HZO_ENOCONV;
                    goto done;
                }
                real_t *fi = &f[i * mf], *fj = &f[j * mf];
                real_t *gi = &g[i * mg], *gj = &g[j * mg];
                real_t aii = dot_r(opt, fi, fi, mf);
                real_t ajj = dot_r(opt, fj, fj, mf);
                real_t aij = dot_r(opt, fi, fj, mf);
                real_t x = dot_r(opt, gi, gj, mg);
                real_t d1 = 1, d2 = 1;
                if (opt->dscale) {
                    real_t bii = dot_r(opt, gi, gi, mg), bjj = dot_r(opt, gj, gj, mg);
                    if (!(bii > 0) || !(bjj > 0)) { status = HZO_ENOTPD; goto done; }
                    dscale_r(bii, bjj, &aii, &ajj, &aij, &x, &d1, &d2);
                }
                /* relative orthogonality (Sec. 2.1) */
                if (fabs(aij) < sqrt(aii) * sqrt(ajj) * tol && fabs(x) < tol) {
                    if (opt->sort && aii < ajj) {
                        swap_cols_r(f, mf, i, j);
                        swap_cols_r(g, mg, i, j);
                        swap_cols_r(z, n, i, j);
                    }
                    continue;
                }
                real_t zh[4];
                int small;
                status = pivot_real(aii, ajj, aij, x, opt->criterion, zh, &small);
                if (status != HZO_OK) goto done;
                ++nall;
                nbig += !small;
                /* transformed diagonal of A-hat (Sec. 3.5.3, real case), reading R9 */
                real_t a1 = zh[0] * zh[0] * aii + 2 * zh[0] * zh[2] * aij + zh[2] * zh[2] * ajj;
                real_t a2 = zh[1] * zh[1] * aii + 2 * zh[3] * zh[1] * aij + zh[3] * zh[3] * ajj;
                drows_r(zh, d1, d2); /* Z-hat = D-hat Z-hat' */
                rot_cols_r(f, mf, i, j, zh);
                rot_cols_r(g, mg, i, j, zh);
                rot_cols_r(z, n, i, j, zh);
                if (opt->sort) {
                    if (a1 < a2) {
                        swap_cols_r(f, mf, i, j);
                        swap_cols_r(g, mg, i, j);
                        swap_cols_r(z, n, i, j);
                    }
                }
            }
        }
        st->transf_all += nall;
        st->transf_big += nbig;
        if (nall == 0) converged = 1;
    }
    st->sweeps = sweep;
    if (!converged) status = HZO_ENOCONV;

    /* final rescaling (Sec. 2.4) */
    for (int64_t j = 0; j < n; ++j) {
        nf[j] = sqrt(dot_r(opt, &f[j * mf], &f[j * mf], mf));
        ng[j] = sqrt(dot_r(opt, &g[j * mg], &g[j * mg], mg));
        perm[j] = j;
    }
    /* stable insertion sort of indices by descending Sigma (reading R8) */
    for (int64_t a = 1; a < n; ++a) {
        int64_t p = perm[a];
        real_t key = nf[p] / ng[p];
        int64_t b = a - 1;
        while (b >= 0 && nf[perm[b]] / ng[perm[b]] < key) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = p;
    }
    st->presorted = 1;
    for (int64_t k = 0; k < n; ++k) if (perm[k] != k) st->presorted = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = perm[k];
        real_t th = 1 / sqrt(nf[j] * nf[j] + ng[j] * ng[j]);
        for (int64_t r = 0; r < mf; ++r) F[k * ldf + r] = (double)(f[j * mf + r] / nf[j]);
        for (int64_t r = 0; r < mg; ++r) G[k * ldg + r] = (double)(g[j * mg + r] / ng[j]);
        for (int64_t r = 0; r < n; ++r) Z[k * ldz + r] = (double)(z[j * n + r] * th);
        sf[k] = (double)(nf[j] * th);
        sg[k] = (double)(ng[j] * th);
        sigma[k] = (double)(nf[j] / ng[j]);
    }
done:
    st->status = status;
    free(f); free(g); free(z); free(nf); free(ng); free(perm);
    return status;
}

/* ------------------------------------------------------------- complex -- */

/* a^* b, sequential */
static cplx_t dot_cc(const cplx_t *a, const cplx_t *b, int64_t m)
{
    cplx_t s = 0;
    for (int64_t r = 0; r < m; ++r) s += conj(a[r]) * b[r];
    return s;
}

/* ||a||^2 as a sum of |a_r|^2 = re^2 + im^2 */
static real_t nrm2sq_c(const cplx_t *a, int64_t m)
{
    real_t s = 0;
    for (int64_t r = 0; r < m; ++r) s += creal(a[r]) * creal(a[r]) + cimag(a[r]) * cimag(a[r]);
    return s;
}

/* ||a||^2, ordinary or enhanced (variants 1, 3, 5, 7) */
static real_t nrm2sq_cv(const hzo_opts *opt, const cplx_t *a, int64_t m)
{
    return opt->enhanced ? nrm2sq_enh_c(a, m) : nrm2sq_c(a, m);
}

static void swap_cols_c(cplx_t *Y, int64_t m, int64_t i, int64_t j)
{
    for (int64_t r = 0; r < m; ++r) {
        cplx_t t = Y[i * m + r];
        Y[i * m + r] = Y[j * m + r];
        Y[j * m + r] = t;
    }
}

static void rot_cols_c(cplx_t *Y, int64_t m, int64_t i, int64_t j, const cplx_t z[4])
{
    for (int64_t r = 0; r < m; ++r) {
        cplx_t yi = Y[i * m + r], yj = Y[j * m + r];
        Y[i * m + r] = yi * z[0] + yj * z[2];
        Y[j * m + r] = yi * z[1] + yj * z[3];
    }
}

/* Complex GSVD: F, G, Z interleaved (re, im) doubles, column-major. */
int HZO(hzo_gsvd_cplx)(int64_t mf, int64_t mg, int64_t n,
                       double *F, int64_t ldf, double *G, int64_t ldg,
                       double *Z, int64_t ldz,
                       double *sf, double *sg, double *sigma,
                       const hzo_opts *opt, hzo_stats *st)
{
    memset(st, 0, sizeof *st);
    if (n < 1 || mf < n || mg < n || ldf < mf || ldg < mg || ldz < n) {
        st->status = HZO_EINVAL;
        return st->status;
    }
    cplx_t *f = malloc(sizeof(cplx_t) * mf * n);
    cplx_t *g = malloc(sizeof(cplx_t) * mg * n);
    cplx_t *z = calloc((size_t)(n * n), sizeof(cplx_t));
    real_t *nf = malloc(sizeof(real_t) * n), *ng = malloc(sizeof(real_t) * n);
    int64_t *perm = malloc(sizeof(int64_t) * n);
    int status = HZO_OK;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t r = 0; r < mf; ++r)
            f[j * mf + r] = (real_t)F[2 * (j * ldf + r)] + I * (real_t)F[2 * (j * ldf + r) + 1];
        for (int64_t r = 0; r < mg; ++r)
            g[j * mg + r] = (real_t)G[2 * (j * ldg + r)] + I * (real_t)G[2 * (j * ldg + r) + 1];
    }
    for (int64_t k = 0; k < mf * n; ++k)
        if (!isfinite(creal(f[k])) || !isfinite(cimag(f[k]))) status = HZO_EINVAL;
    for (int64_t k = 0; k < mg * n; ++k)
        if (!isfinite(creal(g[k])) || !isfinite(cimag(g[k]))) status = HZO_EINVAL;
    if (status != HZO_OK) goto done;

    for (int64_t j = 0; j < n; ++j) {
        real_t s = nrm2sq_cv(opt, &g[j * mg], mg);
        if (!(s > 0)) { status = HZO_ENOTPD; goto done; }
        if (opt->dscale) {
            z[j * n + j] = 1;
            continue;
        }
        real_t zj = 1 / sqrt(s);
        for (int64_t r = 0; r < mf; ++r) f[j * mf + r] *= zj;
        for (int64_t r = 0; r < mg; ++r) g[j * mg + r] *= zj;
        z[j * n + j] = zj;
    }

    const real_t tol = HZO_EPS * sqrt((real_t)n);
    int converged = (n == 1);
    int sweep = 0;
    int64_t pivots = 0;
    while (!converged && sweep < opt->max_sweeps) {
        ++sweep;
        int64_t nall = 0, nbig = 0;
        for (int64_t i = 0; i < n - 1; ++i) {
            for (int64_t j = i + 1; j < n; ++j) {
                if (opt->max_pivots > 0 && pivots++ >= opt->max_pivots) {
                    st->transf_all += nall;
                    st->transf_big += nbig;
                    st->sweeps = sweep;
                    status = HZO_ENOCONV;
                    goto done;
                }
                cplx_t *fi = &f[i * mf], *fj = &f[j * mf];
                cplx_t *gi = &g[i * mg], *gj = &g[j * mg];
                real_t aii = nrm2sq_cv(opt, fi, mf);
                real_t ajj = nrm2sq_cv(opt, fj, mf);
                cplx_t aij = dot_cc(fi, fj, mf);
                cplx_t bij = dot_cc(gi, gj, mg);
                real_t d1 = 1, d2 = 1;
                if (opt->dscale) {
                    real_t bii = nrm2sq_cv(opt, gi, mg), bjj = nrm2sq_cv(opt, gj, mg);
                    if (!(bii > 0) || !(bjj > 0)) { status = HZO_ENOTPD; goto done; }
                    dscale_c(bii, bjj, &aii, &ajj, &aij, &bij, &d1, &d2);
                }
                real_t abs_a = hypot(creal(aij), cimag(aij));
                real_t abs_b = hypot(creal(bij), cimag(bij));
                if (abs_a < sqrt(aii) * sqrt(ajj) * tol && abs_b < tol) {
                    if (opt->sort && aii < ajj) {
                        swap_cols_c(f, mf, i, j);
                        swap_cols_c(g, mg, i, j);
                        swap_cols_c(z, n, i, j);
                    }
                    continue;
                }
                cplx_t zh[4];
                int small;
                status = pivot_cplx(aii, ajj, aij, bij, opt->criterion, zh, &small);
                if (status != HZO_OK) goto done;
                ++nall;
                nbig += !small;
                drows_c(zh, d1, d2); /* Z-hat = D-hat Z-hat' */
                rot_cols_c(f, mf, i, j, zh);
                rot_cols_c(g, mg, i, j, zh);
                rot_cols_c(z, n, i, j, zh);
                if (opt->sort) {
                    /* complex case: recompute the transformed norms (Sec. 3.5.3) */
                    if (nrm2sq_cv(opt, fi, mf) < nrm2sq_cv(opt, fj, mf)) {
                        swap_cols_c(f, mf, i, j);
                        swap_cols_c(g, mg, i, j);
                        swap_cols_c(z, n, i, j);
                    }
                }
            }
        }
        st->transf_all += nall;
        st->transf_big += nbig;
        if (nall == 0) converged = 1;
    }
    st->sweeps = sweep;
    if (!converged) status = HZO_ENOCONV;

    for (int64_t j = 0; j < n; ++j) {
        nf[j] = sqrt(nrm2sq_cv(opt, &f[j * mf], mf));
        ng[j] = sqrt(nrm2sq_cv(opt, &g[j * mg], mg));
        perm[j] = j;
    }
    for (int64_t a = 1; a < n; ++a) {
        int64_t p = perm[a];
        real_t key = nf[p] / ng[p];
        int64_t b = a - 1;
        while (b >= 0 && nf[perm[b]] / ng[perm[b]] < key) {
            perm[b + 1] = perm[b];
            --b;
        }
        perm[b + 1] = p;
    }
    st->presorted = 1;
    for (int64_t k = 0; k < n; ++k) if (perm[k] != k) st->presorted = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = perm[k];
        real_t th = 1 / sqrt(nf[j] * nf[j] + ng[j] * ng[j]);
        for (int64_t r = 0; r < mf; ++r) {
            cplx_t u = f[j * mf + r] / nf[j];
            F[2 * (k * ldf + r)] = (double)creal(u);
            F[2 * (k * ldf + r) + 1] = (double)cimag(u);
        }
        for (int64_t r = 0; r < mg; ++r) {
            cplx_t v = g[j * mg + r] / ng[j];
            G[2 * (k * ldg + r)] = (double)creal(v);
            G[2 * (k * ldg + r) + 1] = (double)cimag(v);
        }
        for (int64_t r = 0; r < n; ++r) {
            cplx_t w = z[j * n + r] * th;
            Z[2 * (k * ldz + r)] = (double)creal(w);
            Z[2 * (k * ldz + r) + 1] = (double)cimag(w);
        }
        sf[k] = (double)(nf[j] * th);
        sg[k] = (double)(ng[j] * th);
        sigma[k] = (double)(nf[j] / ng[j]);
    }
done:
    st->status = status;
    free(f); free(g); free(z); free(nf); free(ng); free(perm);
    return status;
}

/* exported dot products (for the closed-form pins of App. A) */
double HZO(hzo_dot_real)(const double *a, const double *b, int64_t m, int32_t enhanced)
{
    real_t *x = malloc(sizeof(real_t) * (m > 0 ? m : 1)), *y = malloc(sizeof(real_t) * (m > 0 ? m : 1));
    for (int64_t r = 0; r < m; ++r) {
        x[r] = a[r];
        y[r] = b[r];
    }
    real_t s = enhanced ? dot_enh_rr(x, y, m) : dot_rr(x, y, m);
    free(x);
    free(y);
    return (double)s;
}

double HZO(hzo_nrm2sq_cplx)(const double *a, int64_t m, int32_t enhanced)
{
    cplx_t *x = malloc(sizeof(cplx_t) * (m > 0 ? m : 1));
    for (int64_t r = 0; r < m; ++r) x[r] = (real_t)a[2 * r] + I * (real_t)a[2 * r + 1];
    real_t s = enhanced ? nrm2sq_enh_c(x, m) : nrm2sq_c(x, m);
    free(x);
    return (double)s;
}
