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
 *   - variant 0 of Table "Variants" (Sec. 2.6): prescaling of F, G by
 *     Z0 = diag(1/||g_j||) (Sec. 2, "It is assumed that diag(B) = I"),
 *     pivot B-hat taken with unit diagonal, ordinary dot products;
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
} hzo_opts;

typedef struct {
    int32_t status;
    int32_t sweeps;     /* sweeps run, the last one without transformations */
    int64_t transf_all;
    int64_t transf_big;
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

/* ---------------------------------------------------------------- real -- */

static real_t dot_rr(const real_t *a, const real_t *b, int64_t m)
{
    real_t s = 0;
    for (int64_t r = 0; r < m; ++r) s += a[r] * b[r];
    return s;
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

    /* prescaling: Z0 = diag(1/||g_j||), F0 = F Z0, G0 = G Z0 (reading R7) */
    for (int64_t j = 0; j < n; ++j) {
        real_t s = dot_rr(&g[j * mg], &g[j * mg], mg);
        if (!(s > 0)) { status = HZO_ENOTPD; goto done; }
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
                real_t aii = dot_rr(fi, fi, mf);
                real_t ajj = dot_rr(fj, fj, mf);
                real_t aij = dot_rr(fi, fj, mf);
                real_t x = dot_rr(gi, gj, mg);
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
                rot_cols_r(f, mf, i, j, zh);
                rot_cols_r(g, mg, i, j, zh);
                rot_cols_r(z, n, i, j, zh);
                if (opt->sort) {
                    /* transformed diagonal of A-hat (Sec. 3.5.3, real case) */
                    real_t a1 = zh[0] * zh[0] * aii + 2 * zh[0] * zh[2] * aij + zh[2] * zh[2] * ajj;
                    real_t a2 = zh[1] * zh[1] * aii + 2 * zh[3] * zh[1] * aij + zh[3] * zh[3] * ajj;
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
        nf[j] = sqrt(dot_rr(&f[j * mf], &f[j * mf], mf));
        ng[j] = sqrt(dot_rr(&g[j * mg], &g[j * mg], mg));
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
        real_t s = nrm2sq_c(&g[j * mg], mg);
        if (!(s > 0)) { status = HZO_ENOTPD; goto done; }
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
                real_t aii = nrm2sq_c(fi, mf);
                real_t ajj = nrm2sq_c(fj, mf);
                cplx_t aij = dot_cc(fi, fj, mf);
                cplx_t bij = dot_cc(gi, gj, mg);
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
                rot_cols_c(f, mf, i, j, zh);
                rot_cols_c(g, mg, i, j, zh);
                rot_cols_c(z, n, i, j, zh);
                if (opt->sort) {
                    /* complex case: recompute the transformed norms (Sec. 3.5.3) */
                    if (nrm2sq_c(fi, mf) < nrm2sq_c(fj, mf)) {
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
        nf[j] = sqrt(nrm2sq_c(&f[j * mf], mf));
        ng[j] = sqrt(nrm2sq_c(&g[j * mg], mg));
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
