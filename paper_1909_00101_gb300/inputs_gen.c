/*
 * inputs_gen.c -- seeded synthetic GSVD input pairs, bit-identical on every
 * IEEE-754 machine (x86-64 and AArch64 alike).
 *
 * This file holds none of the Hari-Zimmermann method's arithmetic; it only
 * builds inputs.  It exists so that an input pair drawn on one machine is the
 * same bytes on another, which lets reference values computed once (slowly,
 * on a CPU) be checked against a solve of the same pair elsewhere.  To that
 * end every floating-point result here is produced by a fixed sequence of
 * IEEE-754 additions, multiplications, divisions and square roots (all
 * correctly rounded): no libm transcendental, no BLAS/LAPACK, no fused
 * multiply-add (the file is compiled with -ffp-contract=off), no reduction
 * whose order depends on the thread count.  Threads only split independent
 * output entries between them.
 *
 * Pieces:
 *   - xoshiro256** (Blackman & Vigna 2018) seeded by splitmix64 (Steele,
 *     Lea & Flood 2014), one stream per (seed, stream id);
 *   - uniform doubles (x >> 11) * 2^-53;
 *   - standard normal deviates by Marsaglia's polar method (1964);
 *   - ln and exp by argument reduction and truncated series written out
 *     below (accurate to a few ulps, and above all deterministic);
 *   - orthonormal columns by classical Gram-Schmidt with one
 *     re-orthogonalisation (CGS2) of a Gaussian matrix: Q = A R^-1 with a
 *     positive diagonal of R, which is Haar distributed (Mezzadri 2007);
 *   - products C = A B with every entry summed over k in increasing order.
 *
 * Matrices are column-major; complex data are interleaved (re, im) pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG */

typedef struct { uint64_t s[4]; } ig_rng;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_init(ig_rng *r, uint64_t seed, uint64_t stream)
{
    uint64_t x = seed * 0xD1B54A32D192ED03ull + stream * 0x8CB92BA72F3D8DD7ull + 0x632BE59BD9B4E019ull;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static uint64_t rng_next(ig_rng *r)
{
    uint64_t *s = r->s;
    uint64_t out = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return out;
}

static double rng_uniform(ig_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* ------------------------------------------------ deterministic ln, exp */

static const double LN2 = 0.69314718055994530942;

/* ln(x), x > 0 finite: x = 2^e * t with t in [sqrt(1/2), sqrt(2)), then
 * ln t = 2 atanh(s), s = (t - 1)/(t + 1), |s| < 0.1716, by its series to s^25. */
double ig_log(double x)
{
    int e;
    double t = frexp(x, &e);          /* exact: t in [0.5, 1) */
    if (t < 0.70710678118654752440) { t = t * 2.0; e -= 1; }
    double s = (t - 1.0) / (t + 1.0);
    double s2 = s * s;
    double sum = 0.0;
    for (int k = 25; k >= 1; k -= 2) sum = sum * s2 + 1.0 / (double)k;   /* Horner in s^2 */
    return (double)e * LN2 + 2.0 * s * sum;
}

/* exp(y): y = k ln2 + r with |r| <= ln2/2 (k = nearest integer), e^r by its
 * Taylor series to r^20 (Horner), then scaled by 2^k (exact). */
double ig_exp(double y)
{
    if (y > 709.0) return HUGE_VAL;
    if (y < -745.0) return 0.0;
    double kf = floor(y / LN2 + 0.5);
    double r = y - kf * LN2;
    double sum = 1.0;
    for (int k = 20; k >= 1; --k) sum = 1.0 + sum * r / (double)k;
    return ldexp(sum, (int)kf);
}

/* ---------------------------------------------------------- generators */

void ig_uniform(uint64_t seed, uint64_t stream, int64_t count, double *out)
{
    ig_rng r;
    rng_init(&r, seed, stream);
    for (int64_t i = 0; i < count; ++i) out[i] = rng_uniform(&r);
}

/* Standard normal deviates, Marsaglia's polar method, in stream order. */
void ig_gauss(uint64_t seed, uint64_t stream, int64_t count, double *out)
{
    ig_rng r;
    rng_init(&r, seed, stream);
    int64_t i = 0;
    while (i < count) {
        double u = 2.0 * rng_uniform(&r) - 1.0;
        double v = 2.0 * rng_uniform(&r) - 1.0;
        double s = u * u + v * v;
        if (s >= 1.0 || s == 0.0) continue;
        double f = sqrt(-2.0 * ig_log(s) / s);
        out[i++] = u * f;
        if (i < count) out[i++] = v * f;
    }
}

/* A uniformly random permutation of 0..n-1 (Fisher-Yates; the index is the
 * high 64 bits of a 64 x 64-bit product, bias below 2^-40 for n < 2^24). */
void ig_permutation(uint64_t seed, uint64_t stream, int64_t n, int64_t *perm)
{
    ig_rng r;
    rng_init(&r, seed, stream);
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t i = n - 1; i > 0; --i) {
        unsigned __int128 p = (unsigned __int128)rng_next(&r) * (unsigned __int128)(uint64_t)(i + 1);
        int64_t j = (int64_t)(uint64_t)(p >> 64);
        int64_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* out[i] = exp(ln lo + (ln hi - ln lo) i / (n - 1)), i = 0..n-1 (n >= 2). */
void ig_logspace(double lo, double hi, int64_t n, double *out)
{
    double a = ig_log(lo), b = ig_log(hi);
    for (int64_t i = 0; i < n; ++i) out[i] = ig_exp(a + (b - a) * (double)i / (double)(n - 1));
}

/* ---------------------------------------------------- linear algebra */

static void set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

/* Orthonormalise the n columns of the m x n matrix A (ld = m) in place by
 * CGS2: two passes of a_j -= Q_{<j} (Q_{<j}^* a_j), then a_j /= ||a_j||.
 * Returns 0, or -1 if a column vanishes (rank deficiency). */
int ig_orthonormalize(int64_t m, int64_t n, double *A, int32_t cplx, int32_t threads)
{
    const int64_t es = cplx ? 2 : 1;      /* doubles per entry */
    const int64_t ld = m * es;
    const int64_t RB = 256;               /* row chunk of the update */
    double *r = (double *)malloc(sizeof(double) * (size_t)(n * es + 1));
    if (!r) return -2;
    int bad = 0;
    set_threads(threads);
#pragma omp parallel
    for (int64_t j = 0; j < n; ++j) {
        double *a = A + j * ld;
        for (int pass = 0; pass < 2; ++pass) {
#pragma omp for schedule(static)
            for (int64_t k = 0; k < j; ++k) {
                const double *q = A + k * ld;
                if (!cplx) {
                    double s = 0.0;
                    for (int64_t i = 0; i < m; ++i) s = s + q[i] * a[i];
                    r[k] = s;
                } else {
                    double sr = 0.0, si = 0.0;
                    for (int64_t i = 0; i < m; ++i) {
                        double qr = q[2 * i], qi = q[2 * i + 1], ar = a[2 * i], ai = a[2 * i + 1];
                        sr = sr + (qr * ar + qi * ai);
                        si = si + (qr * ai - qi * ar);
                    }
                    r[2 * k] = sr;
                    r[2 * k + 1] = si;
                }
            }
#pragma omp for schedule(static)
            for (int64_t i0 = 0; i0 < m; i0 += RB) {
                int64_t i1 = i0 + RB < m ? i0 + RB : m;
                for (int64_t k = 0; k < j; ++k) {
                    const double *q = A + k * ld;
                    if (!cplx) {
                        double rk = r[k];
                        for (int64_t i = i0; i < i1; ++i) a[i] = a[i] - q[i] * rk;
                    } else {
                        double rr = r[2 * k], ri = r[2 * k + 1];
                        for (int64_t i = i0; i < i1; ++i) {
                            double qr = q[2 * i], qi = q[2 * i + 1];
                            a[2 * i] = a[2 * i] - (qr * rr - qi * ri);
                            a[2 * i + 1] = a[2 * i + 1] - (qr * ri + qi * rr);
                        }
                    }
                }
            }
        }
#pragma omp single
        {
            double s = 0.0;
            for (int64_t i = 0; i < m * es; ++i) s = s + a[i] * a[i];
            double nrm = sqrt(s);
            if (!(nrm > 0.0)) bad = 1;
            else for (int64_t i = 0; i < m * es; ++i) a[i] = a[i] / nrm;
        }
    }
    free(r);
    return bad ? -1 : 0;
}

/* A(:, j) *= s[j] for the m x n matrix A (real scale, real or complex A). */
void ig_scale_cols(int64_t m, int64_t n, double *A, int64_t lda, const double *s, int32_t cplx)
{
    const int64_t es = cplx ? 2 : 1;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m * es; ++i) A[j * lda * es + i] = A[j * lda * es + i] * s[j];
}

/* C = A B (A m x k, B k x n, C m x n), every entry summed over k in
 * increasing order starting from zero; threads split the columns of C. */
void ig_gemm(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B, int64_t ldb,
             double *C, int64_t ldc, int32_t cplx, int32_t threads)
{
    const int64_t es = cplx ? 2 : 1;
    const int64_t NB = 8;
    set_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j0 = 0; j0 < n; j0 += NB) {
        int64_t j1 = j0 + NB < n ? j0 + NB : n;
        for (int64_t j = j0; j < j1; ++j) memset(C + j * ldc * es, 0, sizeof(double) * (size_t)(m * es));
        for (int64_t kk = 0; kk < k; ++kk) {
            const double *a = A + kk * lda * es;
            for (int64_t j = j0; j < j1; ++j) {
                double *c = C + j * ldc * es;
                if (!cplx) {
                    double b = B[j * ldb + kk];
                    for (int64_t i = 0; i < m; ++i) c[i] = c[i] + a[i] * b;
                } else {
                    double br = B[2 * (j * ldb + kk)], bi = B[2 * (j * ldb + kk) + 1];
                    for (int64_t i = 0; i < m; ++i) {
                        double ar = a[2 * i], ai = a[2 * i + 1];
                        c[2 * i] = c[2 * i] + (ar * br - ai * bi);
                        c[2 * i + 1] = c[2 * i + 1] + (ar * bi + ai * br);
                    }
                }
            }
        }
    }
}
