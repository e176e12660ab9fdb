// hz_device.cuh -- device-side building blocks of the implicit Hari-Zimmermann
// GSVD sweep engine for sm_103a: deterministic warp reductions, the 2x2
// transformation parameters (real and complex, FP64 or FP32), and small helpers.
//
// Paper: Novakovic & Singer, "Implicit Hari-Zimmermann algorithm for the
// generalized SVD on the GPUs" (arXiv 1909.00101).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hz {

// status codes (mirrors include/gsvd.h)
enum : int {
  ST_OK = 0,
  ST_EINVAL = -1,
  ST_ENOMEM = -2,
  ST_ENOCONV = -3,
  ST_ENOTPD = -4,
  ST_EOVERFLOW = -5,
  ST_ETIMEOUT = -6,
  ST_ECUDA = -7,
  ST_ETOOBIG = -8,
};

constexpr unsigned FULL = 0xffffffffu;

// Warp sum of one value by a fixed xor butterfly (every lane gets the same
// bits): Appendix C, with native 64-bit shuffles.
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Transposing butterfly: reduce 4 per-lane values with 2+1+1+1+1 = 6 adds
// instead of 20 (FP64 issue cost on sm_103a is per warp instruction, not per
// lane, so the plain butterfly on 4 values costs 3.3x more).  On return every
// lane holds all four sums in v[0..3]; the order of additions is fixed.
template <class T>
__device__ __forceinline__ void warp_sum4(T v[4]) {
  const int lane = threadIdx.x & 31;
  // stage 1 (offset 16): lanes < 16 keep (v0, v1), lanes >= 16 keep (v2, v3)
  const bool hi16 = lane & 16;
  T s0 = hi16 ? v[0] : v[2];
  T s1 = hi16 ? v[1] : v[3];
  T r0 = __shfl_xor_sync(FULL, s0, 16);
  T r1 = __shfl_xor_sync(FULL, s1, 16);
  T k0 = hi16 ? v[2] : v[0];
  T k1 = hi16 ? v[3] : v[1];
  k0 += r0;
  k1 += r1;
  // stage 2 (offset 8): keep one of the two
  const bool hi8 = lane & 8;
  T s = hi8 ? k0 : k1;
  T r = __shfl_xor_sync(FULL, s, 8);
  T k = hi8 ? k1 : k0;
  k += r;
  // stages 3..5: plain butterfly within groups of 8
  k += __shfl_xor_sync(FULL, k, 4);
  k += __shfl_xor_sync(FULL, k, 2);
  k += __shfl_xor_sync(FULL, k, 1);
  // lanes 0-7: sum0, 8-15: sum1, 16-23: sum2, 24-31: sum3
  v[0] = __shfl_sync(FULL, k, 0);
  v[1] = __shfl_sync(FULL, k, 8);
  v[2] = __shfl_sync(FULL, k, 16);
  v[3] = __shfl_sync(FULL, k, 24);
}

// Scalar helpers overloaded on double and float, so that the 2x2 parameters
// below can run in either precision with the same expression order.
__device__ __forceinline__ double sgn1(double y) { return copysign(1.0, y); }
__device__ __forceinline__ float sgn1(float y) { return copysignf(1.0f, y); }
__device__ __forceinline__ double p_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float p_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double p_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float p_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double p_hypot(double x, double y) { return hypot(x, y); }
__device__ __forceinline__ float p_hypot(float x, float y) { return hypotf(x, y); }
__device__ __forceinline__ double p_abs(double x) { return fabs(x); }
__device__ __forceinline__ float p_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double p_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float p_fma(float a, float b, float c) { return fmaf(a, b, c); }
// below lim() the square of a value may lose bits to underflow; up() is a
// power of two that brings such values back into the normal range
template <class T>
struct TinyScale;
template <>
struct TinyScale<double> {
  static __device__ __forceinline__ double lim() { return 0x1p-900; }
  static __device__ __forceinline__ double up() { return 0x1p+450; }
};
template <>
struct TinyScale<float> {
  static __device__ __forceinline__ float lim() { return 0x1p-100f; }
  static __device__ __forceinline__ float up() { return 0x1p+50f; }
};
// "rounds to 1 in FP32" (the small-transformation class of the FP32 sweeps)
__device__ __forceinline__ bool f32_is_one(double x) { return __double2float_rn(x) == 1.0f; }
__device__ __forceinline__ bool f32_is_one(float x) { return x == 1.0f; }

// cos and sin from tan of an angle in (-pi/2, pi/2]; tan = +-inf gives
// cos = 0, sin = +-1 (IEEE signed division decides the sign).
template <class T>
__device__ __forceinline__ void trig_from_tan(T tn, T& c, T& s) {
  if (isinf(tn)) {
    c = T(0);
    s = sgn1(tn);
  } else {
    c = p_rsqrt(p_fma(tn, tn, T(1)));
    s = tn * c;
  }
}

// Result of one 2x2 pivot: Z-hat (row-major), imaginary parts of the two
// off-diagonal entries for complex pivots (the diagonal is real), and flags.
template <class T>
struct PivotOutT {
  T z11, z12, z21, z22;
  T z12i, z21i;
  int flags;  // PV_* bits
};
using PivotOut = PivotOutT<double>;
enum : int { PV_ROT = 1, PV_BIG = 2, PV_SWAP = 4, PV_FAIL = 8 };

// Real pivot, Sec. 2.1.2, in two independent chains that can run on two
// warps (two SM sub-partitions) at once -- on sm_103a a lone warp issues one
// FP64 instruction per ~76 cycles, so the chain length sets the step latency:
//   chain A: skip test, t = sqrt(1 - x^2) (with 1/t), cot 2theta as num/den,
//            tan theta, cos theta, sin theta;
//   chain B: xi = x / (sqrt(1+x) + sqrt(1-x)) and
//            eta = x / ((1 + sqrt(1+x)) (1 + sqrt(1-x)));
//   combine: cos/sin of phi and psi, Z-hat, sorting and the small/big class.
// The chain below is the paper's, rearranged so that every square root and
// division is a reciprocal square root (the shortest FP64 sequence): 1/t and
// t from one rsqrt; with cot 2theta = num/den and r = 1/hypot(num, den),
// cos 2theta = |num| r and sin 2theta = sign(num) den r (the angle with
// |theta| <= pi/4 that sign(1, cot 2theta) / (|cot 2theta| + sqrt(1 +
// cot^2 2theta)) selects), then cos^2 theta = (1 + cos 2theta) / 2 and
// cos theta = q rsqrt(q), sin theta = sin 2theta rsqrt(q) / 2; sqrt(1 +- x)
// = (1 +- x) rsqrt(1 +- x); xi and eta from one rsqrt squared.
// T = double in the FP64 sweeps; T = float in the FP32 bulk sweeps, whose
// inputs (dot products of FP32 columns) carry FP32 errors anyway.
enum : int { RC_SKIP = 0, RC_ROT = 1, RC_EXC = 2, RC_FAIL = 3 };
template <class T>
struct RealChainAT {
  T rt, c, s;
  int mode;
};
using RealChainA = RealChainAT<double>;

// relative orthogonality (Sec. 2.1), |a12| < sqrt(a11) sqrt(a22) tol and
// |x| < tol.  FP64: compared in squares (no FP64 square roots); FP32: with
// square roots (cheap there), so that squares of small FP32 values cannot
// underflow.
__device__ __forceinline__ bool rel_orth(double a11, double a22, double a12, double x, double tol) {
  const double tol2 = tol * tol;
  return a12 * a12 < (a11 * a22) * tol2 && x * x < tol2;
}
__device__ __forceinline__ bool rel_orth(float a11, float a22, float a12, float x, float tol) {
  return fabsf(a12) < (sqrtf(a11) * sqrtf(a22)) * tol && fabsf(x) < tol;
}

template <class T>
__device__ __forceinline__ RealChainAT<T> real_chain_a(T a11, T a22, T a12, T x, T tol) {
  RealChainAT<T> r;
  r.rt = T(1); r.c = T(1); r.s = T(0);
  if (rel_orth(a11, a22, a12, x, tol)) {
    r.mode = RC_SKIP;
    return r;
  }
  const T t2 = p_fma(-x, x, T(1));
  if (!(t2 > T(0))) {
    r.mode = RC_FAIL;
    return r;
  }
  r.rt = p_rsqrt(t2);
  const T t = t2 * r.rt;
  const T num = t * (a22 - a11);
  const T den = T(2) * a12 - (a11 + a22) * x;
  if (num == T(0) && den == T(0)) {
    r.mode = RC_EXC;  // proportional pivots: cot 2theta = 0/0
    return r;
  }
  T h2 = p_fma(num, num, den * den);
  T nu = num, de = den;
  if (h2 < TinyScale<T>::lim()) {  // squares near underflow: scale by a power of two first
    nu = num * TinyScale<T>::up();
    de = den * TinyScale<T>::up();
    h2 = p_fma(nu, nu, de * de);
  }
  const T rh = p_rsqrt(h2);
  const T c2 = p_abs(nu) * rh;            // cos 2theta >= 0
  const T s2 = sgn1(num) * de * rh;       // sin 2theta
  const T q = p_fma(T(0.5), c2, T(0.5));  // cos^2 theta in [1/2, 1]
  const T rq = p_rsqrt(q);
  r.c = q * rq;
  r.s = T(0.5) * s2 * rq;
  r.mode = RC_ROT;
  return r;
}

template <class T>
__device__ __forceinline__ void real_chain_b(T x, T& xi, T& eta) {
  const T up = T(1) + x, um = T(1) - x;
  const T sp = up * p_rsqrt(up), sm = um * p_rsqrt(um);
  const T q1 = sp + sm, q2 = (T(1) + sp) * (T(1) + sm);
  const T rP = p_rsqrt(q1 * q2);
  const T rq = rP * rP;  // 1 / (q1 q2)
  xi = x * q2 * rq;
  eta = x * q1 * rq;
}

template <class T>
__device__ __forceinline__ PivotOutT<T> real_combine(T a11, T a22, T a12, T x, const RealChainAT<T>& r, T xi,
                                                     T eta, bool sort, bool f32cls, bool crit2) {
  PivotOutT<T> o;
  o.z12i = o.z21i = T(0);
  o.flags = 0;
  o.z11 = T(1); o.z12 = T(0); o.z21 = T(0); o.z22 = T(1);
  if (r.mode == RC_SKIP) {
    if (sort && a11 < a22) o.flags |= PV_SWAP;
    return o;
  }
  if (r.mode == RC_FAIL) {
    o.flags = PV_FAIL;
    return o;
  }
  T cphi, cpsi;
  if (r.mode == RC_EXC) {
    // signed form of the exception (reading of Sec. 2.1.2)
    const T s = sgn1(x), ax = p_abs(x);
    const T p = p_rsqrt(T(2) * (T(1) + ax)), q = p_rsqrt(T(2) * (T(1) - ax));
    o.z11 = p; o.z12 = -s * q; o.z21 = s * p; o.z22 = q;
    cphi = o.z11; cpsi = o.z22;  // no t in this form
  } else {
    const T c = r.c, s = r.s;
    cphi = c + xi * (s - eta * c);
    cpsi = c - xi * (s + eta * c);
    const T sphi = s - xi * (c + eta * s);
    const T spsi = s + xi * (c - eta * s);
    o.z11 = cphi * r.rt;
    o.z12 = sphi * r.rt;
    o.z21 = -spsi * r.rt;
    o.z22 = cpsi * r.rt;
  }
  o.flags = PV_ROT;
  bool small;
  if (crit2 && r.mode == RC_ROT)
    small = f32cls ? (f32_is_one(cphi) && f32_is_one(cpsi)) : (cphi == T(1) && cpsi == T(1));
  else
    small = f32cls ? (f32_is_one(o.z11) && f32_is_one(o.z22)) : (o.z11 == T(1) && o.z22 == T(1));
  if (!small) o.flags |= PV_BIG;
  if (sort) {
    // transformed diagonal of A-hat (Sec. 3.5.3, real case)
    const T d1 = o.z11 * o.z11 * a11 + T(2) * o.z11 * o.z21 * a12 + o.z21 * o.z21 * a22;
    const T d2 = o.z12 * o.z12 * a11 + T(2) * o.z22 * o.z12 * a12 + o.z22 * o.z22 * a22;
    if (d1 < d2) o.flags |= PV_SWAP;
  }
  return o;
}

// Real pivot on one thread (both chains in sequence); the same arithmetic as
// the two-warp form, so both give identical bits.
template <class T>
__device__ __forceinline__ PivotOutT<T> pivot_real(T a11, T a22, T a12, T x, T tol, bool sort, bool f32cls,
                                                   bool crit2) {
  const RealChainAT<T> r = real_chain_a(a11, a22, a12, x, tol);
  T xi = T(0), eta = T(0);
  if (r.mode == RC_ROT) real_chain_b(x, xi, eta);
  return real_combine(a11, a22, a12, x, r, xi, eta, sort, f32cls, crit2);
}

// App. A: c = RD(a b), d = a b - c >= 0 (exact, one fma); the enhanced dot
// product is the sum of the c plus the sum of the d
__device__ __forceinline__ void enh_acc(double& c, double& d, double a, double b) {
  const double p = __dmul_rd(a, b);
  c += p;
  d += fma(a, b, -p);
}

// App. A, the simpler procedure for ||a||^2 of complex data: one element's
// term (e + the smaller c) + the larger c, e = d_re + d_im
__device__ __forceinline__ double enh_abs2(double re, double im) {
  const double cr = __dmul_rd(re, re), ci = __dmul_rd(im, im);
  const double e = fma(re, re, -cr) + fma(im, im, -ci);
  return cr <= ci ? (e + cr) + ci : (e + ci) + cr;
}

// Named barrier for the two parameter warps (barrier 1, 64 threads).
__device__ __forceinline__ void param_pair_barrier() { asm volatile("bar.sync 1, 64;\n" ::: "memory"); }

// Complex pivot, Sec. 2.1.1.  a12 = (ar, ai), b12 = (br, bi).
__device__ __forceinline__ bool rel_orth_c(double a11, double a22, double absa2, double x2, double tol) {
  const double tol2 = tol * tol;
  return absa2 < (a11 * a22) * tol2 && x2 < tol2;
}
__device__ __forceinline__ bool rel_orth_c(float a11, float a22, float absa2, float x2, float tol) {
  return sqrtf(absa2) < (sqrtf(a11) * sqrtf(a22)) * tol && sqrtf(x2) < tol;
}

template <class T>
__device__ __forceinline__ PivotOutT<T> pivot_cplx(T a11, T a22, T ar, T ai, T br, T bi, T tol, bool sort,
                                                   bool f32cls, bool crit2) {
  PivotOutT<T> o;
  o.flags = 0;
  // relative orthogonality: |a12|^2 < a11 a22 tol^2, |b12|^2 < tol^2
  const T absa2 = p_fma(ar, ar, ai * ai);
  const T x2 = p_fma(br, br, bi * bi);
  if (rel_orth_c(a11, a22, absa2, x2, tol)) {
    o.z11 = T(1); o.z12 = T(0); o.z21 = T(0); o.z22 = T(1); o.z12i = T(0); o.z21i = T(0);
    if (sort && a11 < a22) o.flags |= PV_SWAP;
    return o;
  }
  const T x = p_hypot(br, bi);
  const T t2 = p_fma(-x, x, T(1));
  if (!(t2 > T(0))) {
    o.z11 = T(1); o.z12 = T(0); o.z21 = T(0); o.z22 = T(1); o.z12i = T(0); o.z21i = T(0);
    o.flags = PV_FAIL;
    return o;
  }
  const T rt = p_rsqrt(t2);
  const T t = t2 * rt;
  // e^{i zeta} = b12 / |b12| (1 if b12 = 0); z = e^{-i zeta} a12
  T er = T(1), ei = T(0);
  if (x != T(0)) {
    const T rx = T(1) / x;
    er = br * rx;
    ei = bi * rx;
  }
  const T u = er * ar + ei * ai;
  const T v = er * ai - ei * ar;
  const T h = a22 - a11;
  T cphi, cpsi;
  if (v == T(0) && h == T(0)) {
    const T p = p_rsqrt(T(2) * (T(1) + x)), q = p_rsqrt(T(2) * (T(1) - x));
    o.z11 = p; o.z22 = q;
    o.z12 = -er * q; o.z12i = -ei * q;   // -e^{i zeta} q
    o.z21 = er * p;  o.z21i = -ei * p;   //  e^{-i zeta} p
    cphi = o.z11; cpsi = o.z22;
    o.flags = PV_ROT;
    const bool small = f32cls ? (f32_is_one(o.z11) && f32_is_one(o.z22)) : (o.z11 == T(1) && o.z22 == T(1));
    if (!small) o.flags |= PV_BIG;
  } else {
    const T tau = sgn1(h);
    const T tan2 = tau * (T(2) * u - (a11 + a22) * x) / (t * p_sqrt(p_fma(h, h, T(4) * v * v)));
    const T tang = T(2) * v / h;
    T c2, s2, cg, sg;
    trig_from_tan(tan2, c2, s2);
    trig_from_tan(tang, cg, sg);
    const T tcc = t * cg * c2;
    cphi = p_sqrt(T(0.5) * (T(1) + x * s2 + tcc));
    cpsi = p_sqrt(T(0.5) * (T(1) - x * s2 + tcc));
    const T w = t * sg * c2;
    // 1/(2 cos psi) and 1/(2 cos phi) from one reciprocal
    const T r4 = T(1) / (T(4) * cphi * cpsi);
    const T ipsi = T(2) * cphi * r4, iphi = T(2) * cpsi * r4;
    // e^{i alpha} sin(phi) = e^{i zeta} ((s2 - x) + i w) / (2 cos psi)
    const T pa = (s2 - x) * ipsi, qa = w * ipsi;
    // e^{-i beta} sin(psi) = e^{-i zeta} ((s2 + x) - i w) / (2 cos phi)
    const T pb = (s2 + x) * iphi, qb = -w * iphi;
    o.z11 = cphi * rt;
    o.z22 = cpsi * rt;
    o.z12 = (er * pa - ei * qa) * rt;
    o.z12i = (er * qa + ei * pa) * rt;
    // -(e^{-i zeta})(pb + i qb) with e^{-i zeta} = (er, -ei)
    o.z21 = -(er * pb + ei * qb) * rt;
    o.z21i = -(er * qb - ei * pb) * rt;
    o.flags = PV_ROT;
    bool small;
    if (crit2)
      small = f32cls ? (f32_is_one(cphi) && f32_is_one(cpsi)) : (cphi == T(1) && cpsi == T(1));
    else
      small = f32cls ? (f32_is_one(o.z11) && f32_is_one(o.z22)) : (o.z11 == T(1) && o.z22 == T(1));
    if (!small) o.flags |= PV_BIG;
  }
  if (sort) {
    // transformed diagonal of A-hat: (Z^* A Z)_11 and _22, Z11 and Z22 real
    const T re21a = o.z21 * ar - o.z21i * ai;          // Re(a12 * z21)
    const T d1 = o.z11 * o.z11 * a11 + T(2) * o.z11 * re21a + (o.z21 * o.z21 + o.z21i * o.z21i) * a22;
    const T re12a = o.z12 * ar + o.z12i * ai;          // Re(conj(z12) * a12)
    const T d2 = (o.z12 * o.z12 + o.z12i * o.z12i) * a11 + T(2) * o.z22 * re12a + o.z22 * o.z22 * a22;
    if (d1 < d2) o.flags |= PV_SWAP;
  }
  return o;
}

// Round-robin ("circle method") pair k of step s for M (even) players:
// player M-1 stays, the others rotate; returns (p, q) with p < q.
__device__ __host__ __forceinline__ void rr_pair(int M, int s, int k, int& p, int& q) {
  int a, b;
  if (k == 0) {
    a = M - 1;
    b = s;
  } else {
    a = (s + k) % (M - 1);
    b = (s - k + (M - 1)) % (M - 1);
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

}  // namespace hz
