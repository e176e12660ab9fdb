// hz_device.cuh -- device-side building blocks of the implicit Hari-Zimmermann
// GSVD sweep engine for sm_103a: deterministic warp reductions, the FP64 2x2
// transformation parameters (real and complex), and small helpers.
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
  // round 1 (offset 16): lanes < 16 keep (v0, v1), lanes >= 16 keep (v2, v3)
  const bool hi16 = lane & 16;
  T s0 = hi16 ? v[0] : v[2];
  T s1 = hi16 ? v[1] : v[3];
  T r0 = __shfl_xor_sync(FULL, s0, 16);
  T r1 = __shfl_xor_sync(FULL, s1, 16);
  T k0 = hi16 ? v[2] : v[0];
  T k1 = hi16 ? v[3] : v[1];
  k0 += r0;
  k1 += r1;
  // round 2 (offset 8): keep one of the two
  const bool hi8 = lane & 8;
  T s = hi8 ? k0 : k1;
  T r = __shfl_xor_sync(FULL, s, 8);
  T k = hi8 ? k1 : k0;
  k += r;
  // rounds 3..5: plain butterfly within groups of 8
  k += __shfl_xor_sync(FULL, k, 4);
  k += __shfl_xor_sync(FULL, k, 2);
  k += __shfl_xor_sync(FULL, k, 1);
  // lanes 0-7: sum0, 8-15: sum1, 16-23: sum2, 24-31: sum3
  v[0] = __shfl_sync(FULL, k, 0);
  v[1] = __shfl_sync(FULL, k, 8);
  v[2] = __shfl_sync(FULL, k, 16);
  v[3] = __shfl_sync(FULL, k, 24);
}

__device__ __forceinline__ double sgn1(double y) { return copysign(1.0, y); }

// cos and sin from tan of an angle in (-pi/2, pi/2]; tan = +-inf gives
// cos = 0, sin = +-1 (IEEE signed division decides the sign).
__device__ __forceinline__ void trig_from_tan(double tn, double& c, double& s) {
  if (isinf(tn)) {
    c = 0.0;
    s = sgn1(tn);
  } else {
    c = rsqrt(fma(tn, tn, 1.0));
    s = tn * c;
  }
}

// Result of one 2x2 pivot: Z-hat (row-major), imaginary parts of the two
// off-diagonal entries for complex pivots (the diagonal is real), and flags.
struct PivotOut {
  double z11, z12, z21, z22;
  double z12i, z21i;
  int flags;  // PV_* bits
};
enum : int { PV_ROT = 1, PV_BIG = 2, PV_SWAP = 4, PV_FAIL = 8 };

// Real pivot, Sec. 2.1.2, in two independent FP64 chains that can run on two
// warps (two SM sub-partitions) at once -- on sm_103a a lone warp issues one
// FP64 instruction per ~76 cycles, so the chain length sets the step latency:
//   chain A: skip test, t = sqrt(1 - x^2) (with 1/t), cot 2theta as num/den,
//            tan theta, cos theta, sin theta;
//   chain B: xi = x / (sqrt(1+x) + sqrt(1-x)) and
//            eta = x / ((1 + sqrt(1+x)) (1 + sqrt(1-x)));
//   combine: cos/sin of phi and psi, Z-hat, sorting and the small/big class.
// The chain below is the paper's, rearranged to need 7 instead of 11 square
// roots and divisions: 1/t and t from one rsqrt; xi and eta from one
// reciprocal; tan theta = sign(1, cot 2theta) / (|cot 2theta| +
// sqrt(1 + cot^2 2theta)) written on num/den without forming the cotangent:
// sign(num) den / (|num| + hypot(num, den)).
enum : int { RC_SKIP = 0, RC_ROT = 1, RC_EXC = 2, RC_FAIL = 3 };
struct RealChainA {
  double rt, c, s;
  int mode;
};

__device__ __forceinline__ RealChainA real_chain_a(double a11, double a22, double a12, double x, double tol) {
  RealChainA r;
  r.rt = 1.0; r.c = 1.0; r.s = 0.0;
  // relative orthogonality (Sec. 2.1), |a12| < sqrt(a11) sqrt(a22) tol and
  // |x| < tol, compared in squares (no FP64 square roots)
  const double tol2 = tol * tol;
  if (a12 * a12 < (a11 * a22) * tol2 && x * x < tol2) {
    r.mode = RC_SKIP;
    return r;
  }
  const double t2 = fma(-x, x, 1.0);
  if (!(t2 > 0.0)) {
    r.mode = RC_FAIL;
    return r;
  }
  r.rt = rsqrt(t2);
  const double t = t2 * r.rt;
  const double num = t * (a22 - a11);
  const double den = 2.0 * a12 - (a11 + a22) * x;
  if (num == 0.0 && den == 0.0) {
    r.mode = RC_EXC;  // proportional pivots: cot 2theta = 0/0
    return r;
  }
  const double hyp = sqrt(fma(num, num, den * den));
  const double tn = sgn1(num) * den / (fabs(num) + hyp);
  r.c = rsqrt(fma(tn, tn, 1.0));
  r.s = tn * r.c;
  r.mode = RC_ROT;
  return r;
}

__device__ __forceinline__ void real_chain_b(double x, double& xi, double& eta) {
  const double sp = sqrt(1.0 + x), sm = sqrt(1.0 - x);
  const double q1 = sp + sm, q2 = (1.0 + sp) * (1.0 + sm);
  const double rq = 1.0 / (q1 * q2);
  xi = x * q2 * rq;
  eta = x * q1 * rq;
}

__device__ __forceinline__ PivotOut real_combine(double a11, double a22, double a12, double x,
                                                 const RealChainA& r, double xi, double eta, bool sort,
                                                 bool f32cls, bool crit2) {
  PivotOut o;
  o.z12i = o.z21i = 0.0;
  o.flags = 0;
  o.z11 = 1.0; o.z12 = 0.0; o.z21 = 0.0; o.z22 = 1.0;
  if (r.mode == RC_SKIP) {
    if (sort && a11 < a22) o.flags |= PV_SWAP;
    return o;
  }
  if (r.mode == RC_FAIL) {
    o.flags = PV_FAIL;
    return o;
  }
  double cphi, cpsi;
  if (r.mode == RC_EXC) {
    // signed form of the exception (reading of Sec. 2.1.2)
    const double s = sgn1(x), ax = fabs(x);
    const double p = rsqrt(2.0 * (1.0 + ax)), q = rsqrt(2.0 * (1.0 - ax));
    o.z11 = p; o.z12 = -s * q; o.z21 = s * p; o.z22 = q;
    cphi = o.z11; cpsi = o.z22;  // no t in this form
  } else {
    const double c = r.c, s = r.s;
    cphi = c + xi * (s - eta * c);
    cpsi = c - xi * (s + eta * c);
    const double sphi = s - xi * (c + eta * s);
    const double spsi = s + xi * (c - eta * s);
    o.z11 = cphi * r.rt;
    o.z12 = sphi * r.rt;
    o.z21 = -spsi * r.rt;
    o.z22 = cpsi * r.rt;
  }
  o.flags = PV_ROT;
  bool small;
  if (crit2 && r.mode == RC_ROT)
    small = f32cls ? (__double2float_rn(cphi) == 1.0f && __double2float_rn(cpsi) == 1.0f)
                   : (cphi == 1.0 && cpsi == 1.0);
  else
    small = f32cls ? (__double2float_rn(o.z11) == 1.0f && __double2float_rn(o.z22) == 1.0f)
                   : (o.z11 == 1.0 && o.z22 == 1.0);
  if (!small) o.flags |= PV_BIG;
  if (sort) {
    // transformed diagonal of A-hat (Sec. 3.5.3, real case)
    const double d1 = o.z11 * o.z11 * a11 + 2.0 * o.z11 * o.z21 * a12 + o.z21 * o.z21 * a22;
    const double d2 = o.z12 * o.z12 * a11 + 2.0 * o.z22 * o.z12 * a12 + o.z22 * o.z22 * a22;
    if (d1 < d2) o.flags |= PV_SWAP;
  }
  return o;
}

// Real pivot on one thread (both chains in sequence); the same arithmetic as
// the two-warp form, so both give identical bits.
__device__ __forceinline__ PivotOut pivot_real(double a11, double a22, double a12, double x, double tol,
                                               bool sort, bool f32cls, bool crit2) {
  const RealChainA r = real_chain_a(a11, a22, a12, x, tol);
  double xi = 0.0, eta = 0.0;
  if (r.mode == RC_ROT) real_chain_b(x, xi, eta);
  return real_combine(a11, a22, a12, x, r, xi, eta, sort, f32cls, crit2);
}

// Named barrier for the two parameter warps (barrier 1, 64 threads).
__device__ __forceinline__ void param_pair_barrier() { asm volatile("bar.sync 1, 64;\n" ::: "memory"); }

// Complex pivot, Sec. 2.1.1.  a12 = (ar, ai), b12 = (br, bi).
__device__ __forceinline__ PivotOut pivot_cplx(double a11, double a22, double ar, double ai,
                                               double br, double bi, double tol, bool sort,
                                               bool f32cls, bool crit2) {
  PivotOut o;
  o.flags = 0;
  // relative orthogonality in squares: |a12|^2 < a11 a22 tol^2, |b12|^2 < tol^2
  const double tol2 = tol * tol;
  const double absa2 = fma(ar, ar, ai * ai);
  const double x2 = fma(br, br, bi * bi);
  if (absa2 < (a11 * a22) * tol2 && x2 < tol2) {
    o.z11 = 1.0; o.z12 = 0.0; o.z21 = 0.0; o.z22 = 1.0; o.z12i = 0.0; o.z21i = 0.0;
    if (sort && a11 < a22) o.flags |= PV_SWAP;
    return o;
  }
  const double x = hypot(br, bi);
  const double t2 = fma(-x, x, 1.0);
  if (!(t2 > 0.0)) {
    o.z11 = 1.0; o.z12 = 0.0; o.z21 = 0.0; o.z22 = 1.0; o.z12i = 0.0; o.z21i = 0.0;
    o.flags = PV_FAIL;
    return o;
  }
  const double rt = rsqrt(t2);
  const double t = t2 * rt;
  // e^{i zeta} = b12 / |b12| (1 if b12 = 0); z = e^{-i zeta} a12
  double er = 1.0, ei = 0.0;
  if (x != 0.0) {
    const double rx = 1.0 / x;
    er = br * rx;
    ei = bi * rx;
  }
  const double u = er * ar + ei * ai;
  const double v = er * ai - ei * ar;
  const double h = a22 - a11;
  double cphi, cpsi;
  if (v == 0.0 && h == 0.0) {
    const double p = rsqrt(2.0 * (1.0 + x)), q = rsqrt(2.0 * (1.0 - x));
    o.z11 = p; o.z22 = q;
    o.z12 = -er * q; o.z12i = -ei * q;   // -e^{i zeta} q
    o.z21 = er * p;  o.z21i = -ei * p;   //  e^{-i zeta} p
    cphi = o.z11; cpsi = o.z22;
    o.flags = PV_ROT;
    const bool small = f32cls ? (__double2float_rn(o.z11) == 1.0f && __double2float_rn(o.z22) == 1.0f)
                              : (o.z11 == 1.0 && o.z22 == 1.0);
    if (!small) o.flags |= PV_BIG;
  } else {
    const double tau = sgn1(h);
    const double tan2 = tau * (2.0 * u - (a11 + a22) * x) / (t * sqrt(fma(h, h, 4.0 * v * v)));
    const double tang = 2.0 * v / h;
    double c2, s2, cg, sg;
    trig_from_tan(tan2, c2, s2);
    trig_from_tan(tang, cg, sg);
    const double tcc = t * cg * c2;
    cphi = sqrt(0.5 * (1.0 + x * s2 + tcc));
    cpsi = sqrt(0.5 * (1.0 - x * s2 + tcc));
    const double w = t * sg * c2;
    // 1/(2 cos psi) and 1/(2 cos phi) from one reciprocal
    const double r4 = 1.0 / (4.0 * cphi * cpsi);
    const double ipsi = 2.0 * cphi * r4, iphi = 2.0 * cpsi * r4;
    // e^{i alpha} sin(phi) = e^{i zeta} ((s2 - x) + i w) / (2 cos psi)
    const double pa = (s2 - x) * ipsi, qa = w * ipsi;
    // e^{-i beta} sin(psi) = e^{-i zeta} ((s2 + x) - i w) / (2 cos phi)
    const double pb = (s2 + x) * iphi, qb = -w * iphi;
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
      small = f32cls ? (__double2float_rn(cphi) == 1.0f && __double2float_rn(cpsi) == 1.0f)
                     : (cphi == 1.0 && cpsi == 1.0);
    else
      small = f32cls ? (__double2float_rn(o.z11) == 1.0f && __double2float_rn(o.z22) == 1.0f)
                     : (o.z11 == 1.0 && o.z22 == 1.0);
    if (!small) o.flags |= PV_BIG;
  }
  if (sort) {
    // transformed diagonal of A-hat: (Z^* A Z)_11 and _22, Z11 and Z22 real
    const double re21a = o.z21 * ar - o.z21i * ai;          // Re(a12 * z21)
    const double d1 = o.z11 * o.z11 * a11 + 2.0 * o.z11 * re21a + (o.z21 * o.z21 + o.z21i * o.z21i) * a22;
    const double re12a = o.z12 * ar + o.z12i * ai;          // Re(conj(z12) * a12)
    const double d2 = (o.z12 * o.z12 + o.z12i * o.z12i) * a11 + 2.0 * o.z22 * re12a + o.z22 * o.z22 * a22;
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
