// k_pointwise.cu -- pointwise one-sided implicit Hari-Zimmermann GSVD of
// small pairs, one CTA per problem, with F, G and Z resident in shared memory
// (Sec. 2.1-2.5 of arXiv 1909.00101, the non-blocked method).
//
// One launch solves a whole batch of independent problems (one CTA each).
// Per parallel step (a row of a pivot table of disjoint pairs, Sec. 2.2):
//   1. one warp per pair forms a_ii, a_jj, a_ij, b_ij (lane-strided partial
//      sums, fixed-order warp reduction);
//   2. the FP64 2x2 parameters of all pairs of the step are computed one pair
//      per lane (FP64 issue cost on sm_103a is per warp instruction, so a
//      warp computing one pair redundantly on 32 lanes wastes 31/32 of it);
//   3. one warp per pair applies Z-hat to the two columns of F, G and Z and
//      swaps them when sorting asks for it.
// A sweep is a full cycle of the table; the solve stops after a sweep with no
// transformation (the pointwise rule of Sec. 2.5) or at the sweep cap.
//
// VAR selects the variants of Sec. 2.6 (C2 is a run-time flag): bit 1 the
// enhanced dot products of App. A (real dots and all norms; complex
// off-diagonal products stay ordinary, App. A defines none for them), bit 2
// the D-hat rescaling (no prescaling; per pivot pair A' = D A D, B' = D B D
// with D_kk = 1/sqrt(b_kk) where b_kk != 1, and Z-hat = D Z-hat'; the sort
// compares the diagonal of Z-hat'^* A' Z-hat').
#include "hz_device.cuh"
#include "hz_kernels.h"

namespace hz {

namespace {

template <class T, bool CPLX>
struct PW {
  static constexpr int E = CPLX ? 2 : 1;  // scalars per element
};

// shared-memory parameter slots of one step
struct PivIn {
  double a11, a22, ar, ai, br, bi;
};

// Pair k of parallel step st for a problem of n columns, from the problem's
// own n (so a problem's sequence of transformations does not depend on the
// other members of a batch).  Row-cyclic wavefront: step st holds the pairs
// (i, j), i < j, i + j = st + 1 -- a parallel table of the sequential
// row-cyclic order (disjoint pairs commute).  Round robin: the circle method.
__device__ __forceinline__ bool pw_pair(bool rowcyc, int n, int st, int k, int& i, int& j) {
  if (rowcyc) {
    const int sum = st + 1;
    i = max(0, sum - (n - 1)) + k;
    j = sum - i;
    return i < j && j < n;
  }
  const int M = n + (n & 1);
  rr_pair(M, st, k, i, j);
  return j < n;
}

// ||y||^2 of column y (m elements, E scalars each) in shared memory, summed
// by one warp: ordinary (fma) or enhanced; the result on every lane
template <class T, bool CPLX, bool ENH>
__device__ __forceinline__ double col_norm2(const T* y, int m, int lane) {
  if constexpr (!ENH) {
    double s = 0.0;
    for (int r = lane; r < (CPLX ? 2 : 1) * m; r += 32) {
      const double v = y[r];
      s = fma(v, v, s);
    }
    return warp_sum(s);
  } else if constexpr (!CPLX) {
    double c = 0.0, d = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double v = y[r];
      enh_acc(c, d, v, v);
    }
    return warp_sum(c) + warp_sum(d);
  } else {
    double s = 0.0;
    for (int r = lane; r < m; r += 32) s += enh_abs2(y[2 * r], y[2 * r + 1]);
    return warp_sum(s);
  }
}

template <class T, bool CPLX, int VAR>
__global__ void __launch_bounds__(512) k_pointwise(const PwProblem* __restrict__ probs, int table_slots,
                                                   PwParams prm) {
  constexpr int E = PW<T, CPLX>::E;
  constexpr bool ENH = (VAR & 1) != 0, DSC = (VAR & 2) != 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PwProblem P = probs[blockIdx.x];
  const int n = P.n, mf = P.mf, mg = P.mg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  // layout: F (mf x n), G (mg x n), Z (n x n), column-major, E scalars each
  T* sF = reinterpret_cast<T*>(smem_raw);
  T* sG = sF + (size_t)E * mf * n;
  T* sZ = sG + (size_t)E * mg * n;
  PivIn* pin = reinterpret_cast<PivIn*>(sZ + (size_t)E * n * n);
  PivotOut* pout = reinterpret_cast<PivotOut*>(pin + table_slots);
  double* colnorm = reinterpret_cast<double*>(pout + table_slots);  // 2n: nf, ng
  int* ctr = reinterpret_cast<int*>(colnorm + 2 * n);               // nall, nbig, fail, overflow
  int* rank = ctr + 4;
  __shared__ double s_xi[32], s_eta[32];  // chain B of the real parameters
  __shared__ double s_d[2][32];            // D-hat of each pair of a step (DSC)

  // load (convert to T), zero Z
  const double* gF = static_cast<const double*>(P.F);
  const double* gG = static_cast<const double*>(P.G);
  for (int idx = threadIdx.x; idx < E * mf * n; idx += blockDim.x) {
    const int j = idx / (E * mf), r = idx % (E * mf);
    sF[idx] = static_cast<T>(gF[(size_t)j * E * P.ldf + r]);
  }
  for (int idx = threadIdx.x; idx < E * mg * n; idx += blockDim.x) {
    const int j = idx / (E * mg), r = idx % (E * mg);
    sG[idx] = static_cast<T>(gG[(size_t)j * E * P.ldg + r]);
  }
  for (int idx = threadIdx.x; idx < E * n * n; idx += blockDim.x) sZ[idx] = T(0);
  if (threadIdx.x < 4) ctr[threadIdx.x] = 0;
  __syncthreads();

  // prescale: z_j = 1/||g_j||, F0 = F Z0, G0 = G Z0, Z = Z0 (the D-hat
  // variants start from Z0 = I and only check g_j != 0)
  for (int j = warp; j < n; j += nwarps) {
    double s = col_norm2<T, CPLX, ENH>(sG + (size_t)j * E * mg, mg, lane);
    if (!(s > 0.0)) {
      if (lane == 0) atomicOr(&ctr[2], 1);
      s = 1.0;
    }
    if constexpr (DSC) {
      if (lane == 0) sZ[(size_t)j * E * n + E * j] = T(1);
      continue;
    }
    const double zj = 1.0 / sqrt(s);
    for (int r = lane; r < E * mf; r += 32) sF[(size_t)j * E * mf + r] = static_cast<T>(sF[(size_t)j * E * mf + r] * zj);
    for (int r = lane; r < E * mg; r += 32) sG[(size_t)j * E * mg + r] = static_cast<T>(sG[(size_t)j * E * mg + r] * zj);
    if (lane == 0) sZ[(size_t)j * E * n + E * j] = static_cast<T>(zj);
  }
  __syncthreads();
  if (ctr[2]) {
    if (threadIdx.x == 0) {
      P.stats->status = ST_ENOTPD;
    }
    return;
  }

  const double tol = prm.eps * sqrt((double)n);
  const int M = n + (n & 1);
  const int nsteps = prm.rowcyc ? max(1, 2 * n - 3) : max(1, M - 1);
  const int nslots = prm.rowcyc ? max(1, n / 2) : max(1, M / 2);
  int sweeps = 0;
  long long tall = 0, tbig = 0;
  bool converged = (n == 1);
  int status = ST_OK;
  while (!converged && sweeps < prm.max_sweeps) {
    ++sweeps;
    int sweep_all = 0;
    for (int st = 0; st < nsteps; ++st) {
      // 1. dots, one warp per pair
      for (int k = warp; k < nslots; k += nwarps) {
        int i, j;
        if (!pw_pair(prm.rowcyc, n, st, k, i, j)) continue;
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        double w[2] = {0.0, 0.0};
        double bii = 1.0, bjj = 1.0;  // DSC: ||g_i||^2, ||g_j||^2
        if constexpr (!CPLX && ENH) {
          double dd[4] = {0.0, 0.0, 0.0, 0.0};
          for (int r = lane; r < mf; r += 32) {
            const double fi = sF[(size_t)i * mf + r], fj = sF[(size_t)j * mf + r];
            enh_acc(v[0], dd[0], fi, fi);
            enh_acc(v[1], dd[1], fj, fj);
            enh_acc(v[2], dd[2], fi, fj);
          }
          for (int r = lane; r < mg; r += 32) enh_acc(v[3], dd[3], (double)sG[(size_t)i * mg + r], (double)sG[(size_t)j * mg + r]);
          warp_sum4(v);
          warp_sum4(dd);
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] += dd[q];
        } else if constexpr (!CPLX) {
          for (int r = lane; r < mf; r += 32) {
            const double fi = sF[(size_t)i * mf + r], fj = sF[(size_t)j * mf + r];
            v[0] = fma(fi, fi, v[0]);
            v[1] = fma(fj, fj, v[1]);
            v[2] = fma(fi, fj, v[2]);
          }
          for (int r = lane; r < mg; r += 32) v[3] = fma((double)sG[(size_t)i * mg + r], (double)sG[(size_t)j * mg + r], v[3]);
          warp_sum4(v);
        } else if constexpr (ENH) {
          // the norms enhanced; Re, Im of conj(f_i) f_j and b_ij ordinary
          for (int r = lane; r < mf; r += 32) {
            const double fir = sF[(size_t)i * 2 * mf + 2 * r], fii = sF[(size_t)i * 2 * mf + 2 * r + 1];
            const double fjr = sF[(size_t)j * 2 * mf + 2 * r], fji = sF[(size_t)j * 2 * mf + 2 * r + 1];
            v[0] += enh_abs2(fir, fii);
            v[1] += enh_abs2(fjr, fji);
            v[2] = fma(fir, fjr, fma(fii, fji, v[2]));
            v[3] = fma(fir, fji, fma(-fii, fjr, v[3]));
          }
          for (int r = lane; r < mg; r += 32) {
            const double gir = sG[(size_t)i * 2 * mg + 2 * r], gii = sG[(size_t)i * 2 * mg + 2 * r + 1];
            const double gjr = sG[(size_t)j * 2 * mg + 2 * r], gji = sG[(size_t)j * 2 * mg + 2 * r + 1];
            w[0] = fma(gir, gjr, fma(gii, gji, w[0]));
            w[1] = fma(gir, gji, fma(-gii, gjr, w[1]));
          }
          warp_sum4(v);
          w[0] = warp_sum(w[0]);
          w[1] = warp_sum(w[1]);
        } else {
          for (int r = lane; r < mf; r += 32) {
            const double fir = sF[(size_t)i * 2 * mf + 2 * r], fii = sF[(size_t)i * 2 * mf + 2 * r + 1];
            const double fjr = sF[(size_t)j * 2 * mf + 2 * r], fji = sF[(size_t)j * 2 * mf + 2 * r + 1];
            v[0] = fma(fir, fir, fma(fii, fii, v[0]));
            v[1] = fma(fjr, fjr, fma(fji, fji, v[1]));
            v[2] = fma(fir, fjr, fma(fii, fji, v[2]));    // Re(conj(fi) fj)
            v[3] = fma(fir, fji, fma(-fii, fjr, v[3]));   // Im(conj(fi) fj)
          }
          for (int r = lane; r < mg; r += 32) {
            const double gir = sG[(size_t)i * 2 * mg + 2 * r], gii = sG[(size_t)i * 2 * mg + 2 * r + 1];
            const double gjr = sG[(size_t)j * 2 * mg + 2 * r], gji = sG[(size_t)j * 2 * mg + 2 * r + 1];
            w[0] = fma(gir, gjr, fma(gii, gji, w[0]));
            w[1] = fma(gir, gji, fma(-gii, gjr, w[1]));
          }
          warp_sum4(v);
          w[0] = warp_sum(w[0]);
          w[1] = warp_sum(w[1]);
        }
        if constexpr (DSC) {
          bii = col_norm2<T, CPLX, ENH>(sG + (size_t)i * E * mg, mg, lane);
          bjj = col_norm2<T, CPLX, ENH>(sG + (size_t)j * E * mg, mg, lane);
        }
        if (lane == 0) {
          PivIn p;
          p.a11 = v[0]; p.a22 = v[1]; p.ar = v[2];
          if constexpr (CPLX) { p.ai = v[3]; p.br = w[0]; p.bi = w[1]; }
          else { p.ai = 0.0; p.br = v[3]; p.bi = 0.0; }
          if constexpr (DSC) {
            // A' = D A D, B' = D B D: the diagonal of A' by a division by
            // b_kk, the off-diagonals times D_kk, where b_kk != 1
            double d1 = 1.0, d2 = 1.0;
            if (!(bii > 0.0) || !(bjj > 0.0)) atomicOr(&ctr[2], 1);
            if (bii != 1.0) {
              p.a11 = p.a11 / bii;
              d1 = 1.0 / sqrt(bii);
              p.ar *= d1; p.ai *= d1; p.br *= d1; p.bi *= d1;
            }
            if (bjj != 1.0) {
              p.a22 = p.a22 / bjj;
              d2 = 1.0 / sqrt(bjj);
              p.ar *= d2; p.ai *= d2; p.br *= d2; p.bi *= d2;
            }
            s_d[0][k] = d1;
            s_d[1][k] = d2;
          }
          pin[k] = p;
        }
      }
      __syncthreads();
      // 2. parameters, one pair per lane (nslots <= 32 for n <= 64); real
      //    pivots run their two independent FP64 chains on warps 0 and 1,
      //    complex pivots on warp 0; counters warp-aggregated
      if (warp <= 1) {
        const int k = lane;
        int i = 0, j = 0;
        const bool act = k < nslots && pw_pair(prm.rowcyc, n, st, k, i, j);
        int fl = 0;
        PivotOut o;
        bool have = false;
        if constexpr (!CPLX) {
          if (warp == 1) {
            double xi = 0.0, eta = 0.0;
            if (act) real_chain_b(pin[k].br, xi, eta);
            s_xi[lane] = xi;
            s_eta[lane] = eta;
            param_pair_barrier();
          } else {
            RealChainA r;
            PivIn p{};
            if (act) {
              p = pin[k];
              r = real_chain_a(p.a11, p.a22, p.ar, p.br, tol);
            }
            param_pair_barrier();
            if (act) {
              o = real_combine(p.a11, p.a22, p.ar, p.br, r, s_xi[lane], s_eta[lane], prm.sort, prm.f32cls, prm.crit2);
              have = true;
            }
          }
        } else {
          if (warp == 0 && act) {
            const PivIn p = pin[k];
            o = pivot_cplx(p.a11, p.a22, p.ar, p.ai, p.br, p.bi, tol, prm.sort, prm.f32cls, prm.crit2);
            have = true;
          }
        }
        if (warp == 0) {
          if (have) {
            if constexpr (DSC) {
              if (o.flags & PV_ROT) {  // Z-hat = D Z-hat': rows times D11, D22
                const double d1 = s_d[0][k], d2 = s_d[1][k];
                o.z11 *= d1; o.z12 *= d1; o.z12i *= d1;
                o.z21 *= d2; o.z21i *= d2; o.z22 *= d2;
              }
            }
            pout[k] = o;
            fl = o.flags;
          }
          const unsigned rot = __ballot_sync(FULL, fl & PV_ROT), big = __ballot_sync(FULL, fl & PV_BIG);
          const unsigned bad = __ballot_sync(FULL, fl & PV_FAIL);
          if (lane == 0) {
            if (rot) ctr[0] += __popc(rot);
            if (big) ctr[1] += __popc(big);
            if (bad) ctr[2] = 1;
          }
        }
      }
      __syncthreads();
      // 3. apply and swap, one warp per pair
      for (int k = warp; k < nslots; k += nwarps) {
        int i, j;
        if (!pw_pair(prm.rowcyc, n, st, k, i, j)) continue;
        const PivotOut o = pout[k];
        const bool rot = o.flags & PV_ROT, sw = o.flags & PV_SWAP;
        if (!rot && !sw) continue;
        auto upd = [&](T* Y, int m) {
          if constexpr (!CPLX) {
            for (int r = lane; r < m; r += 32) {
              const double yi = Y[(size_t)i * m + r], yj = Y[(size_t)j * m + r];
              double ni = yi, nj = yj;
              if (rot) {
                ni = fma(yj, o.z21, yi * o.z11);
                nj = fma(yi, o.z12, yj * o.z22);
              }
              Y[(size_t)i * m + r] = static_cast<T>(sw ? nj : ni);
              Y[(size_t)j * m + r] = static_cast<T>(sw ? ni : nj);
            }
          } else {
            for (int r = lane; r < m; r += 32) {
              const double yir = Y[(size_t)i * 2 * m + 2 * r], yii = Y[(size_t)i * 2 * m + 2 * r + 1];
              const double yjr = Y[(size_t)j * 2 * m + 2 * r], yji = Y[(size_t)j * 2 * m + 2 * r + 1];
              double nir = yir, nii = yii, njr = yjr, nji = yji;
              if (rot) {
                // y_i' = y_i z11 + y_j z21 ; y_j' = y_i z12 + y_j z22 (z11, z22 real)
                nir = fma(yjr, o.z21, fma(-yji, o.z21i, yir * o.z11));
                nii = fma(yjr, o.z21i, fma(yji, o.z21, yii * o.z11));
                njr = fma(yir, o.z12, fma(-yii, o.z12i, yjr * o.z22));
                nji = fma(yir, o.z12i, fma(yii, o.z12, yji * o.z22));
              }
              Y[(size_t)i * 2 * m + 2 * r] = static_cast<T>(sw ? njr : nir);
              Y[(size_t)i * 2 * m + 2 * r + 1] = static_cast<T>(sw ? nji : nii);
              Y[(size_t)j * 2 * m + 2 * r] = static_cast<T>(sw ? nir : njr);
              Y[(size_t)j * 2 * m + 2 * r + 1] = static_cast<T>(sw ? nii : nji);
            }
          }
        };
        upd(sF, mf);
        upd(sG, mg);
        upd(sZ, n);
      }
      __syncthreads();
      if (ctr[2]) break;
    }
    __syncthreads();
    const int nall = ctr[0], nbig = ctr[1], fail = ctr[2];
    __syncthreads();
    if (threadIdx.x == 0) { ctr[0] = 0; ctr[1] = 0; }
    tall += nall;
    tbig += nbig;
    sweep_all = nall;
    if (fail) { status = ST_ENOTPD; break; }
    if (sweep_all == 0) converged = true;
    __syncthreads();
  }
  if (status == ST_OK && !converged) status = ST_ENOCONV;

  // final rescaling (Sec. 2.4): column norms of F and G
  for (int j = warp; j < n; j += nwarps) {
    const double sf = col_norm2<T, CPLX, ENH>(sF + (size_t)j * E * mf, mf, lane);
    const double sg = col_norm2<T, CPLX, ENH>(sG + (size_t)j * E * mg, mg, lane);
    if (lane == 0) {
      colnorm[j] = sqrt(sf);
      colnorm[n + j] = sqrt(sg);
      if (!isfinite(sf) || !isfinite(sg) || !(sg > 0.0)) atomicOr(&ctr[3], 1);  // overflow
    }
  }
  __syncthreads();
  // stable rank by descending sigma = ||f_j|| / ||g_j|| (ties: lower index first)
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double sj = colnorm[j] / colnorm[n + j];
    int rk = 0;
    for (int k = 0; k < n; ++k) {
      const double sk = colnorm[k] / colnorm[n + k];
      rk += (sk > sj) || (sk == sj && k < j);
    }
    rank[j] = rk;
  }
  __syncthreads();
  double* oF = static_cast<double*>(P.F);
  double* oG = static_cast<double*>(P.G);
  double* oZ = static_cast<double*>(P.Z);
  for (int idx = threadIdx.x; idx < E * mf * n; idx += blockDim.x) {
    const int j = idx / (E * mf), r = idx % (E * mf);
    oF[(size_t)rank[j] * E * P.ldf + r] = (double)sF[idx] / colnorm[j];
  }
  for (int idx = threadIdx.x; idx < E * mg * n; idx += blockDim.x) {
    const int j = idx / (E * mg), r = idx % (E * mg);
    oG[(size_t)rank[j] * E * P.ldg + r] = (double)sG[idx] / colnorm[n + j];
  }
  for (int idx = threadIdx.x; idx < E * n * n; idx += blockDim.x) {
    const int j = idx / (E * n), r = idx % (E * n);
    const double th = 1.0 / sqrt(fma(colnorm[j], colnorm[j], colnorm[n + j] * colnorm[n + j]));
    oZ[(size_t)rank[j] * E * P.ldz + r] = (double)sZ[idx] * th;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double nf = colnorm[j], ng = colnorm[n + j];
    const double th = 1.0 / sqrt(fma(nf, nf, ng * ng));
    P.sigma_f[rank[j]] = nf * th;
    P.sigma_g[rank[j]] = ng * th;
    P.sigma[rank[j]] = nf / ng;
  }
  if (threadIdx.x == 0) {
    P.stats->status = (status == ST_OK && ctr[3]) ? ST_EOVERFLOW : status;
    P.stats->sweeps = sweeps;
    P.stats->transf_all = tall;
    P.stats->transf_big = tbig;
  }
}

}  // namespace

size_t pointwise_smem_bytes(int mf, int mg, int n, bool cplx, bool fp32, int slots) {
  const size_t e = (cplx ? 2 : 1) * (fp32 ? 4 : 8);
  size_t b = e * ((size_t)mf * n + (size_t)mg * n + (size_t)n * n);
  b = (b + 15) & ~size_t(15);
  b += sizeof(PivIn) * slots + sizeof(PivotOut) * slots + sizeof(double) * 2 * n + sizeof(int) * (4 + n);
  return b;
}

using Kern = void (*)(const PwProblem*, int, PwParams);
template <int VAR>
Kern pick(bool cplx, bool fp32) {
  if (cplx) return fp32 ? k_pointwise<float, true, VAR> : k_pointwise<double, true, VAR>;
  return fp32 ? k_pointwise<float, false, VAR> : k_pointwise<double, false, VAR>;
}

cudaError_t launch_pointwise(const PwProblem* d_probs, int count, int slots, bool cplx, bool fp32, size_t smem,
                             const PwParams& prm, cudaStream_t stream) {
  const int threads = slots >= 16 ? 512 : (slots >= 8 ? 256 : 128);
  const int var = (prm.enhanced ? 1 : 0) | (prm.dscale ? 2 : 0);
  const Kern kern = var == 0 ? pick<0>(cplx, fp32)
                             : var == 1 ? pick<1>(cplx, fp32) : var == 2 ? pick<2>(cplx, fp32) : pick<3>(cplx, fp32);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<count, threads, smem, stream>>>(d_probs, slots, prm);
  return cudaGetLastError();
}

}  // namespace hz
