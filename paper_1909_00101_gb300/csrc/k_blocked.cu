// k_blocked.cu -- one outer step of the blocked one-sided implicit
// Hari-Zimmermann GSVD (Sec. 2.3-2.5 of arXiv 1909.00101), re-designed for
// sm_103a as three kernels per step instead of the paper's one fused kernel:
//
//   Gram     grid (pair, row split): partial pivot Grams A-hat = [F_p F_q]^* [F_p F_q]
//            and B-hat = [G_p G_q]^* [G_p G_q] over a slab of rows.  FP32 sweeps:
//            k_gram32 (upper 8x8 blocks per thread, tiles staged by cp.async);
//            FP64 sweeps: the exact BF16-digit form in k_ozaki.cu, or k_gram
//            (DMMA m8n8k4).
//   pivot    grid (pair): fixed-order sum of the partials, Choleskys of A-hat
//            and B-hat, the pointwise implicit HZ on (F-hat, G-hat) in shared
//            memory, and the Theta-tilde rescaling that gives Z-tilde = Z-hat
//            Theta-tilde.  FP64 sweeps: k_inner2, a two-CTA cluster per pair,
//            FP64 2x2 parameters one pair per lane; FP32 sweeps: k_inner with
//            FP32 Choleskys and one pair per half-warp.
//   apply    grid (pair, row tile): [Y_p Y_q] <- [Y_p Y_q] Z-tilde in place for
//            Y = F, G, Z.  FP32 sweeps: k_apply32 (4 x 8 outputs per thread);
//            FP64 sweeps: k_ozaki.cu, or k_apply (DMMA).
//
// Splitting the row dimension of the Gram and the apply over many CTAs fills
// the 152 SMs even when a step has few block pairs (the paper's one CTA per
// pair leaves most SMs idle for n = 2048).  Complex data is handled by real
// views: with W = [Re Y, Im Y], Re(Y^*Y) and Im(Y^*Y) are sums and differences
// of blocks of W^T W, and Y Z = [Re Y, Im Y] [[Re Z, Im Z], [-Im Z, Re Z]].
#include <cstdlib>
#include <type_traits>

#include <cooperative_groups.h>

#include "blk_pair.cuh"
#include "hz_device.cuh"
#include "hz_kernels.h"

namespace hz {

namespace {

constexpr int TR = 64;  // rows per tile of the Gram and the apply

__device__ __forceinline__ void dmma884(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// Load rows [r0, r0+TR) of the real view of [Y_p Y_q] (zero outside) into
// shared memory: column-major (Ws[c * ld + r]) or row-major (Ws[r * ld + c]).
template <class T, bool CPLX, bool COLMAJ>
__device__ __forceinline__ void load_tile(T* Ws, int ld, const T* Y, long long ldy, int m, int r0,
                                          const PairCols& pc, int V) {
  if constexpr (!CPLX) {
    for (int idx = threadIdx.x; idx < V * TR; idx += blockDim.x) {
      const int c = idx / TR, r = idx % TR;
      T v = T(0);
      if (c < pc.bb && r0 + r < m) v = Y[(size_t)pc.gcol(c) * ldy + r0 + r];
      if (COLMAJ) Ws[c * ld + r] = v; else Ws[r * ld + c] = v;
    }
  } else {
    using T2 = typename std::conditional<std::is_same<T, double>::value, double2, float2>::type;
    const T2* Y2 = reinterpret_cast<const T2*>(Y);
    for (int idx = threadIdx.x; idx < (V / 2) * TR; idx += blockDim.x) {
      const int c = idx / TR, r = idx % TR;
      T re = T(0), im = T(0);
      if (c < pc.bb && r0 + r < m) {
        const T2 v = Y2[(size_t)pc.gcol(c) * ldy + r0 + r];
        re = v.x;
        im = v.y;
      }
      // real view: column c is Re, column bb + c is Im; for c >= bb the two
      // zero padding columns 2c and 2c + 1 (together they cover [2 bb, V))
      const int cr = (c < pc.bb) ? c : 2 * c;
      const int ci = (c < pc.bb) ? pc.bb + c : 2 * c + 1;
      if (COLMAJ) {
        Ws[cr * ld + r] = re;
        Ws[ci * ld + r] = im;
      } else {
        Ws[r * ld + cr] = re;
        Ws[r * ld + ci] = im;
      }
    }
  }
}

// ---------------------------------------------------------------- Gram ----
// FP64: one warp per upper-triangle 8x8 tile of the V x V Gram (DMMA m8n8k4),
// so the tiles (3, 10 or 36 for V = 16, 32, 64) are balanced over the warps.
template <class T, int V>
__host__ __device__ constexpr int gram_threads() {
  return std::is_same<T, double>::value ? 32 * ((V / 8) * (V / 8 + 1) / 2 > 16 ? ((V / 8) * (V / 8 + 1) / 2 + 2) / 3
                                                                                : (V / 8) * (V / 8 + 1) / 2)
                                        : 256;
}

template <class T, bool CPLX, int V>
__global__ void __launch_bounds__(gram_threads<T, V>()) k_gram(BlkDims d, BlkBuffers b, int step, BlkBatch bt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);
  int slot;
  if (!batch_item(bt, blockIdx.x, step, d, b, slot)) return;
  const int s = blockIdx.y;
  if (s >= d.rf + d.rg) return;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  const bool isF = s < d.rf;
  const int m = isF ? d.mf : d.mg;
  const int nsplit = isF ? d.rf : d.rg;
  const int si = isF ? s : s - d.rf;
  const int tiles = (m + TR - 1) / TR;
  const int per = (tiles + nsplit - 1) / nsplit * TR;  // whole tiles per split
  const int r0 = si * per, r1 = min(m, r0 + per);
  const T* Y = static_cast<const T*>(isF ? b.F : b.G);
  const long long ld = isF ? b.ldf : b.ldg;
  T* out = static_cast<T*>(b.partial) + ((size_t)slot * (d.rf + d.rg) + s) * V * V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if constexpr (std::is_same<T, double>::value) {
    constexpr int LDT = TR + 4;
    constexpr int NB = V / 8;
    constexpr int NT = NB * (NB + 1) / 2;  // upper-triangle 8x8 tiles
    constexpr int NW = gram_threads<T, V>() / 32;
    constexpr int PER = (NT + NW - 1) / NW;  // tiles per warp
    double acc[PER][2];
    int ti[PER], tj[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      acc[u][0] = acc[u][1] = 0.0;
      int t = warp + NW * u, a = 0;
      ti[u] = -1;
      tj[u] = 0;
      if (t < NT) {
        while (t >= NB - a) { t -= NB - a; ++a; }
        ti[u] = a;
        tj[u] = a + t;
      }
    }
    for (int rt = r0; rt < r1; rt += TR) {
      load_tile<T, CPLX, true>(Ws, LDT, Y, ld, r1, rt, pc, V);
      __syncthreads();
#pragma unroll 4
      for (int k0 = 0; k0 < TR; k0 += 4) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          if (ti[u] < 0) continue;
          const double a = Ws[(ti[u] * 8 + (lane >> 2)) * LDT + k0 + (lane & 3)];
          const double bv = Ws[(tj[u] * 8 + (lane >> 2)) * LDT + k0 + (lane & 3)];
          dmma884(acc[u][0], acc[u][1], a, bv);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (ti[u] < 0) continue;
      const int i = ti[u] * 8 + (lane >> 2), j = tj[u] * 8 + 2 * (lane & 3);
      out[i * V + j] = acc[u][0];
      out[i * V + j + 1] = acc[u][1];
    }
  } else {
    constexpr int LDT = V + 4;            // row stride of the staged tile (16-byte aligned rows)
    constexpr int TPG = (V / 4) * (V / 4);  // threads of a row group: one 4 x 4 block of the Gram each
    constexpr int NG = 256 / TPG;           // row groups: each sums its rows of the tile, then all add up
    const int g = threadIdx.x / TPG, tq = threadIdx.x % TPG;
    const int bi = 4 * (tq % (V / 4)), bj = 4 * (tq / (V / 4));
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    // the next row tile is prefetched into registers while this one is used
    constexpr int E = CPLX ? 2 : 1;
    constexpr int PERT = (V / E) * TR / 256;
    float pre[PERT][E];
    auto fetch = [&](int rt) {
#pragma unroll
      for (int i = 0; i < PERT; ++i) {
        const int idx = threadIdx.x + 256 * i, c = idx / TR, r = idx % TR;
        pre[i][0] = 0.0f;
        if constexpr (CPLX) pre[i][1] = 0.0f;
        if (c < pc.bb && rt + r < r1) {
          if constexpr (CPLX) {
            const float2 v = reinterpret_cast<const float2*>(Y)[(size_t)pc.gcol(c) * ld + rt + r];
            pre[i][0] = v.x;
            pre[i][1] = v.y;
          } else {
            pre[i][0] = Y[(size_t)pc.gcol(c) * ld + rt + r];
          }
        }
      }
    };
    if (r0 < r1) fetch(r0);
    for (int rt = r0; rt < r1; rt += TR) {
#pragma unroll
      for (int i = 0; i < PERT; ++i) {
        const int idx = threadIdx.x + 256 * i, c = idx / TR, r = idx % TR;
        if constexpr (CPLX) {
          const int cr = (c < pc.bb) ? c : 2 * c, ci = (c < pc.bb) ? pc.bb + c : 2 * c + 1;
          Ws[r * LDT + cr] = pre[i][0];
          Ws[r * LDT + ci] = pre[i][1];
        } else {
          Ws[r * LDT + c] = pre[i][0];
        }
      }
      if (rt + TR < r1) fetch(rt + TR);
      __syncthreads();
      // group g takes rows g, g + NG, ... of the tile; 8 loads, 16 FMAs a row
#pragma unroll 4
      for (int r = g; r < TR; r += NG) {
        const float4 a = *reinterpret_cast<const float4*>(&Ws[r * LDT + bi]);
        const float4 bv = *reinterpret_cast<const float4*>(&Ws[r * LDT + bj]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bw[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bw[v], acc[u][v]);
      }
      __syncthreads();
    }
    // the groups' partial Grams added in group order (a fixed order): group
    // g's block goes through shared memory, group 0 sums and writes
    float* part = Ws;  // reuse: the buffer holds (NG - 1) V x V floats (gram_smem)
    if (g > 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) part[((g - 1) * V + bi + u) * V + bj + v] = acc[u][v];
    }
    __syncthreads();
    if (g == 0) {
      for (int gg = 1; gg < NG; ++gg)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += part[((gg - 1) * V + bi + u) * V + bj + v];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float4 w4;
        w4.x = acc[u][0]; w4.y = acc[u][1]; w4.z = acc[u][2]; w4.w = acc[u][3];
        *reinterpret_cast<float4*>(&out[(bi + u) * V + bj]) = w4;
      }
    }
  }
}

// --------------------------------------------------------------- inner ----
// Per-pair inputs and outputs of one inner step, in the inner data type Ti:
// the FP64 parameter warp widens the inputs and narrows Z-hat once per pair,
// so the pair warps never issue FP64 conversions (on sm_103a every FP64
// instruction, conversions included, costs a full FP64 warp slot).
template <class Ti>
struct PivInT {
  Ti a11, a22, ar, ai, br, bi;
};
// Sums over the 16 lanes of a half-warp (both halves at once, each its own
// values), in a fixed order.  half_sum4_all leaves all four sums in every
// lane of the half: a transposing butterfly (offsets 8 and 4 halve the
// values, 2 and 1 finish), then one broadcast per sum.
__device__ __forceinline__ void half_sum4_all(float v[4]) {
  const int lane = threadIdx.x & 31;
  const bool b8 = lane & 8, b4 = lane & 4;
  const float s0 = b8 ? v[0] : v[2], s1 = b8 ? v[1] : v[3];
  float k0 = b8 ? v[2] : v[0], k1 = b8 ? v[3] : v[1];
  k0 += __shfl_xor_sync(FULL, s0, 8);
  k1 += __shfl_xor_sync(FULL, s1, 8);
  const float sx = b4 ? k0 : k1;
  float k = b4 ? k1 : k0;
  k += __shfl_xor_sync(FULL, sx, 4);
  k += __shfl_xor_sync(FULL, k, 2);
  k += __shfl_xor_sync(FULL, k, 1);
  // lanes 0-3 of the half hold sum 0, 4-7 sum 1, 8-11 sum 2, 12-15 sum 3
  const int base = lane & 16;
  v[0] = __shfl_sync(FULL, k, base);
  v[1] = __shfl_sync(FULL, k, base + 4);
  v[2] = __shfl_sync(FULL, k, base + 8);
  v[3] = __shfl_sync(FULL, k, base + 12);
}
__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

template <class Ti>
struct PivZ {
  Ti z11, z12, z21, z22, z12i, z21i;
  int flags;
};

// Packed upper triangle (i <= j) of an order-n matrix, column by column:
// u = j (j + 1) / 2 + i.  Unpacks u into (i, j).
__device__ __forceinline__ void unpack_upper(int u, int& i, int& j) {
  int jj = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while (jj * (jj + 1) / 2 > u) --jj;
  while ((jj + 1) * (jj + 2) / 2 <= u) ++jj;
  j = jj;
  i = u - jj * (jj + 1) / 2;
}

constexpr int INNER_THREADS = 512;  // threads of the pivot kernel

// Ti: data type of the inner sweeps (double, or float in FP32 bulk sweeps);
// To: type of the outer data (partials and Z-tilde).  P32 (FP32 bulk sweeps
// only): the whole pivot-pair step in FP32 -- partial sums, Choleskys and
// 2x2 parameters, the latter taken by each pair's own warp; its inputs are
// FP32 Gram partials, so FP32 arithmetic is as accurate as they are.
// Otherwise the sums and Choleskys are FP64 and one warp (two for real
// pivots) takes all pairs' FP64 parameters, one pair per lane.
template <class Ti, class To, bool CPLX, int V, bool P32>
__global__ void __launch_bounds__(INNER_THREADS) k_inner(BlkDims d, BlkBuffers b, int step, InnerParams prm,
                                                         BlkBatch bt) {
  constexpr int E = CPLX ? 2 : 1;
  constexpr int NTH = INNER_THREADS;
  constexpr int BMAX = CPLX ? V / 2 : V;  // max columns of the pair
  using Tc = typename std::conditional<P32, float, double>::type;  // sums and Choleskys
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Ad = reinterpret_cast<double*>(smem_raw);       // E * BMAX * BMAX
  double* Bd = Ad + E * BMAX * BMAX;                      // E * BMAX * BMAX
  Ti* Zh = reinterpret_cast<Ti*>(Bd + E * BMAX * BMAX);   // E * BMAX * BMAX
  PivInT<Ti>* pin = reinterpret_cast<PivInT<Ti>*>(Zh + E * BMAX * BMAX);
  PivZ<Ti>* pout = reinterpret_cast<PivZ<Ti>*>(pin + BMAX / 2 + 1);
  uint16_t* s_tri = reinterpret_cast<uint16_t*>(pout + BMAX / 2 + 1);  // BMAX (BMAX + 1) / 2
  Tc* A = reinterpret_cast<Tc*>(Ad);
  Tc* Bm = reinterpret_cast<Tc*>(Bd);
  __shared__ int s_ctr[4];  // all, big, fail, any-change
  __shared__ Tc s_inv[2];
  __shared__ int s_bad;
  __shared__ double s_xi[32], s_eta[32];  // chain B of the real parameters
  __shared__ unsigned char s_pair[63][32][2];  // inner round-robin table (M - 1 steps x M / 2 pairs)

  int slot;
  if (!batch_item(bt, blockIdx.x, step, d, b, slot, &prm)) return;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  const int bb = pc.bb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int S = d.rf + d.rg;
  const To* P = static_cast<const To*>(b.partial) + (size_t)slot * S * V * V;
  if (threadIdx.x < 4) s_ctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    s_bad = 0;
    atomicAdd(&b.ctr[4], 1ull);
  }

  // packed upper triangle (i <= j) of the pair's order, column by column:
  // entry u = j (j + 1) / 2 + i holds i | j << 8.  Its first r (r + 1) / 2
  // entries are the packed triangle of order r, for every r <= bb.
  const int nup = bb * (bb + 1) / 2;
  for (int u = threadIdx.x; u < nup; u += blockDim.x) {
    int i, j;
    unpack_upper(u, i, j);
    s_tri[u] = (uint16_t)(i | (j << 8));
  }
  __syncthreads();

  // 1. fixed-order sum of the partials into A-hat and B-hat (column-major,
  //    both triangles): the upper-triangle entries of both matrices as one
  //    packed list, so that every lane of a warp has an entry; the loads of
  //    eight partials are issued before their (sequential) sum.  Entries go
  //    row by row (i fixed, j rising along the lanes) so that a warp reads
  //    consecutive addresses of each partial: row-major entry u is the
  //    column-major entry nup - 1 - u of the flipped index pair.
  for (int t = threadIdx.x; t < 2 * nup; t += blockDim.x) {
    const int mat = t >= nup ? 1 : 0;
    const int ij = s_tri[nup - 1 - (t - mat * nup)];
    const int i = bb - 1 - (ij >> 8), j = bb - 1 - (ij & 255);
    const int s0 = mat ? d.rf : 0, s1 = mat ? S : d.rf;
    Tc* M = mat ? Bm : A;
    Tc re = Tc(0), im = Tc(0);
#pragma unroll 8
    for (int s = s0; s < s1; ++s) {
      const To* Q = P + (size_t)s * V * V;
      if constexpr (!CPLX) {
        re += (Tc)Q[i * V + j];
      } else {
        re += (Tc)Q[i * V + j] + (Tc)Q[(bb + i) * V + bb + j];
        im += (Tc)Q[i * V + bb + j] - (Tc)Q[j * V + bb + i];
      }
    }
    if constexpr (!CPLX) {
      M[j * BMAX + i] = re;
      M[i * BMAX + j] = re;
    } else {
      M[2 * (j * BMAX + i)] = re;
      M[2 * (j * BMAX + i) + 1] = (i == j) ? Tc(0) : im;
      M[2 * (i * BMAX + j)] = re;
      M[2 * (i * BMAX + j) + 1] = (i == j) ? Tc(0) : -im;
    }
  }
  __syncthreads();

  // 2. Choleskys A-hat = R^* R and B-hat = R^* R (upper R) side by side,
  //    1/sqrt from one rsqrt, the trailing updates as packed lists.  FP32:
  //    one warp per matrix, warp barriers only; the update scales the two
  //    row entries it reads, then the row is stored scaled.  FP64: the pivots
  //    of A and B on warps 0 and 1 (two SM sub-partitions; the pivot chain is
  //    the serial part), the row k of R scaled in its own pass before the
  //    block-wide update (one FP64 multiply per entry).  A non-positive pivot
  //    fails the visit.  Strict lower triangles are not read afterwards
  //    (zeroed in step 3).
  auto update = [&](int k) {  // row k already scaled
    const int rem = bb - k - 1;
    const int nrem = rem * (rem + 1) / 2;
    for (int t = threadIdx.x; t < 2 * nrem; t += blockDim.x) {
      const int mat = t >= nrem ? 1 : 0;
      const int ij = s_tri[t - mat * nrem];
      const int i = k + 1 + (ij & 255), j = k + 1 + (ij >> 8);
      Tc* M = mat ? Bm : A;
      if constexpr (!CPLX) {
        M[j * BMAX + i] = p_fma(-M[i * BMAX + k], M[j * BMAX + k], M[j * BMAX + i]);
      } else {
        // M_ij -= conj(R_ki) R_kj
        const Tc kir = M[2 * (i * BMAX + k)], kii = M[2 * (i * BMAX + k) + 1];
        const Tc kjr = M[2 * (j * BMAX + k)], kji = M[2 * (j * BMAX + k) + 1];
        M[2 * (j * BMAX + i)] -= kir * kjr + kii * kji;
        M[2 * (j * BMAX + i) + 1] -= kir * kji - kii * kjr;
      }
    }
  };
  auto scale_row = [&](int k, Tc inv0, Tc inv1) {
    const int rem = bb - k - 1;
    for (int t = threadIdx.x; t < 2 * rem; t += blockDim.x) {
      const int mat = t >= rem ? 1 : 0;
      const int j = k + 1 + t - mat * rem;
      Tc* M = mat ? Bm : A;
      const Tc inv = mat ? inv1 : inv0;
      M[E * (j * BMAX + k)] *= inv;
      if constexpr (CPLX) M[E * (j * BMAX + k) + 1] *= inv;
    }
  };
  if constexpr (P32) {
    // FP32: eight warps per matrix (A on warps 0-7, B on warps 8-15), one
    // named barrier of the eight per step.  Lane l holds rows l, l + 32, ...;
    // warp w of a matrix updates the columns j = w (mod 8) beyond k: its
    // rows' entries of column j, with row k's entry of column j read as a
    // broadcast (the products of the block-wide form below: both row-k
    // factors scaled by 1/sqrt(pivot), then one fma).  After the barrier
    // each warp stores row k's entries of its columns scaled; the next step
    // reads only row k + 1 and its pivot, which the barrier has published.
    static_assert(INNER_THREADS == 512, "eight warps per matrix");
    constexpr int RPL = (BMAX + 31) / 32;
    const int mat = warp >> 3, wl = warp & 7;
    Tc* M = mat ? Bm : A;
    bool bad = false;
    for (int k = 0; k < bb; ++k) {
      const Tc dkk = M[E * (k * BMAX + k)];
      if (!(dkk > Tc(0)) || !isfinite(dkk)) {
        bad = true;  // the same for the eight warps of the matrix
        break;
      }
      const Tc inv = p_rsqrt(dkk);
      Tc rr[RPL], ri[RPL];  // R_ki of this lane's rows i (scaled)
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int ir = lane + 32 * q;
        rr[q] = ri[q] = Tc(0);
        if (ir > k && ir < bb) {
          rr[q] = M[E * (ir * BMAX + k)] * inv;
          if constexpr (CPLX) ri[q] = M[E * (ir * BMAX + k) + 1] * inv;
        }
      }
      // this warp's columns beyond k: jc = j0 + 8 u, loads before stores
      const int j0 = k + 1 + ((wl - (k + 1)) & 7);
      constexpr int CG = (BMAX + 7) / 8;
      Tc kjr[CG], kji[CG], mr[RPL][CG], mi[RPL][CG];
#pragma unroll
      for (int u = 0; u < CG; ++u) {
        const int jc = j0 + 8 * u;
        kjr[u] = kji[u] = Tc(0);
        if (jc < bb) {
          kjr[u] = M[E * (jc * BMAX + k)] * inv;
          if constexpr (CPLX) kji[u] = M[E * (jc * BMAX + k) + 1] * inv;
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int ir = lane + 32 * q;
          mr[q][u] = mi[q][u] = Tc(0);
          if (ir > k && ir <= jc && jc < bb) {
            mr[q][u] = M[E * (jc * BMAX + ir)];
            if constexpr (CPLX) mi[q][u] = M[E * (jc * BMAX + ir) + 1];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < CG; ++u) {
        const int jc = j0 + 8 * u;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int ir = lane + 32 * q;
          if (ir > k && ir <= jc && jc < bb) {
            if constexpr (!CPLX) {
              M[jc * BMAX + ir] = p_fma(-rr[q], kjr[u], mr[q][u]);
            } else {
              M[2 * (jc * BMAX + ir)] = mr[q][u] - (rr[q] * kjr[u] + ri[q] * kji[u]);
              M[2 * (jc * BMAX + ir) + 1] = mi[q][u] - (rr[q] * kji[u] - ri[q] * kjr[u]);
            }
          }
        }
      }
      if (mat)  // warp-uniform: each matrix's eight warps on their own barrier
        asm volatile("bar.sync 3, 256;\n" ::: "memory");
      else
        asm volatile("bar.sync 2, 256;\n" ::: "memory");
      if (wl == 0 && lane == 0) M[E * (k * BMAX + k)] = dkk * inv;
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < CG; ++u) {
          const int jc = j0 + 8 * u;
          if (jc < bb) {
            M[E * (jc * BMAX + k)] = kjr[u];
            if constexpr (CPLX) M[E * (jc * BMAX + k) + 1] = kji[u];
          }
        }
      }
    }
    if (bad && wl == 0 && lane == 0) s_bad = 1;
    __syncthreads();
  } else
  for (int k = 0; k < bb; ++k) {
    if (threadIdx.x == 0 || threadIdx.x == 32) {
      const int mat = threadIdx.x >> 5;
      Tc* M = mat ? Bm : A;
      const Tc dkk = M[E * (k * BMAX + k)];
      if (!(dkk > Tc(0)) || !isfinite(dkk)) {
        s_bad = 1;
        s_inv[mat] = Tc(0);
      } else {
        const Tc inv = p_rsqrt(dkk);
        M[E * (k * BMAX + k)] = dkk * inv;
        s_inv[mat] = inv;
      }
    }
    __syncthreads();
    if (s_bad) break;
    scale_row(k, s_inv[0], s_inv[1]);
    __syncthreads();
    update(k);
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) {
      b.flags[slot] = 0;
      atomicAdd(&b.ctr[prm.chol_skip ? 3 : 2], 1ull);
    }
    return;
  }

  // 3. F-hat, G-hat (inner data type, in place), Z-hat = I
  {
    Tc tmpA[E * BMAX * BMAX / NTH + 1], tmpB[E * BMAX * BMAX / NTH + 1];
    int cnt = 0;
    for (int idx = threadIdx.x; idx < E * bb * bb; idx += blockDim.x, ++cnt) {
      const int j = idx / (E * bb), i = (idx % (E * bb)) / E, part = idx % E;
      const bool low = i > j;
      tmpA[cnt] = low ? Tc(0) : A[E * (j * BMAX + i) + part];
      tmpB[cnt] = low ? Tc(0) : Bm[E * (j * BMAX + i) + part];
    }
    __syncthreads();
    Ti* Fh = reinterpret_cast<Ti*>(Ad);
    Ti* Gh = reinterpret_cast<Ti*>(Bd);
    cnt = 0;
    for (int idx = threadIdx.x; idx < E * bb * bb; idx += blockDim.x, ++cnt) {
      Fh[idx] = static_cast<Ti>(tmpA[cnt]);
      Gh[idx] = static_cast<Ti>(tmpB[cnt]);
      Zh[idx] = Ti(0);
    }
    __syncthreads();
  }
  Ti* Fh = reinterpret_cast<Ti*>(Ad);  // bb x bb, ld bb (E scalars per element)
  Ti* Gh = reinterpret_cast<Ti*>(Bd);

  // 4. inner prescale (variant 0): z_j = 1/||g-hat_j||
  for (int j = warp; j < bb; j += nwarps) {
    Ti s = Ti(0);
    for (int r = lane; r < E * bb; r += 32) {
      const Ti v = Gh[j * E * bb + r];
      s += v * v;
    }
    s = warp_sum(s);
    const Ti zj = Ti(1) / sqrt(s);
    for (int r = lane; r < E * bb; r += 32) {
      Fh[j * E * bb + r] *= zj;
      Gh[j * E * bb + r] *= zj;
    }
    if (lane == 0) Zh[j * E * bb + E * j] = zj;
  }
  __syncthreads();

  const int M = bb + (bb & 1);
  const int npairs = M / 2;
  const double tol = prm.tol > 0.0 ? prm.tol : prm.eps * sqrt((double)bb);
  for (int idx = threadIdx.x; idx < (M - 1) * npairs; idx += blockDim.x) {
    int i, j;
    rr_pair(M, idx / npairs, idx % npairs, i, j);
    s_pair[idx / npairs][idx % npairs][0] = (unsigned char)i;
    s_pair[idx / npairs][idx % npairs][1] = (unsigned char)j;
  }
  __syncthreads();
  for (int sw = 0; sw < prm.inner_max; ++sw) {
    int sweep_all = 0;
    if constexpr (P32) {
      // FP32 sweeps: one pair per half-warp (16 lanes; rows hl, hl + 16):
      // both halves of a warp form their pair's dot products, take its 2x2
      // parameters (every lane of the half the same FP32 values) and update
      // its columns in the same instructions, so a step issues half the
      // instructions of a warp per pair; one barrier per step; counters per
      // half-warp
      int n_rot = 0, n_big = 0;
      bool chg = false;
      const float tolf = (float)tol;
      const int hl = lane & 15;
      for (int st = 0; st < M - 1; ++st) {
        for (int kb = 2 * warp; kb < npairs; kb += 2 * nwarps) {
          const int k = kb + (lane >> 4);
          int i = 0, j = 0;
          bool valid = false;
          if (k < npairs) {
            i = s_pair[st][k][0];
            j = s_pair[st][k][1];
            valid = j < bb;
          }
          float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          float w2[2] = {0.0f, 0.0f};
          if constexpr (!CPLX) {
            if (valid) {
              for (int r = hl; r < bb; r += 16) {
                const float fi = Fh[i * bb + r], fj = Fh[j * bb + r];
                v[0] += fi * fi;
                v[1] += fj * fj;
                v[2] += fi * fj;
                v[3] += Gh[i * bb + r] * Gh[j * bb + r];
              }
            }
            half_sum4_all(v);
          } else {
            if (valid) {
              for (int r = hl; r < bb; r += 16) {
                const float fir = Fh[2 * (i * bb + r)], fii = Fh[2 * (i * bb + r) + 1];
                const float fjr = Fh[2 * (j * bb + r)], fji = Fh[2 * (j * bb + r) + 1];
                const float gir = Gh[2 * (i * bb + r)], gii = Gh[2 * (i * bb + r) + 1];
                const float gjr = Gh[2 * (j * bb + r)], gji = Gh[2 * (j * bb + r) + 1];
                v[0] += fir * fir + fii * fii;
                v[1] += fjr * fjr + fji * fji;
                v[2] += fir * fjr + fii * fji;
                v[3] += fir * fji - fii * fjr;
                w2[0] += gir * gjr + gii * gji;
                w2[1] += gir * gji - gii * gjr;
              }
            }
            half_sum4_all(v);
            w2[0] = half_sum(w2[0]);
            w2[1] = half_sum(w2[1]);
          }
          if (!valid) continue;
          PivotOutT<float> o;
          if constexpr (!CPLX) {
            // the two chains of the real parameters have independent inputs:
            // both issued here, they overlap (chain B is not used unless
            // chain A rotates, which is what pivot_real computes)
            const RealChainAT<float> ra = real_chain_a(v[0], v[1], v[2], v[3], tolf);
            float xi, eta;
            real_chain_b(v[3], xi, eta);
            o = real_combine(v[0], v[1], v[2], v[3], ra, xi, eta, false, true, prm.crit2);
          } else {
            o = pivot_cplx<float>(v[0], v[1], v[2], v[3], w2[0], w2[1], tolf, prm.sort, true, prm.crit2);
          }
          const bool rot = o.flags & PV_ROT;
          bool swp = o.flags & PV_SWAP;
          if (o.flags & PV_FAIL) {
            if (hl == 0) s_ctr[2] = 1;
            continue;
          }
          if constexpr (!CPLX) {
            // sort decision: transformed diagonal of A-hat (Sec. 3.5.3)
            if (prm.sort) {
              if (rot) {
                const float d1 = o.z11 * o.z11 * v[0] + 2.0f * o.z11 * o.z21 * v[2] + o.z21 * o.z21 * v[1];
                const float d2 = o.z12 * o.z12 * v[0] + 2.0f * o.z22 * o.z12 * v[2] + o.z22 * o.z22 * v[1];
                swp = d1 < d2;
              } else {
                swp = v[0] < v[1];
              }
            }
          }
          n_rot += rot ? 1 : 0;
          n_big += (o.flags & PV_BIG) ? 1 : 0;
          chg = chg || rot || swp;
          if (!rot && !swp) continue;
          const float z11 = o.z11, z12 = o.z12, z21 = o.z21, z22 = o.z22, z12i = o.z12i, z21i = o.z21i;
          // the three matrices' operands of a row are loaded before any of
          // them is stored (shared loads are not reordered past stores that
          // may alias)
          float* Ym[3] = {reinterpret_cast<float*>(Fh), reinterpret_cast<float*>(Gh), reinterpret_cast<float*>(Zh)};
          for (int r = hl; r < bb; r += 16) {
            if constexpr (!CPLX) {
              float yi[3], yj[3];
#pragma unroll
              for (int mm = 0; mm < 3; ++mm) {
                yi[mm] = Ym[mm][i * bb + r];
                yj[mm] = Ym[mm][j * bb + r];
              }
#pragma unroll
              for (int mm = 0; mm < 3; ++mm) {
                float ni = yi[mm], nj = yj[mm];
                if (rot) {
                  ni = fmaf(yj[mm], z21, yi[mm] * z11);
                  nj = fmaf(yi[mm], z12, yj[mm] * z22);
                }
                Ym[mm][i * bb + r] = swp ? nj : ni;
                Ym[mm][j * bb + r] = swp ? ni : nj;
              }
            } else {
              float yir[3], yii[3], yjr[3], yji[3];
#pragma unroll
              for (int mm = 0; mm < 3; ++mm) {
                yir[mm] = Ym[mm][2 * (i * bb + r)];
                yii[mm] = Ym[mm][2 * (i * bb + r) + 1];
                yjr[mm] = Ym[mm][2 * (j * bb + r)];
                yji[mm] = Ym[mm][2 * (j * bb + r) + 1];
              }
#pragma unroll
              for (int mm = 0; mm < 3; ++mm) {
                float nir = yir[mm], nii = yii[mm], njr = yjr[mm], nji = yji[mm];
                if (rot) {
                  nir = fmaf(yjr[mm], z21, fmaf(-yji[mm], z21i, yir[mm] * z11));
                  nii = fmaf(yjr[mm], z21i, fmaf(yji[mm], z21, yii[mm] * z11));
                  njr = fmaf(yir[mm], z12, fmaf(-yii[mm], z12i, yjr[mm] * z22));
                  nji = fmaf(yir[mm], z12i, fmaf(yii[mm], z12, yji[mm] * z22));
                }
                Ym[mm][2 * (i * bb + r)] = swp ? njr : nir;
                Ym[mm][2 * (i * bb + r) + 1] = swp ? nji : nii;
                Ym[mm][2 * (j * bb + r)] = swp ? nir : njr;
                Ym[mm][2 * (j * bb + r) + 1] = swp ? nii : nji;
              }
            }
          }
        }
        __syncthreads();
        if (s_ctr[2]) break;
      }
      if (hl == 0) {
        if (n_rot) atomicAdd(&s_ctr[0], n_rot);
        if (n_big) atomicAdd(&s_ctr[1], n_big);
        if (chg) s_ctr[3] = 1;
      }
    } else
    for (int st = 0; st < M - 1; ++st) {
      for (int k = warp; k < npairs; k += nwarps) {
        const int i = s_pair[st][k][0], j = s_pair[st][k][1];
        if (j >= bb) continue;
        Ti v[4] = {Ti(0), Ti(0), Ti(0), Ti(0)};
        Ti w2[2] = {Ti(0), Ti(0)};
        if constexpr (!CPLX) {
          for (int r = lane; r < bb; r += 32) {
            const Ti fi = Fh[i * bb + r], fj = Fh[j * bb + r];
            v[0] += fi * fi;
            v[1] += fj * fj;
            v[2] += fi * fj;
            v[3] += Gh[i * bb + r] * Gh[j * bb + r];
          }
          warp_sum4(v);
        } else {
          for (int r = lane; r < bb; r += 32) {
            const Ti fir = Fh[2 * (i * bb + r)], fii = Fh[2 * (i * bb + r) + 1];
            const Ti fjr = Fh[2 * (j * bb + r)], fji = Fh[2 * (j * bb + r) + 1];
            const Ti gir = Gh[2 * (i * bb + r)], gii = Gh[2 * (i * bb + r) + 1];
            const Ti gjr = Gh[2 * (j * bb + r)], gji = Gh[2 * (j * bb + r) + 1];
            v[0] += fir * fir + fii * fii;
            v[1] += fjr * fjr + fji * fji;
            v[2] += fir * fjr + fii * fji;
            v[3] += fir * fji - fii * fjr;
            w2[0] += gir * gjr + gii * gji;
            w2[1] += gir * gji - gii * gjr;
          }
          warp_sum4(v);
          w2[0] = warp_sum(w2[0]);
          w2[1] = warp_sum(w2[1]);
        }
        if (lane == 0) {
          PivInT<Ti> p;
          p.a11 = v[0]; p.a22 = v[1]; p.ar = v[2];
          if constexpr (CPLX) { p.ai = v[3]; p.br = w2[0]; p.bi = w2[1]; }
          else { p.ai = Ti(0); p.br = v[3]; p.bi = Ti(0); }
          pin[k] = p;
        }
      }
      __syncthreads();
      // 2x2 parameters in FP64, one pair per lane (npairs <= 32): real pivots
      // run their two independent chains on warps 0 and 1 (two SM
      // sub-partitions), complex pivots on warp 0.  Counters are
      // warp-aggregated.
      auto count_flags = [&](int fl) {
        const unsigned rot = __ballot_sync(FULL, fl & PV_ROT), big = __ballot_sync(FULL, fl & PV_BIG);
        const unsigned bad = __ballot_sync(FULL, fl & PV_FAIL), chg = __ballot_sync(FULL, fl & (PV_ROT | PV_SWAP));
        if (lane == 0) {
          s_ctr[0] += __popc(rot);
          s_ctr[1] += __popc(big);
          if (bad) s_ctr[2] = 1;
          if (chg) s_ctr[3] = 1;
        }
      };
      if (warp <= 1) {
        const bool act = lane < npairs && s_pair[st][lane < npairs ? lane : 0][1] < bb;
        int fl = 0;
        PivotOut o;
        bool have = false;
        if constexpr (!CPLX) {
          if (warp == 1) {
            double xi = 0.0, eta = 0.0;
            if (act) real_chain_b((double)pin[lane].br, xi, eta);
            s_xi[lane] = xi;
            s_eta[lane] = eta;
            param_pair_barrier();
          } else {
            RealChainA r;
            double a11 = 0.0, a22 = 0.0, a12 = 0.0, x = 0.0;
            if (act) {
              const PivInT<Ti> p = pin[lane];
              a11 = p.a11; a22 = p.a22; a12 = p.ar; x = p.br;
              r = real_chain_a(a11, a22, a12, x, tol);
            }
            param_pair_barrier();
            if (act) {
              // FP32 bulk sweeps: the sort decision (a heuristic) is taken in
              // FP32 by the pair's own warp, off this FP64 critical path
              constexpr bool sort_here = !std::is_same<Ti, float>::value;
              o = real_combine(a11, a22, a12, x, r, s_xi[lane], s_eta[lane], sort_here && prm.sort, prm.f32cls,
                               prm.crit2);
              have = true;
            }
          }
        } else {
          if (warp == 0 && act) {
            const PivInT<Ti> p = pin[lane];
            o = pivot_cplx((double)p.a11, (double)p.a22, (double)p.ar, (double)p.ai, (double)p.br, (double)p.bi, tol,
                           prm.sort, prm.f32cls, prm.crit2);
            have = true;
          }
        }
        if (warp == 0) {
          if (have) {
            PivZ<Ti> q;
            q.z11 = (Ti)o.z11; q.z12 = (Ti)o.z12; q.z21 = (Ti)o.z21; q.z22 = (Ti)o.z22;
            if constexpr (CPLX) { q.z12i = (Ti)o.z12i; q.z21i = (Ti)o.z21i; }
            else { q.z12i = Ti(0); q.z21i = Ti(0); }
            q.flags = o.flags;
            pout[lane] = q;
            fl = o.flags;
          }
          count_flags(fl);
        }
      }
      __syncthreads();
      for (int k = warp; k < npairs; k += nwarps) {
        const int i = s_pair[st][k][0], j = s_pair[st][k][1];
        if (j >= bb) continue;
        const PivZ<Ti> o = pout[k];
        const bool rot = o.flags & PV_ROT;
        bool swp = o.flags & PV_SWAP;
        if constexpr (!CPLX && std::is_same<Ti, float>::value) {
          // FP32 bulk sweeps: transformed diagonal of A-hat (Sec. 3.5.3) in FP32
          if (prm.sort) {
            const PivInT<Ti> p = pin[k];
            if (rot) {
              const float d1 = o.z11 * o.z11 * p.a11 + 2.0f * o.z11 * o.z21 * p.ar + o.z21 * o.z21 * p.a22;
              const float d2 = o.z12 * o.z12 * p.a11 + 2.0f * o.z22 * o.z12 * p.ar + o.z22 * o.z22 * p.a22;
              swp = d1 < d2;
            } else if (!(o.flags & PV_FAIL)) {
              swp = p.a11 < p.a22;
            }
            if (swp && lane == 0) s_ctr[3] = 1;
          }
        }
        if (!rot && !swp) continue;
        const Ti z11 = o.z11, z12 = o.z12, z21 = o.z21, z22 = o.z22;
        const Ti z12i = o.z12i, z21i = o.z21i;
        auto upd = [&](Ti* Y) {
          for (int r = lane; r < bb; r += 32) {
            if constexpr (!CPLX) {
              const Ti yi = Y[i * bb + r], yj = Y[j * bb + r];
              Ti ni = yi, nj = yj;
              if (rot) {
                ni = fma(yj, z21, yi * z11);
                nj = fma(yi, z12, yj * z22);
              }
              Y[i * bb + r] = swp ? nj : ni;
              Y[j * bb + r] = swp ? ni : nj;
            } else {
              const Ti yir = Y[2 * (i * bb + r)], yii = Y[2 * (i * bb + r) + 1];
              const Ti yjr = Y[2 * (j * bb + r)], yji = Y[2 * (j * bb + r) + 1];
              Ti nir = yir, nii = yii, njr = yjr, nji = yji;
              if (rot) {
                nir = fma(yjr, z21, fma(-yji, z21i, yir * z11));
                nii = fma(yjr, z21i, fma(yji, z21, yii * z11));
                njr = fma(yir, z12, fma(-yii, z12i, yjr * z22));
                nji = fma(yir, z12i, fma(yii, z12, yji * z22));
              }
              Y[2 * (i * bb + r)] = swp ? njr : nir;
              Y[2 * (i * bb + r) + 1] = swp ? nji : nii;
              Y[2 * (j * bb + r)] = swp ? nir : njr;
              Y[2 * (j * bb + r) + 1] = swp ? nii : nji;
            }
          }
        };
        upd(Fh);
        upd(Gh);
        upd(Zh);
      }
      __syncthreads();
      if (s_ctr[2]) break;
    }
    __syncthreads();
    sweep_all = s_ctr[0];
    const int fail = s_ctr[2];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_ctr[0]) atomicAdd(&b.ctr[0], (unsigned long long)s_ctr[0]);
      if (s_ctr[1]) atomicAdd(&b.ctr[1], (unsigned long long)s_ctr[1]);
      s_ctr[0] = 0;
      s_ctr[1] = 0;
    }
    __syncthreads();
    if (fail) {
      if (threadIdx.x == 0) {
        b.flags[slot] = 0;
        atomicAdd(&b.ctr[prm.chol_skip ? 3 : 2], 1ull);
      }
      return;
    }
    if (sweep_all == 0) break;
  }

  // 5. Theta-tilde: theta_j = (||f-hat_j||^2 + ||g-hat_j||^2)^{-1/2}, Z-tilde = Z-hat Theta
  const bool changed = s_ctr[3] != 0;
  if (!changed) {
    if (threadIdx.x == 0) b.flags[slot] = 0;
    return;
  }
  for (int j = warp; j < bb; j += nwarps) {
    Ti s = Ti(0);
    for (int r = lane; r < E * bb; r += 32) {
      const Ti f = Fh[j * E * bb + r], g = Gh[j * E * bb + r];
      s += f * f + g * g;
    }
    s = warp_sum(s);
    const Ti th = Ti(1) / sqrt(s);
    for (int r = lane; r < E * bb; r += 32) Zh[j * E * bb + r] *= th;
  }
  __syncthreads();
  // 6. real view of Z-tilde, row-major V x V, zero padded
  To* zt = static_cast<To*>(b.ztil) + (size_t)slot * V * V;
  for (int idx = threadIdx.x; idx < V * V; idx += blockDim.x) {
    const int k = idx / V, j = idx % V;
    To val = To(0);
    if constexpr (!CPLX) {
      if (k < bb && j < bb) val = (To)Zh[j * bb + k];
    } else {
      const bool kr = k < bb, jr = j < bb;
      const int kk = kr ? k : k - bb, jj = jr ? j : j - bb;
      if (kk < bb && jj < bb) {
        const Ti zr = Zh[2 * (jj * bb + kk)], zi = Zh[2 * (jj * bb + kk) + 1];
        if (kr && jr) val = (To)zr;
        else if (kr && !jr) val = (To)zi;
        else if (!kr && jr) val = (To)(-zi);
        else val = (To)zr;
      }
    }
    zt[idx] = val;
  }
  if (threadIdx.x == 0) {
    b.flags[slot] = 1;
    atomicAdd(&b.ctr[5], 1ull);
  }
}

// ------------------------------------------- inner, two-CTA cluster ----
// The FP64 pivot step of one pair on a cluster of two CTAs, i.e. two SMs.
// On sm_103a an SM issues about one FP64 warp instruction per 16 cycles, so
// one CTA per pair leaves the dots and column updates of every inner step
// throughput-bound on one SM while, with 64 pairs, 88 of the 152 SMs idle.
// Here the rows of F-hat, G-hat and Z-hat are split between the two CTAs:
//   * both CTAs sum the Gram partials and factor A-hat and B-hat (the same
//     fixed-order arithmetic, so the same bits), then keep their own half of
//     the rows of the Cholesky factors;
//   * per inner step each CTA forms the dot products over its rows, two
//     pairs per warp (one per 16-lane half), and the two halves of every
//     dot product are added through distributed shared memory -- a + b is
//     the same in both CTAs, so both compute the same 2x2 parameters and
//     take the same decisions (sorting, counters, stopping) without further
//     exchange;
//   * each CTA applies the transformations to its own rows; Theta-tilde
//     takes one more exchange of partial column norms.
// One cluster barrier per inner step; the partial dot products are double
// buffered so that a CTA never overwrites values its peer has yet to read.
// Every exit after the first exchange passes one more cluster barrier, so no
// CTA leaves while its peer may still read its shared memory.
constexpr int INNER2_THREADS = 256;

// Reduce-scatter of four per-lane values inside each 16-lane half of a warp
// (2 + 1 + 1 + 1 = 5 adds, fixed order): value q = 2 (lane bit 3) + (lane
// bit 2), summed over the half, is returned on its four lanes.
__device__ __forceinline__ double half_sum4(const double v[4]) {
  const int lane = threadIdx.x & 31;
  const bool b8 = lane & 8;
  const double s0 = b8 ? v[0] : v[2], s1 = b8 ? v[1] : v[3];
  double k0 = b8 ? v[2] : v[0], k1 = b8 ? v[3] : v[1];
  k0 += __shfl_xor_sync(FULL, s0, 8);
  k1 += __shfl_xor_sync(FULL, s1, 8);
  const bool b4 = lane & 4;
  const double sx = b4 ? k0 : k1;
  double k = b4 ? k1 : k0;
  k += __shfl_xor_sync(FULL, sx, 4);
  k += __shfl_xor_sync(FULL, k, 2);
  k += __shfl_xor_sync(FULL, k, 1);
  return k;
}

template <bool CPLX, int V>
size_t inner2_smem() {
  constexpr int E = CPLX ? 2 : 1;
  constexpr int BMAX = CPLX ? V / 2 : V;
  constexpr int RH = (BMAX + 1) / 2;
  constexpr int NPMAX = BMAX / 2;
  return sizeof(double) * (2 * E * BMAX * BMAX + 3 * E * RH * BMAX + 2 * NPMAX * 16 + 2 * BMAX + 64) +
         sizeof(PivInT<double>) * (NPMAX + 1) + sizeof(PivZ<double>) * (NPMAX + 1) +
         sizeof(uint16_t) * (BMAX * (BMAX + 1) / 2) + 16;
}

template <bool CPLX, int V>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(INNER2_THREADS)
    k_inner2(BlkDims d, BlkBuffers b, int step, InnerParams prm, BlkBatch bt) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int E = CPLX ? 2 : 1;
  constexpr int BMAX = CPLX ? V / 2 : V;  // max columns of the pair
  constexpr int RH = (BMAX + 1) / 2;      // max rows of a CTA
  constexpr int NPMAX = BMAX / 2;         // max pairs of an inner step
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);  // E BMAX x BMAX, column-major (ld BMAX)
  double* Bm = A + E * BMAX * BMAX;
  double* Fl = Bm + E * BMAX * BMAX;                // own rows: E RH x BMAX, column-major
  double* Gl = Fl + E * RH * BMAX;
  double* Zl = Gl + E * RH * BMAX;
  double* part = Zl + E * RH * BMAX;                // [2][NPMAX][16] partial dot products
  double* nrm = part + 2 * NPMAX * 16;              // [BMAX] partial column norms
  double* th = nrm + BMAX;                          // [BMAX] prescale z_j, then theta_j
  double* s_d = th + BMAX;                          // [2][32] D-hat of each pair of a step
  PivInT<double>* pin = reinterpret_cast<PivInT<double>*>(s_d + 64);
  PivZ<double>* pout = reinterpret_cast<PivZ<double>*>(pin + NPMAX + 1);
  uint16_t* s_tri = reinterpret_cast<uint16_t*>(pout + NPMAX + 1);
  __shared__ int s_ctr[4];  // all, big, fail, any-change
  __shared__ double s_inv[2];
  __shared__ int s_bad;
  __shared__ double s_xi[32], s_eta[32];
  __shared__ unsigned char s_pair[63][32][2];

  const int rank = (int)cluster.block_rank();
  int slot;
  if (!batch_item(bt, blockIdx.x >> 1, step, d, b, slot, &prm)) return;  // the same answer in both CTAs
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  const int bb = pc.bb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int S = d.rf + d.rg;
  const double* P = static_cast<const double*>(b.partial) + (size_t)slot * S * V * V;
  const bool lead = rank == 0 && threadIdx.x == 0;
  if (threadIdx.x < 4) s_ctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_bad = 0;
  if (lead) atomicAdd(&b.ctr[4], 1ull);
  const int nup = bb * (bb + 1) / 2;
  for (int u = threadIdx.x; u < nup; u += blockDim.x) {
    int i, j;
    unpack_upper(u, i, j);
    s_tri[u] = (uint16_t)(i | (j << 8));
  }
  __syncthreads();

  // 1. fixed-order sum of the partials into A-hat and B-hat (both triangles)
  for (int t = threadIdx.x; t < 2 * nup; t += blockDim.x) {
    const int mat = t >= nup ? 1 : 0;
    const int ij = s_tri[nup - 1 - (t - mat * nup)];
    const int i = bb - 1 - (ij >> 8), j = bb - 1 - (ij & 255);
    const int s0 = mat ? d.rf : 0, s1 = mat ? S : d.rf;
    double* M = mat ? Bm : A;
    double re = 0.0, im = 0.0;
#pragma unroll 8
    for (int sp = s0; sp < s1; ++sp) {
      const double* Q = P + (size_t)sp * V * V;
      if constexpr (!CPLX) {
        re += Q[i * V + j];
      } else {
        re += Q[i * V + j] + Q[(bb + i) * V + bb + j];
        im += Q[i * V + bb + j] - Q[j * V + bb + i];
      }
    }
    if constexpr (!CPLX) {
      M[j * BMAX + i] = re;
      M[i * BMAX + j] = re;
    } else {
      M[2 * (j * BMAX + i)] = re;
      M[2 * (j * BMAX + i) + 1] = (i == j) ? 0.0 : im;
      M[2 * (i * BMAX + j)] = re;
      M[2 * (i * BMAX + j) + 1] = (i == j) ? 0.0 : -im;
    }
  }
  __syncthreads();

  // 2. Choleskys of A-hat and B-hat side by side (pivots on warps 0 and 1)
  for (int k = 0; k < bb; ++k) {
    if (threadIdx.x == 0 || threadIdx.x == 32) {
      const int mat = threadIdx.x >> 5;
      double* M = mat ? Bm : A;
      const double dkk = M[E * (k * BMAX + k)];
      if (!(dkk > 0.0) || !isfinite(dkk)) {
        s_bad = 1;
        s_inv[mat] = 0.0;
      } else {
        const double inv = rsqrt(dkk);
        M[E * (k * BMAX + k)] = dkk * inv;
        s_inv[mat] = inv;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int rem = bb - k - 1;
    for (int t = threadIdx.x; t < 2 * rem; t += blockDim.x) {
      const int mat = t >= rem ? 1 : 0;
      const int j = k + 1 + t - mat * rem;
      double* M = mat ? Bm : A;
      const double inv = s_inv[mat];
      M[E * (j * BMAX + k)] *= inv;
      if constexpr (CPLX) M[E * (j * BMAX + k) + 1] *= inv;
    }
    __syncthreads();
    const int nrem = rem * (rem + 1) / 2;
    for (int t = threadIdx.x; t < 2 * nrem; t += blockDim.x) {
      const int mat = t >= nrem ? 1 : 0;
      const int ij = s_tri[t - mat * nrem];
      const int i = k + 1 + (ij & 255), j = k + 1 + (ij >> 8);
      double* M = mat ? Bm : A;
      if constexpr (!CPLX) {
        M[j * BMAX + i] = fma(-M[i * BMAX + k], M[j * BMAX + k], M[j * BMAX + i]);
      } else {
        const double kir = M[2 * (i * BMAX + k)], kii = M[2 * (i * BMAX + k) + 1];
        const double kjr = M[2 * (j * BMAX + k)], kji = M[2 * (j * BMAX + k) + 1];
        M[2 * (j * BMAX + i)] -= kir * kjr + kii * kji;
        M[2 * (j * BMAX + i) + 1] -= kir * kji - kii * kjr;
      }
    }
    __syncthreads();
  }
  if (s_bad) {
    if (lead) {
      b.flags[slot] = 0;
      atomicAdd(&b.ctr[prm.chol_skip ? 3 : 2], 1ull);
    }
    return;  // no shared memory of the peer has been read yet
  }

  // 3. this CTA's rows [r0, r0 + nr) of F-hat = R_A, G-hat = R_B (upper
  //    triangular), Z-hat = 0; the prescale z_j = 1/||g-hat_j|| (variant 0)
  //    from the whole column of R_B, which both CTAs hold
  const int rh = (bb + 1) / 2;
  const int ldl = E * rh;
  const int r0 = rank * rh;
  const int nr = max(0, min(bb, r0 + rh) - r0);
  for (int j = warp; j < bb; j += nwarps) {
    double sq = 0.0;
    for (int r = lane; r < E * (j + 1); r += 32) {
      const double v = Bm[E * j * BMAX + r];
      sq = fma(v, v, sq);
    }
    sq = warp_sum(sq);
    if (lane == 0) th[j] = prm.dscale ? 1.0 : 1.0 / sqrt(sq);  // D-hat variants: no inner prescale
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ldl * bb; idx += blockDim.x) {
    const int j = idx / ldl, rem = idx % ldl, rl = rem / E, pt = rem % E;
    const int r = r0 + rl;
    const bool in = rl < nr && r <= j;
    const double z = th[j];
    Fl[idx] = in ? A[E * (j * BMAX + r) + pt] * z : 0.0;
    Gl[idx] = in ? Bm[E * (j * BMAX + r) + pt] * z : 0.0;
    Zl[idx] = (rl < nr && r == j && pt == 0) ? z : 0.0;
  }
  const int M = bb + (bb & 1);
  const int npairs = M / 2;
  const double tol = prm.tol > 0.0 ? prm.tol : prm.eps * sqrt((double)bb);
  for (int idx = threadIdx.x; idx < (M - 1) * npairs; idx += blockDim.x) {
    int i, j;
    rr_pair(M, idx / npairs, idx % npairs, i, j);
    s_pair[idx / npairs][idx % npairs][0] = (unsigned char)i;
    s_pair[idx / npairs][idx % npairs][1] = (unsigned char)j;
  }
  __syncthreads();

  const int hl = lane & 15;
  int xs = 0;  // exchanges so far: the parity selects the buffer
  bool exchanged = false;
  for (int sw = 0; sw < prm.inner_max; ++sw) {
    for (int st = 0; st < M - 1; ++st, ++xs) {
      const int buf = xs & 1;
      // a. partial dot products over this CTA's rows, one pair per half-warp
      for (int kb = 2 * warp; kb < npairs; kb += 2 * nwarps) {
        const int k = kb + (lane >> 4);
        int i = 0, j = 0;
        bool valid = false;
        if (k < npairs) {
          i = s_pair[st][k][0];
          j = s_pair[st][k][1];
          valid = j < bb;
        }
        // slots of a pair: [0, 4) a11, a22, a12 (complex: Re, Im), real x;
        // [4, 8) the App. A error parts of those (real, enhanced) or Re, Im
        // of b12 (complex); [8, 12) b11, b22 (D-hat) and their error parts
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        double w[4] = {0.0, 0.0, 0.0, 0.0};
        double u[4] = {0.0, 0.0, 0.0, 0.0};
        if (valid && hl < nr) {
          if constexpr (!CPLX) {
            const double fi = Fl[i * ldl + hl], fj = Fl[j * ldl + hl];
            const double gi = Gl[i * ldl + hl], gj = Gl[j * ldl + hl];
            if (prm.enhanced) {  // App. A: RD(a b) and the exact remainder a b - RD(a b), summed apart
              const double p[4] = {fi, fj, fi, gi}, r[4] = {fi, fj, fj, gj};
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                v[t] = __dmul_rd(p[t], r[t]);
                w[t] = fma(p[t], r[t], -v[t]);
              }
              if (prm.dscale) {
                u[0] = __dmul_rd(gi, gi);
                u[1] = __dmul_rd(gj, gj);
                u[2] = fma(gi, gi, -u[0]);
                u[3] = fma(gj, gj, -u[1]);
              }
            } else {
              v[0] = fi * fi;
              v[1] = fj * fj;
              v[2] = fi * fj;
              v[3] = gi * gj;
              if (prm.dscale) {
                u[0] = gi * gi;
                u[1] = gj * gj;
              }
            }
          } else {
            const double fir = Fl[i * ldl + 2 * hl], fii = Fl[i * ldl + 2 * hl + 1];
            const double fjr = Fl[j * ldl + 2 * hl], fji = Fl[j * ldl + 2 * hl + 1];
            const double gir = Gl[i * ldl + 2 * hl], gii = Gl[i * ldl + 2 * hl + 1];
            const double gjr = Gl[j * ldl + 2 * hl], gji = Gl[j * ldl + 2 * hl + 1];
            if (prm.enhanced) {  // the norms by App. A's simpler procedure; off-diagonals ordinary
              v[0] = enh_abs2(fir, fii);
              v[1] = enh_abs2(fjr, fji);
              if (prm.dscale) {
                u[0] = enh_abs2(gir, gii);
                u[1] = enh_abs2(gjr, gji);
              }
            } else {
              v[0] = fma(fir, fir, fii * fii);
              v[1] = fma(fjr, fjr, fji * fji);
              if (prm.dscale) {
                u[0] = fma(gir, gir, gii * gii);
                u[1] = fma(gjr, gjr, gji * gji);
              }
            }
            v[2] = fma(fir, fjr, fii * fji);   // Re(conj(f_i) f_j)
            v[3] = fma(fir, fji, -fii * fjr);  // Im(conj(f_i) f_j)
            w[0] = fma(gir, gjr, gii * gji);
            w[1] = fma(gir, gji, -gii * gjr);
          }
        }
        const bool need_w = CPLX || prm.enhanced;
        const double sv = half_sum4(v);
        const double swv = need_w ? half_sum4(w) : 0.0;
        const double suv = prm.dscale ? half_sum4(u) : 0.0;
        const int q = ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (valid && (lane & 3) == 0) {
          double* pp = part + (buf * NPMAX + k) * 16;
          pp[q] = sv;
          if (need_w) pp[4 + q] = swv;
          if (prm.dscale) pp[8 + q] = suv;
        }
      }
      // b. the two halves of every dot product meet
      cluster.sync();
      exchanged = true;
      {
        const double* peer = cluster.map_shared_rank(part, rank ^ 1);
        constexpr int NV = CPLX ? 6 : 4;
        for (int t = threadIdx.x; t < npairs * NV; t += blockDim.x) {
          const int k = t / NV, qq = t % NV;
          if (s_pair[st][k][1] >= bb) continue;
          const int off = (buf * NPMAX + k) * 16 + qq;
          double tot = part[off] + peer[off];  // a + b = b + a: the same bits in both CTAs
          if (!CPLX && prm.enhanced) tot = tot + (part[off + 4] + peer[off + 4]);
          double* pk = reinterpret_cast<double*>(&pin[k]);  // a11, a22, ar, ai, br, bi
          if constexpr (!CPLX) {
            if (qq < 3) pk[qq] = tot;
            else { pk[4] = tot; pk[3] = 0.0; pk[5] = 0.0; }
          } else {
            pk[qq] = tot;
          }
        }
        if (prm.dscale) {
          // D-hat variants (Sec. 2.1): A' = D A D, B' = D B D with
          // D_kk = 1/sqrt(b_kk) where b_kk != 1 (as the pointwise kernel)
          __syncthreads();
          for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
            if (s_pair[st][k][1] >= bb) continue;
            const int off = (buf * NPMAX + k) * 16 + 8;
            double bii = part[off] + peer[off], bjj = part[off + 1] + peer[off + 1];
            if (!CPLX && prm.enhanced) {
              bii = bii + (part[off + 2] + peer[off + 2]);
              bjj = bjj + (part[off + 3] + peer[off + 3]);
            }
            PivInT<double> pv = pin[k];
            double d1 = 1.0, d2 = 1.0;
            if (bii != 1.0 && bii > 0.0) {
              pv.a11 = pv.a11 / bii;
              d1 = 1.0 / sqrt(bii);
              pv.ar *= d1; pv.ai *= d1; pv.br *= d1; pv.bi *= d1;
            }
            if (bjj != 1.0 && bjj > 0.0) {
              pv.a22 = pv.a22 / bjj;
              d2 = 1.0 / sqrt(bjj);
              pv.ar *= d2; pv.ai *= d2; pv.br *= d2; pv.bi *= d2;
            }
            if (!(bii > 0.0) || !(bjj > 0.0)) {  // a zero column of G-hat: b12 = 1 makes the pivot fail (ENOTPD)
              pv.br = 1.0;
              pv.bi = 0.0;
            }
            pin[k] = pv;
            s_d[k] = d1;
            s_d[32 + k] = d2;
          }
        }
      }
      __syncthreads();
      // c. 2x2 parameters in FP64, one pair per lane (as in the one-CTA kernel)
      auto count_flags = [&](int fl) {
        const unsigned rot = __ballot_sync(FULL, fl & PV_ROT), big = __ballot_sync(FULL, fl & PV_BIG);
        const unsigned bad = __ballot_sync(FULL, fl & PV_FAIL), chg = __ballot_sync(FULL, fl & (PV_ROT | PV_SWAP));
        if (lane == 0) {
          s_ctr[0] += __popc(rot);
          s_ctr[1] += __popc(big);
          if (bad) s_ctr[2] = 1;
          if (chg) s_ctr[3] = 1;
        }
      };
      if (warp <= 1) {
        const bool act = lane < npairs && s_pair[st][lane < npairs ? lane : 0][1] < bb;
        int fl = 0;
        PivotOut o;
        bool have = false;
        if constexpr (!CPLX) {
          if (warp == 1) {
            double xi = 0.0, eta = 0.0;
            if (act) real_chain_b(pin[lane].br, xi, eta);
            s_xi[lane] = xi;
            s_eta[lane] = eta;
            param_pair_barrier();
          } else {
            RealChainA r;
            double a11 = 0.0, a22 = 0.0, a12 = 0.0, x = 0.0;
            if (act) {
              const PivInT<double> pv = pin[lane];
              a11 = pv.a11; a22 = pv.a22; a12 = pv.ar; x = pv.br;
              r = real_chain_a(a11, a22, a12, x, tol);
            }
            param_pair_barrier();
            if (act) {
              o = real_combine(a11, a22, a12, x, r, s_xi[lane], s_eta[lane], prm.sort, prm.f32cls, prm.crit2);
              have = true;
            }
          }
        } else {
          if (warp == 0 && act) {
            const PivInT<double> pv = pin[lane];
            o = pivot_cplx(pv.a11, pv.a22, pv.ar, pv.ai, pv.br, pv.bi, tol, prm.sort, prm.f32cls, prm.crit2);
            have = true;
          }
        }
        if (warp == 0) {
          if (have) {
            if (prm.dscale && (o.flags & PV_ROT)) {  // Z-hat = D Z-hat': rows times D11, D22
              const double d1 = s_d[lane], d2 = s_d[32 + lane];
              o.z11 *= d1; o.z12 *= d1; o.z12i *= d1;
              o.z21 *= d2; o.z21i *= d2; o.z22 *= d2;
            }
            PivZ<double> zq;
            zq.z11 = o.z11; zq.z12 = o.z12; zq.z21 = o.z21; zq.z22 = o.z22;
            zq.z12i = CPLX ? o.z12i : 0.0;
            zq.z21i = CPLX ? o.z21i : 0.0;
            zq.flags = o.flags;
            pout[lane] = zq;
            fl = o.flags;
          }
          count_flags(fl);
        }
      }
      __syncthreads();
      // d. the transformations on this CTA's rows, one pair per half-warp
      for (int kb = 2 * warp; kb < npairs; kb += 2 * nwarps) {
        const int k = kb + (lane >> 4);
        if (k >= npairs || hl >= nr) continue;
        const int i = s_pair[st][k][0], j = s_pair[st][k][1];
        if (j >= bb) continue;
        const PivZ<double> o = pout[k];
        const bool rot = o.flags & PV_ROT, swp = o.flags & PV_SWAP;
        if (!rot && !swp) continue;
        auto upd = [&](double* Y) {
          if constexpr (!CPLX) {
            const double yi = Y[i * ldl + hl], yj = Y[j * ldl + hl];
            double ni = yi, nj = yj;
            if (rot) {
              ni = fma(yj, o.z21, yi * o.z11);
              nj = fma(yi, o.z12, yj * o.z22);
            }
            Y[i * ldl + hl] = swp ? nj : ni;
            Y[j * ldl + hl] = swp ? ni : nj;
          } else {
            const double yir = Y[i * ldl + 2 * hl], yii = Y[i * ldl + 2 * hl + 1];
            const double yjr = Y[j * ldl + 2 * hl], yji = Y[j * ldl + 2 * hl + 1];
            double nir = yir, nii = yii, njr = yjr, nji = yji;
            if (rot) {
              nir = fma(yjr, o.z21, fma(-yji, o.z21i, yir * o.z11));
              nii = fma(yjr, o.z21i, fma(yji, o.z21, yii * o.z11));
              njr = fma(yir, o.z12, fma(-yii, o.z12i, yjr * o.z22));
              nji = fma(yir, o.z12i, fma(yii, o.z12, yji * o.z22));
            }
            Y[i * ldl + 2 * hl] = swp ? njr : nir;
            Y[i * ldl + 2 * hl + 1] = swp ? nji : nii;
            Y[j * ldl + 2 * hl] = swp ? nir : njr;
            Y[j * ldl + 2 * hl + 1] = swp ? nii : nji;
          }
        };
        upd(Fl);
        upd(Gl);
        upd(Zl);
      }
      __syncthreads();
      if (s_ctr[2]) break;
    }
    __syncthreads();
    const int sweep_all = s_ctr[0];
    const int fail = s_ctr[2];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (rank == 0) {
        if (s_ctr[0]) atomicAdd(&b.ctr[0], (unsigned long long)s_ctr[0]);
        if (s_ctr[1]) atomicAdd(&b.ctr[1], (unsigned long long)s_ctr[1]);
      }
      s_ctr[0] = 0;
      s_ctr[1] = 0;
    }
    __syncthreads();
    if (fail) {
      if (lead) {
        b.flags[slot] = 0;
        atomicAdd(&b.ctr[prm.chol_skip ? 3 : 2], 1ull);
      }
      if (exchanged) cluster.sync();
      return;
    }
    if (sweep_all == 0) break;
  }

  // 5. Theta-tilde: theta_j = (||f-hat_j||^2 + ||g-hat_j||^2)^{-1/2} from the
  //    two CTAs' partial norms, Z-tilde = Z-hat Theta-tilde on own rows
  if (s_ctr[3] == 0) {
    if (lead) b.flags[slot] = 0;
    if (exchanged) cluster.sync();
    return;
  }
  for (int j = warp; j < bb; j += nwarps) {
    double sq = 0.0;
    for (int r = lane; r < E * nr; r += 32) {
      const double f = Fl[j * ldl + r], g = Gl[j * ldl + r];
      sq = fma(f, f, fma(g, g, sq));
    }
    sq = warp_sum(sq);
    if (lane == 0) nrm[j] = sq;
  }
  cluster.sync();
  {
    const double* pn = cluster.map_shared_rank(nrm, rank ^ 1);
    for (int j = threadIdx.x; j < bb; j += blockDim.x) th[j] = 1.0 / sqrt(nrm[j] + pn[j]);
  }
  cluster.sync();  // the peer's norms are read: no further access to its shared memory
  // 6. this CTA's rows of the real view of Z-tilde (row-major V x V, zero
  //    padded; CTA 0 also writes the padding rows)
  double* zt = static_cast<double*>(b.ztil) + (size_t)slot * V * V;
  for (int idx = threadIdx.x; idx < V * V; idx += blockDim.x) {
    const int k = idx / V, j = idx % V;
    const int kk = k < bb ? k : k - bb;  // complex: rows bb.. are the -Im / Re block row
    const bool pad = k >= E * bb;
    if (pad ? rank != 0 : (kk < r0 || kk >= r0 + nr)) continue;
    double val = 0.0;
    if (!pad) {
      const int rl = kk - r0;
      if constexpr (!CPLX) {
        if (j < bb) val = Zl[j * ldl + rl] * th[j];
      } else {
        const bool kr = k < bb, jr = j < bb;
        const int jj = jr ? j : j - bb;
        if (jj < bb) {
          const double zr = Zl[jj * ldl + 2 * rl] * th[jj], zi = Zl[jj * ldl + 2 * rl + 1] * th[jj];
          if (kr && jr) val = zr;
          else if (kr && !jr) val = zi;
          else if (!kr && jr) val = -zi;
          else val = zr;
        }
      }
    }
    zt[idx] = val;
  }
  if (lead) {
    b.flags[slot] = 1;
    atomicAdd(&b.ctr[5], 1ull);
  }
}

// --------------------------------------------------------------- apply ----
template <class T, bool CPLX, int V>
__global__ void __launch_bounds__(256) k_apply(BlkDims d, BlkBuffers b, int step, int tile0, BlkBatch bt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int slot;
  if (!batch_item(bt, blockIdx.x, step, d, b, slot)) return;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  if (!b.flags[slot]) return;
  const int tf = (d.mf + TR - 1) / TR, tg = (d.mg + TR - 1) / TR;
  int tile = tile0 + blockIdx.y;
  if (tile >= tf + tg + (d.n + TR - 1) / TR) return;
  T* Y;
  long long ld;
  int m;
  if (tile < tf) {
    Y = static_cast<T*>(b.F); ld = b.ldf; m = d.mf;
  } else if (tile < tf + tg) {
    tile -= tf; Y = static_cast<T*>(b.G); ld = b.ldg; m = d.mg;
  } else {
    tile -= tf + tg; Y = static_cast<T*>(b.Z); ld = b.ldz; m = d.n;
  }
  const int r0 = tile * TR;
  const T* zt = static_cast<const T*>(b.ztil) + (size_t)slot * V * V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if constexpr (std::is_same<T, double>::value) {
    constexpr int LDT = TR + 8, LDM = V + 8;
    double* Ys = reinterpret_cast<double*>(smem_raw);  // [V][LDT] column-major
    double* Ms = Ys + V * LDT;                          // [V][LDM] row-major
    for (int idx = threadIdx.x; idx < V * V; idx += blockDim.x) Ms[(idx / V) * LDM + idx % V] = zt[idx];
    load_tile<T, CPLX, true>(Ys, LDT, Y, ld, m, r0, pc, V);
    __syncthreads();
    constexpr int NJ = V / 8;
    double acc[NJ][2];
#pragma unroll
    for (int t = 0; t < NJ; ++t) acc[t][0] = acc[t][1] = 0.0;
    // warp w owns output rows [8w, 8w+8) of the tile
#pragma unroll 4
    for (int k0 = 0; k0 < V; k0 += 4) {
      const double a = Ys[(k0 + (lane & 3)) * LDT + warp * 8 + (lane >> 2)];
#pragma unroll
      for (int t = 0; t < NJ; ++t) {
        const double bv = Ms[(k0 + (lane & 3)) * LDM + t * 8 + (lane >> 2)];
        dmma884(acc[t][0], acc[t][1], a, bv);
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NJ; ++t) {
      const int r = warp * 8 + (lane >> 2), c = t * 8 + 2 * (lane & 3);
      Ys[c * LDT + r] = acc[t][0];
      Ys[(c + 1) * LDT + r] = acc[t][1];
    }
    __syncthreads();
    if constexpr (!CPLX) {
      for (int idx = threadIdx.x; idx < pc.bb * TR; idx += blockDim.x) {
        const int c = idx / TR, r = idx % TR;
        if (r0 + r < m) Y[(size_t)pc.gcol(c) * ld + r0 + r] = Ys[c * LDT + r];
      }
    } else {
      double2* Y2 = reinterpret_cast<double2*>(Y);
      for (int idx = threadIdx.x; idx < pc.bb * TR; idx += blockDim.x) {
        const int c = idx / TR, r = idx % TR;
        if (r0 + r < m) Y2[(size_t)pc.gcol(c) * ld + r0 + r] = make_double2(Ys[c * LDT + r], Ys[(pc.bb + c) * LDT + r]);
      }
    }
  } else {
    constexpr int LDT = V + 1;
    float* Ws = reinterpret_cast<float*>(smem_raw);  // [TR][LDT] row-major
    float* Ms = Ws + TR * LDT;                        // [V][V] row-major
    for (int idx = threadIdx.x; idx < V * V; idx += blockDim.x) Ms[idx] = zt[idx];
    load_tile<T, CPLX, false>(Ws, LDT, Y, ld, m, r0, pc, V);
    __syncthreads();
    constexpr int NV = V / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][NV];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[u][v] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < V; ++k) {
      float a[4], bv[NV];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Ws[(tx + 16 * u) * LDT + k];
#pragma unroll
      for (int v = 0; v < NV; ++v) bv[v] = Ms[k * V + ty + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[u][v] = fmaf(a[u], bv[v], acc[u][v]);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) Ws[(tx + 16 * u) * LDT + ty + 16 * v] = acc[u][v];
    __syncthreads();
    if constexpr (!CPLX) {
      for (int idx = threadIdx.x; idx < pc.bb * TR; idx += blockDim.x) {
        const int c = idx / TR, r = idx % TR;
        if (r0 + r < m) Y[(size_t)pc.gcol(c) * ld + r0 + r] = Ws[r * LDT + c];
      }
    } else {
      float2* Y2 = reinterpret_cast<float2*>(Y);
      for (int idx = threadIdx.x; idx < pc.bb * TR; idx += blockDim.x) {
        const int c = idx / TR, r = idx % TR;
        if (r0 + r < m) Y2[(size_t)pc.gcol(c) * ld + r0 + r] = make_float2(Ws[r * LDT + c], Ws[r * LDT + pc.bb + c]);
      }
    }
  }
}

template <class T, int V>
size_t gram_smem() {
  // FP32: the staged row tile, or the row groups' partial Grams at the end
  // (groups of (V/4)^2 threads, 256 / (V/4)^2 groups), whichever is larger
  constexpr size_t tile32 = (size_t)TR * (V + 4), parts32 = (size_t)(256 / ((V / 4) * (V / 4)) - 1) * V * V;
  return std::is_same<T, double>::value ? sizeof(double) * V * (TR + 4)
                                        : sizeof(float) * (tile32 > parts32 ? tile32 : parts32);
}
// ---------------------------------------------------------- FP32 kernels ----
// The FP32 bulk sweeps' Gram and apply for real-view widths V = 16 and 32:
// tiles staged in shared memory column by column with 4-byte cp.async
// (coalesced reads of the column-major operands, zero fill outside the
// matrix and beyond the pair's columns), register blocks of 8 x 8 (Gram) and
// 4 x 8 (apply) per thread so that one 16-byte shared load feeds 16 or 32
// FMAs.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit32() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait32_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait32_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Rows [rt, rt + NR) of the real view of [Y_p Y_q] into Ys (column c at
// Ys[c * NR + r]), one source column per warp at a time: rows at or beyond
// rend are zero-filled by the copy, columns beyond the pair are zeroed with
// plain stores.  Complex column c < bb gives real-view columns c (Re) and
// bb + c (Im); the real-view columns [E bb, V) are zero.
template <bool CPLX, int V, int NR, int NW>
__device__ __forceinline__ void stage32(float* Ys, const float* Y, long long ld, int rt, int rend,
                                        const PairCols& pc) {
  static_assert(NR % 32 == 0, "rows per stage");
  constexpr int E = CPLX ? 2 : 1;
  const int bb = pc.bb, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < bb; c += NW) {
    const float* col = Y + (size_t)E * ((size_t)pc.gcol(c) * ld + rt);
#pragma unroll
    for (int q = 0; q < NR / 32; ++q) {
      const int r = lane + 32 * q;
      const bool ok = rt + r < rend;
      if constexpr (!CPLX) {
        cp_async4(&Ys[c * NR + r], ok ? col + r : Y, ok);
      } else {
        cp_async4(&Ys[c * NR + r], ok ? col + 2 * r : Y, ok);
        cp_async4(&Ys[(bb + c) * NR + r], ok ? col + 2 * r + 1 : Y, ok);
      }
    }
  }
  for (int c = E * bb + warp; c < V; c += NW) {
#pragma unroll
    for (int q = 0; q < NR / 32; ++q) Ys[c * NR + lane + 32 * q] = 0.0f;
  }
}

// Gram of a row slab: thread block (bi, bj), bi <= bj, of the (V/8)^2 8 x 8
// blocks (the upper triangle is what the pivot step reads; diagonal blocks
// are full); the 32 lanes of a warp take 4-row chunks of each staged tile,
// R warps per block split the chunks further.  The lanes' sums meet in a
// halving shuffle tree, the R warps' in shared memory (both in a fixed order).
template <int V>
struct Gram32Cfg {
  static constexpr int NB = V / 8, NBT = NB * (NB + 1) / 2;
  static constexpr int R = V == 16 ? 2 : 1;
  static constexpr int THREADS = 32 * NBT * R;
  static constexpr int CPL = 2;             // 4-row chunks per lane and stage
  static constexpr int NR = 128 * R * CPL;  // rows per stage
};

template <bool CPLX, int V>
__global__ void __launch_bounds__(Gram32Cfg<V>::THREADS, 1) k_gram32(BlkDims d, BlkBuffers b, int step, BlkBatch bt) {
  using C = Gram32Cfg<V>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ys = reinterpret_cast<float*>(smem_raw);  // [2][V][NR]; at the end [R-1][NBT][64] sums
  int slot;
  if (!batch_item(bt, blockIdx.x, step, d, b, slot)) return;
  const int s = blockIdx.y;
  if (s >= d.rf + d.rg) return;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  const bool isF = s < d.rf;
  const int m = isF ? d.mf : d.mg;
  const int nsplit = isF ? d.rf : d.rg;
  const int si = isF ? s : s - d.rf;
  const int tiles = (m + TR - 1) / TR;
  const int per = (tiles + nsplit - 1) / nsplit * TR;
  const int r0 = si * per, r1 = min(m, r0 + per);
  const float* Y = static_cast<const float*>(isF ? b.F : b.G);
  const long long ld = isF ? b.ldf : b.ldg;
  float* out = static_cast<float*>(b.partial) + ((size_t)slot * (d.rf + d.rg) + s) * V * V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int blk = warp % C::NBT, rg = warp / C::NBT;
  int bi = 0, bj = blk;
  while (bj >= C::NB - bi) { bj -= C::NB - bi; ++bi; }
  bj += bi;
  const bool diag = bi == bj;
  const int chunk0 = rg * 32 + lane;  // this thread's 4-row chunks of a stage: chunk0 + 32 R c

  float x[64];  // x[8 u + v]: entry (8 bi + u, 8 bj + v) of this thread's rows
#pragma unroll
  for (int e = 0; e < 64; ++e) x[e] = 0.0f;

  const int nst = r0 < r1 ? (r1 - r0 + C::NR - 1) / C::NR : 0;
  if (nst > 0) stage32<CPLX, V, C::NR, C::THREADS / 32>(Ys, Y, ld, r0, r1, pc);
  cp_async_commit32();
  for (int st = 0; st < nst; ++st) {
    float* cur = Ys + (st & 1) * V * C::NR;
    if (st + 1 < nst)
      stage32<CPLX, V, C::NR, C::THREADS / 32>(Ys + ((st + 1) & 1) * V * C::NR, Y, ld, r0 + (st + 1) * C::NR, r1, pc);
    cp_async_commit32();
    cp_async_wait32_1();
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < C::CPL; ++cc) {
      const int chunk = chunk0 + 32 * C::R * cc;
      if (r0 + st * C::NR + 4 * chunk >= r1) break;
      float4 a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = *reinterpret_cast<const float4*>(&cur[(8 * bi + u) * C::NR + 4 * chunk]);
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const float4 bv = diag ? a[v] : *reinterpret_cast<const float4*>(&cur[(8 * bj + v) * C::NR + 4 * chunk]);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float& xe = x[8 * u + v];
          xe = fmaf(a[u].x, bv.x, xe);
          xe = fmaf(a[u].y, bv.y, xe);
          xe = fmaf(a[u].z, bv.z, xe);
          xe = fmaf(a[u].w, bv.w, xe);
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait32_0();

  // halving tree over the lanes: after the step with offset o, a lane keeps
  // the half of its entries selected by its bit o; entry e = 8u + v ends on
  // lane e / 2 (element e % 2)
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int o = 16 >> lvl, half = 32 >> lvl;
    const bool hi = lane & o;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = hi ? x[i] : x[i + half];
      const float keep = hi ? x[i + half] : x[i];
      x[i] = keep + __shfl_xor_sync(FULL, send, o);
    }
  }
  const int e0 = 2 * lane, u = e0 >> 3, v = e0 & 7;
  if constexpr (C::R > 1) {
    float* red = Ys;  // the stage buffers are no longer read
    __syncthreads();
    if (rg > 0) {
      red[((rg - 1) * C::NBT + blk) * 64 + e0] = x[0];
      red[((rg - 1) * C::NBT + blk) * 64 + e0 + 1] = x[1];
    }
    __syncthreads();
    if (rg == 0) {
#pragma unroll
      for (int g = 1; g < C::R; ++g) {
        x[0] += red[((g - 1) * C::NBT + blk) * 64 + e0];
        x[1] += red[((g - 1) * C::NBT + blk) * 64 + e0 + 1];
      }
    }
  }
  if (rg == 0) *reinterpret_cast<float2*>(&out[(8 * bi + u) * V + 8 * bj + v]) = make_float2(x[0], x[1]);
}

template <int V>
constexpr size_t gram32_smem() {
  return sizeof(float) * 2 * V * Gram32Cfg<V>::NR;
}

// FP32 bulk sweeps: [Y_p Y_q] <- [Y_p Y_q] Z-tilde on a tile of TRW rows;
// thread (row group rg, column group cg) computes rows 4 rg + [0, 4) and
// columns 8 cg + [0, 8) as sums over k in increasing order; the outputs go
// back through shared memory so that the global stores are coalesced.
template <int V>
struct Apply32Cfg {
  static constexpr int NCG = V / 8, NRG = 256 / NCG, TRW = 4 * NRG;
};

template <bool CPLX, int V>
__global__ void __launch_bounds__(256, 3) k_apply32(BlkDims d, BlkBuffers b, int step, int tile0, BlkBatch bt) {
  using C = Apply32Cfg<V>;
  __shared__ __align__(16) float Ys[V * C::TRW];  // column-major tile (real view)
  __shared__ __align__(16) float Ms[V * V];       // row-major Z-tilde (real view)
  int slot;
  if (!batch_item(bt, blockIdx.x, step, d, b, slot)) return;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  if (!b.flags[slot]) return;
  const int tf = (d.mf + C::TRW - 1) / C::TRW, tg = (d.mg + C::TRW - 1) / C::TRW;
  int tile = tile0 + blockIdx.y;
  if (tile >= tf + tg + (d.n + C::TRW - 1) / C::TRW) return;
  float* Y;
  long long ld;
  int m;
  if (tile < tf) {
    Y = static_cast<float*>(b.F); ld = b.ldf; m = d.mf;
  } else if (tile < tf + tg) {
    tile -= tf; Y = static_cast<float*>(b.G); ld = b.ldg; m = d.mg;
  } else {
    tile -= tf + tg; Y = static_cast<float*>(b.Z); ld = b.ldz; m = d.n;
  }
  const int rt = tile * C::TRW;
  stage32<CPLX, V, C::TRW, 8>(Ys, Y, ld, rt, m, pc);
  cp_async_commit32();
  const float* zt = static_cast<const float*>(b.ztil) + (size_t)slot * V * V;
  for (int idx = threadIdx.x; idx < V * V; idx += blockDim.x) Ms[idx] = zt[idx];
  cp_async_wait32_0();
  __syncthreads();
  const int rg = threadIdx.x % C::NRG, cg = threadIdx.x / C::NRG;
  float acc[4][8];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.0f;
#pragma unroll 8
  for (int k = 0; k < V; ++k) {
    const float4 y = *reinterpret_cast<const float4*>(&Ys[k * C::TRW + 4 * rg]);
    const float4 z0 = *reinterpret_cast<const float4*>(&Ms[k * V + 8 * cg]);
    const float4 z1 = *reinterpret_cast<const float4*>(&Ms[k * V + 8 * cg + 4]);
    const float yv[4] = {y.x, y.y, y.z, y.w}, zv[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(yv[u], zv[v], acc[u][v]);
  }
  __syncthreads();  // every thread is done reading the tile
#pragma unroll
  for (int v = 0; v < 8; ++v)
    *reinterpret_cast<float4*>(&Ys[(8 * cg + v) * C::TRW + 4 * rg]) =
        make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
  __syncthreads();
  // one column per warp at a time, 128 bytes (complex: 256) per store
  const int bb = pc.bb, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < bb; c += 8) {
    if constexpr (!CPLX) {
      float* col = Y + (size_t)pc.gcol(c) * ld + rt;
#pragma unroll
      for (int q = 0; q < C::TRW / 32; ++q) {
        const int r = lane + 32 * q;
        if (rt + r < m) col[r] = Ys[c * C::TRW + r];
      }
    } else {
      float2* col = reinterpret_cast<float2*>(Y) + (size_t)pc.gcol(c) * ld + rt;
#pragma unroll
      for (int q = 0; q < C::TRW / 32; ++q) {
        const int r = lane + 32 * q;
        if (rt + r < m) col[r] = make_float2(Ys[c * C::TRW + r], Ys[(bb + c) * C::TRW + r]);
      }
    }
  }
}

template <class T, int V>
size_t apply_smem() {
  return std::is_same<T, double>::value ? sizeof(double) * (V * (TR + 8) + V * (V + 8))
                                        : sizeof(float) * (TR * (V + 1) + V * V);
}
template <class Ti, bool CPLX, int V>
size_t inner_smem() {
  constexpr int E = CPLX ? 2 : 1;
  constexpr int BMAX = CPLX ? V / 2 : V;
  return sizeof(double) * 2 * E * BMAX * BMAX + sizeof(Ti) * E * BMAX * BMAX +
         sizeof(PivInT<Ti>) * (BMAX / 2 + 1) + sizeof(PivZ<Ti>) * (BMAX / 2 + 1) +
         sizeof(uint16_t) * (BMAX * (BMAX + 1) / 2) + 16;
}

template <class K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <class T, bool CPLX, int V>
cudaError_t gram_v(const BlkDims& d, const BlkBuffers& b, int step, cudaStream_t s, const BlkBatch* bt, int nitems,
                   int grid_y) {
  if constexpr (std::is_same<T, float>::value && V <= 32) {
    constexpr size_t smem32 = gram32_smem<V>();
    auto kern32 = k_gram32<CPLX, V>;
    cudaError_t e32 = set_smem(kern32, smem32);
    if (e32 != cudaSuccess) return e32;
    const BlkBatch one;
    dim3 grid(bt ? nitems : d.nslots, bt ? grid_y : d.rf + d.rg);
    kern32<<<grid, Gram32Cfg<V>::THREADS, smem32, s>>>(d, b, step, bt ? *bt : one);
    return cudaGetLastError();
  }
  const size_t smem = gram_smem<T, V>();
  auto kern = k_gram<T, CPLX, V>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const BlkBatch one;
  dim3 grid(bt ? nitems : d.nslots, bt ? grid_y : d.rf + d.rg);
  kern<<<grid, gram_threads<T, V>(), smem, s>>>(d, b, step, bt ? *bt : one);
  return cudaGetLastError();
}
template <class T, bool CPLX, int V>
cudaError_t apply_v(const BlkDims& d, const BlkBuffers& b, int step, cudaStream_t s, const BlkBatch* bt, int nitems,
                    int grid_y) {
  if constexpr (std::is_same<T, float>::value && V <= 32) {
    const BlkBatch one;
    auto kern32 = k_apply32<CPLX, V>;
    if (bt) {  // batched: grid y sized for 64-row tiles; the extra blocks leave at once
      kern32<<<dim3(nitems, grid_y), 256, 0, s>>>(d, b, step, 0, *bt);
      return cudaGetLastError();
    }
    constexpr int TRW = Apply32Cfg<V>::TRW;
    const int tiles = (d.mf + TRW - 1) / TRW + (d.mg + TRW - 1) / TRW + (d.n + TRW - 1) / TRW;
    for (int t0 = 0; t0 < tiles; t0 += 65535) {
      kern32<<<dim3(d.nslots, std::min(65535, tiles - t0)), 256, 0, s>>>(d, b, step, t0, one);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const size_t smem = apply_smem<T, V>();
  auto kern = k_apply<T, CPLX, V>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  if (bt) {  // batched: one launch, grid y = the largest problem's row tiles (the planner keeps it <= 65535)
    kern<<<dim3(nitems, grid_y), 256, smem, s>>>(d, b, step, 0, *bt);
    return cudaGetLastError();
  }
  const BlkBatch one;
  const int tiles = (d.mf + TR - 1) / TR + (d.mg + TR - 1) / TR + (d.n + TR - 1) / TR;
  // tiles of F, G, Z on grid y, in launches of at most 65535 tiles each
  for (int t0 = 0; t0 < tiles; t0 += 65535) {
    dim3 grid(d.nslots, std::min(65535, tiles - t0));
    kern<<<grid, 256, smem, s>>>(d, b, step, t0, one);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
// the two-CTA pivot step for the FP64 sweeps (GSVD_INNER_CLUSTER=0 selects
// the one-CTA kernel, for comparisons)
bool inner_cluster_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("GSVD_INNER_CLUSTER");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <class Ti, class To, bool CPLX, int V>
cudaError_t inner_v(const BlkDims& d, const BlkBuffers& b, int step, const InnerParams& p, cudaStream_t s,
                    const BlkBatch* bt, int nitems) {
  const BlkBatch one;
  const int nx = bt ? nitems : d.nslots;
  if constexpr (std::is_same<Ti, double>::value && V <= 32) {
    if (inner_cluster_enabled()) {
      const size_t smem2 = inner2_smem<CPLX, V>();
      auto kern2 = k_inner2<CPLX, V>;
      cudaError_t e2 = set_smem(kern2, smem2);
      if (e2 != cudaSuccess) return e2;
      kern2<<<2 * nx, INNER2_THREADS, smem2, s>>>(d, b, step, p, bt ? *bt : one);
      return cudaGetLastError();
    }
  }
  const size_t smem = inner_smem<Ti, CPLX, V>();
  constexpr bool can32 = std::is_same<Ti, float>::value;
  auto kern = (can32 && p.par32) ? k_inner<Ti, To, CPLX, V, can32> : k_inner<Ti, To, CPLX, V, false>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<nx, INNER_THREADS, smem, s>>>(d, b, step, p, bt ? *bt : one);
  return cudaGetLastError();
}

}  // namespace

bool inner_variants_supported(int V) { return V <= 32 && inner_cluster_enabled(); }

int blk_vmax(int w, bool cplx) {
  const int v = cplx ? 4 * w : 2 * w;
  if (v <= 16) return 16;
  if (v <= 32) return 32;
  if (v <= 64) return 64;
  return 0;  // unsupported
}

#define HZ_DISPATCH_V(V, CALL)            \
  switch (V) {                            \
    case 16: { constexpr int VV = 16; return CALL; } \
    case 32: { constexpr int VV = 32; return CALL; } \
    case 64: { constexpr int VV = 64; return CALL; } \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_gram(const BlkDims& d, const BlkBuffers& b, bool cplx, bool fp32, int step, cudaStream_t s,
                        const BlkBatch* bt, int nitems, int grid_y) {
  const int V = blk_vmax(d.w, cplx);
  if (cplx) {
    if (fp32) { HZ_DISPATCH_V(V, (gram_v<float, true, VV>(d, b, step, s, bt, nitems, grid_y))); }
    else { HZ_DISPATCH_V(V, (gram_v<double, true, VV>(d, b, step, s, bt, nitems, grid_y))); }
  } else {
    if (fp32) { HZ_DISPATCH_V(V, (gram_v<float, false, VV>(d, b, step, s, bt, nitems, grid_y))); }
    else { HZ_DISPATCH_V(V, (gram_v<double, false, VV>(d, b, step, s, bt, nitems, grid_y))); }
  }
}

cudaError_t launch_apply(const BlkDims& d, const BlkBuffers& b, bool cplx, bool fp32, int step, cudaStream_t s,
                         const BlkBatch* bt, int nitems, int grid_y) {
  const int V = blk_vmax(d.w, cplx);
  if (cplx) {
    if (fp32) { HZ_DISPATCH_V(V, (apply_v<float, true, VV>(d, b, step, s, bt, nitems, grid_y))); }
    else { HZ_DISPATCH_V(V, (apply_v<double, true, VV>(d, b, step, s, bt, nitems, grid_y))); }
  } else {
    if (fp32) { HZ_DISPATCH_V(V, (apply_v<float, false, VV>(d, b, step, s, bt, nitems, grid_y))); }
    else { HZ_DISPATCH_V(V, (apply_v<double, false, VV>(d, b, step, s, bt, nitems, grid_y))); }
  }
}


cudaError_t launch_inner(const BlkDims& d, const BlkBuffers& b, bool cplx, bool fp32, int step,
                         const InnerParams& p, cudaStream_t s, const BlkBatch* bt, int nitems) {
  const int V = blk_vmax(d.w, cplx);
  if (cplx) {
    if (fp32) { HZ_DISPATCH_V(V, (inner_v<float, float, true, VV>(d, b, step, p, s, bt, nitems))); }
    else { HZ_DISPATCH_V(V, (inner_v<double, double, true, VV>(d, b, step, p, s, bt, nitems))); }
  } else {
    if (fp32) { HZ_DISPATCH_V(V, (inner_v<float, float, false, VV>(d, b, step, p, s, bt, nitems))); }
    else { HZ_DISPATCH_V(V, (inner_v<double, double, false, VV>(d, b, step, p, s, bt, nitems))); }
  }
}

}  // namespace hz
