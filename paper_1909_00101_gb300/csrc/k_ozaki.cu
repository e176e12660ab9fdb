// k_ozaki.cu -- the FP64 pivot Grams and block applies of the blocked sweeps
// (Sec. 2.3-2.5 of arXiv 1909.00101) on the BF16 tensor cores, with FP64
// accuracy: an error-free splitting of the FP64 operands into 8-bit integer
// slices (Ozaki, Ogita, Oishi and Rump's splitting for matrix products, in a
// fixed-point form), products of slices on mma.sync BF16 with exact FP32
// accumulation, and an exact integer recombination rounded once to FP64.
//
// Why: on sm_103a the FP64 pipe delivers about 1 TFLOP/s (DFMA and DMMA
// alike) while mma.sync with BF16 inputs delivers about 600 TFLOP/s.
//
// The arithmetic, per contraction sum_k x_k y_k:
//   * every x in a set that shares a scale (a column of the Gram slab, a
//     column of the Y tile, a column of Z-tilde) is written exactly as
//     x = s 2^e sum_{a=1..7} c_a 2^(-8a) + r, with 2^e above the set's
//     largest |x|, digits c_a in [0, 255], s the sign of x, |r| < 2^(e-56);
//     s c_a is an integer that BF16 holds exactly;
//   * a product of two such expansions is sum_{a,b} 2^(-8(a+b)) (s c_a)(s' c_b);
//     the terms with a + b <= 8 are kept (the rest weigh below 2^-56 of the
//     scales' product); for each level L = a + b the slice products are summed
//     by the tensor cores in FP32, exactly, because a level of at most 7
//     products over at most 32 terms stays below 2^24;
//   * the levels are combined exactly in 128-bit integers,
//     T = sum_L A_L 2^(8(8-L)), and T 2^(e + e' - 64) is rounded once to the
//     nearest FP64 value (ties to even).
// The error of an entry is below about 2^-53 times (number of terms) times
// the product of the two scales: the size of an FP64 dot product's own error
// bound, column by column, which is what the one-sided method's accuracy
// rests on.  Longer sums (the Gram over a row slab) flush the FP32 level sums
// every 32 rows into exact FP32 double-word accumulators (TwoSum), which stay
// exact integers below 2^48.
//
// Scales: the Gram uses one scale per slab column; the apply Y Z scales Y by
// column (D^-1), Z-tilde by row (D) and then by column, so every Y column
// keeps its own relative accuracy.
#include <cstdint>
#include <type_traits>

#include "blk_pair.cuh"
#include "hz_device.cuh"
#include "hz_kernels.h"

namespace hz {

namespace {

constexpr int NSL = 7;  // slices (56 bits)
constexpr int NLV = 7;  // levels L = 2..8
constexpr int OZ_CHUNK = 32;  // Gram rows per FP32 level sum

__device__ __forceinline__ int exp_field(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return e ? e : 1;
}

// The seven signed 8-bit digits of x relative to the scale whose exponent
// field is emax (|x| < 2^(emax - 1022)), as BF16 bit patterns; eadd is added
// to x's exponent first (x 2^eadd is sliced; x != 0 assumed normal).
__device__ __forceinline__ void slice7(double x, int emax, int eadd, uint16_t out[NSL]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int sh = (e ? e + eadd : 1 + eadd) - emax + 3;
  unsigned long long X = 0;
  if (m != 0) {
    if (sh >= 0)
      X = m << sh;  // sh <= 3: X < 2^56
    else if (sh > -64)
      X = m >> (-sh);
  }
  const uint16_t sgn = (bits >> 63) ? 0x8000u : 0u;
#pragma unroll
  for (int a = 0; a < NSL; ++a) {
    const unsigned c = (unsigned)(X >> (48 - 8 * a)) & 255u;
    // an integer below 256 has at most 8 significant bits: its FP32 pattern's
    // low 16 bits are zero and the high half is its BF16 pattern
    out[a] = c ? (uint16_t)((__float_as_uint((float)c) >> 16) | sgn) : (uint16_t)0;
  }
}

// T 2^e2 rounded to the nearest FP64 value (ties to even); T 2^e2 is assumed
// to be 0 or in the normal range.
__device__ __forceinline__ double i128_to_double(__int128 T, int e2) {
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  unsigned __int128 U = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const unsigned long long h = (unsigned long long)(U >> 64), l = (unsigned long long)U;
  const int lz = h ? __clzll((long long)h) : 64 + __clzll((long long)l);
  U <<= lz;
  const unsigned long long top = (unsigned long long)(U >> 64), rest = (unsigned long long)U;
  unsigned long long m = top >> 11;
  const unsigned long long r = top & 0x7FFull;
  const bool up = r > 0x400ull || (r == 0x400ull && (rest != 0 || (m & 1ull)));
  m += up ? 1ull : 0ull;
  int ex = 127 - lz + e2;
  if (m >> 53) {
    m >>= 1;
    ++ex;
  }
  const unsigned long long out = (neg ? (1ull << 63) : 0ull) | ((unsigned long long)(ex + 1023) << 52) |
                                 (m & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)out);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// level products of one k-step: acc[L - 2] += A_a B_b for a + b = L <= 8
__device__ __forceinline__ void level_mmas(float acc[NLV][4], const uint32_t A[NSL][4], const uint32_t B[NSL][2]) {
#pragma unroll
  for (int a = 0; a < NSL; ++a)
#pragma unroll
    for (int b = 0; b < NSL; ++b)
      if (a + b + 2 <= 8) mma_bf16(acc[a + b], A[a], B[b]);
}

// ---------------------------------------------------------------- Gram ----
// One warp per upper m16 x n8 tile of the V x V Gram of the slab: V = 16 has
// 2 such tiles, V = 32 has 6.
template <int V>
__host__ __device__ constexpr int oz_gram_warps() {
  return V == 16 ? 2 : 6;
}
template <int V>
__device__ __forceinline__ void oz_gram_tile(int w, int& mt, int& nt) {
  if constexpr (V == 16) {
    mt = 0;
    nt = w;
  } else {
    // m-tile 0: n-tiles 0..3; m-tile 1: n-tiles 2, 3
    mt = w < 4 ? 0 : 1;
    nt = w < 4 ? w : w - 2;
  }
}

constexpr int GRS = OZ_CHUNK + 8;  // padded row stride of a slice column (bf16)

template <int V, bool CPLX>
__global__ void __launch_bounds__(32 * oz_gram_warps<V>()) k_gram_oz(BlkDims d, BlkBuffers b, int step) {
  constexpr int NW = oz_gram_warps<V>();
  constexpr int NT = 32 * NW;
  __shared__ __align__(16) uint16_t Ss[NSL][V][GRS];
  __shared__ int s_emax[V];
  const int slot = blockIdx.x, s = blockIdx.y;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  const bool isF = s < d.rf;
  const int m = isF ? d.mf : d.mg;
  const int nsplit = isF ? d.rf : d.rg;
  const int si = isF ? s : s - d.rf;
  const int tiles = (m + 63) / 64;
  const int per = (tiles + nsplit - 1) / nsplit * 64;
  const int r0 = si * per, r1 = min(m, r0 + per);
  const double* Y = static_cast<const double*>(isF ? b.F : b.G);
  const long long ld = isF ? b.ldf : b.ldg;
  double* out = static_cast<double*>(b.partial) + ((size_t)slot * (d.rf + d.rg) + s) * V * V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bb = pc.bb;
  constexpr int E = CPLX ? 2 : 1;

  // 1. exponent field of each real-view column's largest |x| over the slab
  for (int c = threadIdx.x; c < V; c += NT) s_emax[c] = 1;
  __syncthreads();
  for (int c = warp; c < bb; c += NW) {  // stored columns (complex: Re and Im)
    const double* col = Y + (size_t)pc.gcol(c) * E * ld;
    int mr = 1, mi = 1;
    for (int r = r0 + lane; r < r1; r += 32) {
      if constexpr (CPLX) {
        mr = max(mr, exp_field(col[2 * r]));
        mi = max(mi, exp_field(col[2 * r + 1]));
      } else {
        mr = max(mr, exp_field(col[r]));
      }
    }
    mr = __reduce_max_sync(FULL, mr);
    if constexpr (CPLX) mi = __reduce_max_sync(FULL, mi);
    if (lane == 0) {
      s_emax[c] = mr;
      if constexpr (CPLX) s_emax[bb + c] = mi;
    }
  }
  __syncthreads();

  int mt, nt;
  oz_gram_tile<V>(warp, mt, nt);
  const int g = lane >> 2, t = lane & 3;
  float hi[NLV][4], lo[NLV][4];
#pragma unroll
  for (int L = 0; L < NLV; ++L)
#pragma unroll
    for (int q = 0; q < 4; ++q) hi[L][q] = lo[L][q] = 0.0f;

  // 2. chunks of 32 rows: slices of the real view into shared memory, then
  //    the level products of this warp's tile, then the exact flush
  for (int c0 = r0; c0 < r1; c0 += OZ_CHUNK) {
    // row pairs (r, r + 1) of real-view column c; 16 pairs per column
    for (int it = threadIdx.x; it < (V / E) * (OZ_CHUNK / 2); it += NT) {
      const int c = it / (OZ_CHUNK / 2), rp = 2 * (it % (OZ_CHUNK / 2));
      uint16_t s0[NSL], s1[NSL];
      if constexpr (!CPLX) {
        double x0 = 0.0, x1 = 0.0;
        if (c < bb) {
          const double* col = Y + (size_t)pc.gcol(c) * ld;
          if (c0 + rp < r1) x0 = col[c0 + rp];
          if (c0 + rp + 1 < r1) x1 = col[c0 + rp + 1];
        }
        const int em = s_emax[c];
        slice7(x0, em, 0, s0);
        slice7(x1, em, 0, s1);
#pragma unroll
        for (int a = 0; a < NSL; ++a)
          *reinterpret_cast<uint32_t*>(&Ss[a][c][rp]) = (uint32_t)s0[a] | ((uint32_t)s1[a] << 16);
      } else {
        // complex column c (< bb) gives real-view columns c (Re) and bb + c
        // (Im); for c >= bb the zero columns 2c and 2c + 1 (they cover the
        // padding [2 bb, V))
        double2 v0 = make_double2(0.0, 0.0), v1 = make_double2(0.0, 0.0);
        if (c < bb) {
          const double2* col = reinterpret_cast<const double2*>(Y) + (size_t)pc.gcol(c) * ld;
          if (c0 + rp < r1) v0 = col[c0 + rp];
          if (c0 + rp + 1 < r1) v1 = col[c0 + rp + 1];
        }
        const int cr = c < bb ? c : 2 * c, ci = c < bb ? bb + c : 2 * c + 1;
        const int er = s_emax[cr], ei = s_emax[ci];
        slice7(v0.x, er, 0, s0);
        slice7(v1.x, er, 0, s1);
#pragma unroll
        for (int a = 0; a < NSL; ++a)
          *reinterpret_cast<uint32_t*>(&Ss[a][cr][rp]) = (uint32_t)s0[a] | ((uint32_t)s1[a] << 16);
        slice7(v0.y, ei, 0, s0);
        slice7(v1.y, ei, 0, s1);
#pragma unroll
        for (int a = 0; a < NSL; ++a)
          *reinterpret_cast<uint32_t*>(&Ss[a][ci][rp]) = (uint32_t)s0[a] | ((uint32_t)s1[a] << 16);
      }
    }
    __syncthreads();
    float acc[NLV][4];
#pragma unroll
    for (int L = 0; L < NLV; ++L)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[L][q] = 0.0f;
#pragma unroll
    for (int kb = 0; kb < OZ_CHUNK; kb += 16) {
      // A = S_a^T (rows: columns 16 mt + ...; k: rows of the chunk), B = S_b
      uint32_t A[NSL][4], B[NSL][2];
#pragma unroll
      for (int a = 0; a < NSL; ++a) {
        A[a][0] = ld32(&Ss[a][16 * mt + g][kb + 2 * t]);
        A[a][1] = ld32(&Ss[a][16 * mt + g + 8][kb + 2 * t]);
        A[a][2] = ld32(&Ss[a][16 * mt + g][kb + 2 * t + 8]);
        A[a][3] = ld32(&Ss[a][16 * mt + g + 8][kb + 2 * t + 8]);
        B[a][0] = ld32(&Ss[a][8 * nt + g][kb + 2 * t]);
        B[a][1] = ld32(&Ss[a][8 * nt + g][kb + 2 * t + 8]);
      }
      level_mmas(acc, A, B);
    }
    // exact flush: (hi, lo) += acc by TwoSum (all values are integers)
#pragma unroll
    for (int L = 0; L < NLV; ++L)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float x = acc[L][q], h = hi[L][q];
        const float sum = h + x;
        const float bv = sum - h;
        const float err = (h - (sum - bv)) + (x - bv);
        hi[L][q] = sum;
        lo[L][q] += err;
      }
    __syncthreads();
  }

  // 3. entries of this warp's tile: exact level combination, one rounding
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 16 * mt + g + ((q & 2) ? 8 : 0);
    const int j = 8 * nt + 2 * t + (q & 1);
    __int128 T = 0;
#pragma unroll
    for (int L = 0; L < NLV; ++L) {
      const long long x = __float2ll_rn(hi[L][q]) + __float2ll_rn(lo[L][q]);
      T += (__int128)x << (8 * (NLV - 1 - L));
    }
    const int e2 = (s_emax[i] - 1022) + (s_emax[j] - 1022) - 64;
    out[i * V + j] = i128_to_double(T, e2);
  }
}

// --------------------------------------------------------------- apply ----
// [Y_p Y_q] <- [Y_p Y_q] Z-tilde on a tile of 64 rows (real view, V <= 32):
// eight warps, warp w owns rows 16 (w & 3) + [0, 16) and V / 16 of the V / 8
// column tiles.
constexpr int ATR = 64;

template <int V, bool CPLX>
__global__ void __launch_bounds__(256) k_apply_oz(BlkDims d, BlkBuffers b, int step) {
  constexpr int YS = V + 8;  // padded row stride of the Y slices (bf16)
  constexpr int TS = V + 8;  // padded stride of a Z slice column (bf16)
  constexpr int NNW = V / 16;  // column tiles (n8) per warp
  constexpr int PER = V * ATR / 256;  // real-view values per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint16_t* Ys = reinterpret_cast<uint16_t*>(smem_raw);  // [NSL][ATR][YS]
  uint16_t* Ts = Ys + NSL * ATR * YS;                    // [NSL][V][TS]
  double* Zd = reinterpret_cast<double*>(Ts + NSL * V * TS);  // [V][V], row k = Z-tilde row
  __shared__ int s_ey[V], s_fz[V];

  const int slot = blockIdx.x;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  if (!b.flags[slot]) return;
  const int tf = (d.mf + ATR - 1) / ATR, tg = (d.mg + ATR - 1) / ATR;
  int tile = blockIdx.y;
  double* Y;
  long long ld;
  int m;
  if (tile < tf) {
    Y = static_cast<double*>(b.F); ld = b.ldf; m = d.mf;
  } else if (tile < tf + tg) {
    tile -= tf; Y = static_cast<double*>(b.G); ld = b.ldg; m = d.mg;
  } else {
    tile -= tf + tg; Y = static_cast<double*>(b.Z); ld = b.ldz; m = d.n;
  }
  const int r0 = tile * ATR;
  const int bb = pc.bb;
  const double* zt = static_cast<const double*>(b.ztil) + (size_t)slot * V * V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // 1. Z-tilde into shared memory; the tile's real view into registers:
  //    value i of thread x is row (x + 256 i) % 64 of real-view column
  //    (x + 256 i) / 64 (complex: complex column (x + 256 i) / 64 gives the
  //    values i (Re) and PER / 2 + i (Im))
  for (int idx = threadIdx.x; idx < V * V; idx += 256) Zd[idx] = zt[idx];
  if (threadIdx.x < V) s_ey[threadIdx.x] = 1;
  double y[PER];
  const int rr = threadIdx.x & (ATR - 1);
  if constexpr (!CPLX) {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int c = (threadIdx.x + 256 * i) / ATR;
      y[i] = (c < bb && r0 + rr < m) ? Y[(size_t)pc.gcol(c) * ld + r0 + rr] : 0.0;
    }
  } else {
#pragma unroll
    for (int i = 0; i < PER / 2; ++i) {
      const int c = (threadIdx.x + 256 * i) / ATR;
      double2 v = make_double2(0.0, 0.0);
      if (c < bb && r0 + rr < m) v = reinterpret_cast<const double2*>(Y)[(size_t)pc.gcol(c) * ld + r0 + rr];
      y[i] = v.x;
      y[PER / 2 + i] = v.y;
    }
  }
  __syncthreads();
  // real-view column of value i
  auto vcol = [&](int i) -> int {
    if constexpr (!CPLX) {
      return (threadIdx.x + 256 * i) / ATR;
    } else {
      const int ii = i < PER / 2 ? i : i - PER / 2;
      const int c = (threadIdx.x + 256 * ii) / ATR;
      if (i < PER / 2) return c < bb ? c : 2 * c;
      return c < bb ? bb + c : 2 * c + 1;
    }
  };
  // 2. column exponents of the tile (two warps share a column: 64 rows)
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int mx = __reduce_max_sync(FULL, exp_field(y[i]));
    if (lane == 0) atomicMax(&s_ey[vcol(i)], mx);
  }
  __syncthreads();
  // 3. Z' = D Z-tilde (row k scaled by 2^(e_k)), its column exponents, slices
  for (int j = warp; j < V; j += 8) {
    int mx = 1;
    for (int k = lane; k < V; k += 32) {
      const double z = Zd[k * V + j];
      if (z != 0.0) mx = max(mx, exp_field(z) + s_ey[k] - 1022);
    }
    mx = __reduce_max_sync(FULL, mx);
    if (lane == 0) s_fz[j] = mx;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < V * V; idx += 256) {
    const int k = idx / V, j = idx % V;
    uint16_t sl[NSL];
    slice7(Zd[idx], s_fz[j], s_ey[k] - 1022, sl);
#pragma unroll
    for (int a = 0; a < NSL; ++a) Ts[(a * V + j) * TS + k] = sl[a];
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int c = vcol(i);
    uint16_t sl[NSL];
    slice7(y[i], s_ey[c], 0, sl);
#pragma unroll
    for (int a = 0; a < NSL; ++a) Ys[(a * ATR + rr) * YS + c] = sl[a];
  }
  __syncthreads();

  // 4. level products: warp w, rows 16 mt + [0, 16), column tiles nt0 + [0, NNW)
  const int mt = warp & 3, nt0 = (warp >> 2) * NNW;
  const int g = lane >> 2, t = lane & 3;
  float acc[NNW][NLV][4];
#pragma unroll
  for (int u = 0; u < NNW; ++u)
#pragma unroll
    for (int L = 0; L < NLV; ++L)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[u][L][q] = 0.0f;
#pragma unroll
  for (int kb = 0; kb < V; kb += 16) {
    uint32_t A[NSL][4];
#pragma unroll
    for (int a = 0; a < NSL; ++a) {
      const uint16_t* base = Ys + (a * ATR + 16 * mt) * YS;
      A[a][0] = ld32(base + g * YS + kb + 2 * t);
      A[a][1] = ld32(base + (g + 8) * YS + kb + 2 * t);
      A[a][2] = ld32(base + g * YS + kb + 2 * t + 8);
      A[a][3] = ld32(base + (g + 8) * YS + kb + 2 * t + 8);
    }
#pragma unroll
    for (int u = 0; u < NNW; ++u) {
      uint32_t B[NSL][2];
#pragma unroll
      for (int a = 0; a < NSL; ++a) {
        const uint16_t* base = Ts + (a * V + 8 * (nt0 + u) + g) * TS;
        B[a][0] = ld32(base + kb + 2 * t);
        B[a][1] = ld32(base + kb + 2 * t + 8);
      }
      level_mmas(acc[u], A, B);
    }
  }
  __syncthreads();  // the slices are no longer read: reuse as the output tile

  // 5. exact level combination, one rounding, staged column-major
  constexpr int OS = ATR + 1;
  double* Ob = reinterpret_cast<double*>(smem_raw);  // [V][OS]
#pragma unroll
  for (int u = 0; u < NNW; ++u)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = 16 * mt + g + ((q & 2) ? 8 : 0);
      const int j = 8 * (nt0 + u) + 2 * t + (q & 1);
      __int128 T = 0;
#pragma unroll
      for (int L = 0; L < NLV; ++L) T += (__int128)__float2int_rn(acc[u][L][q]) << (8 * (NLV - 1 - L));
      Ob[j * OS + r] = i128_to_double(T, s_fz[j] - 1022 - 64);
    }
  __syncthreads();
  if constexpr (!CPLX) {
    for (int idx = threadIdx.x; idx < bb * ATR; idx += 256) {
      const int c = idx / ATR, r = idx % ATR;
      if (r0 + r < m) Y[(size_t)pc.gcol(c) * ld + r0 + r] = Ob[c * OS + r];
    }
  } else {
    double2* Y2 = reinterpret_cast<double2*>(Y);
    for (int idx = threadIdx.x; idx < bb * ATR; idx += 256) {
      const int c = idx / ATR, r = idx % ATR;
      if (r0 + r < m) Y2[(size_t)pc.gcol(c) * ld + r0 + r] = make_double2(Ob[c * OS + r], Ob[(bb + c) * OS + r]);
    }
  }
}

template <int V>
size_t apply_oz_smem() {
  const size_t slices = sizeof(uint16_t) * NSL * ((size_t)ATR * (V + 8) + (size_t)V * (V + 8));
  const size_t out = sizeof(double) * V * (ATR + 1);
  return (slices > out ? slices : out) + sizeof(double) * V * V + 16;
}

}  // namespace

bool oz_supported(int V) { return V == 16 || V == 32; }

cudaError_t launch_gram_oz(const BlkDims& d, const BlkBuffers& b, bool cplx, int step, cudaStream_t s) {
  const int V = blk_vmax(d.w, cplx);
  dim3 grid(d.nslots, d.rf + d.rg);
  if (V == 16) {
    if (cplx) k_gram_oz<16, true><<<grid, 32 * oz_gram_warps<16>(), 0, s>>>(d, b, step);
    else k_gram_oz<16, false><<<grid, 32 * oz_gram_warps<16>(), 0, s>>>(d, b, step);
  } else if (V == 32) {
    if (cplx) k_gram_oz<32, true><<<grid, 32 * oz_gram_warps<32>(), 0, s>>>(d, b, step);
    else k_gram_oz<32, false><<<grid, 32 * oz_gram_warps<32>(), 0, s>>>(d, b, step);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int V, bool CPLX>
static cudaError_t apply_oz_v(const BlkDims& d, const BlkBuffers& b, int step, cudaStream_t s) {
  const size_t smem = apply_oz_smem<V>();
  auto kern = k_apply_oz<V, CPLX>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int tiles = (d.mf + ATR - 1) / ATR + (d.mg + ATR - 1) / ATR + (d.n + ATR - 1) / ATR;
  dim3 grid(d.nslots, tiles);
  kern<<<grid, 256, smem, s>>>(d, b, step);
  return cudaGetLastError();
}

cudaError_t launch_apply_oz(const BlkDims& d, const BlkBuffers& b, bool cplx, int step, cudaStream_t s) {
  const int V = blk_vmax(d.w, cplx);
  if (V == 16) return cplx ? apply_oz_v<16, true>(d, b, step, s) : apply_oz_v<16, false>(d, b, step, s);
  if (V == 32) return cplx ? apply_oz_v<32, true>(d, b, step, s) : apply_oz_v<32, false>(d, b, step, s);
  return cudaErrorInvalidValue;
}

}  // namespace hz
