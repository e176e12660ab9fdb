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
//     x = s 2^e sum_{a=1..8} c_a 2^(-8a) + r, with 2^e above the set's
//     largest |x|, digits c_a in [0, 255], s the sign of x, |r| < 2^(e-64);
//     s c_a is an integer that BF16 holds exactly.  Eight digits (64 bits)
//     keep the full 53-bit significand of every entry within 2^-11 of its
//     set's largest, so graded data (the rows of a triangular QR factor, a
//     spread of column norms inside a tile) keep the accuracy of an FP64
//     product;
//   * a product of two such expansions is sum_{a,b} 2^(-8(a+b)) (s c_a)(s' c_b);
//     the terms with a + b <= 9 are kept (the rest weigh below 2^-64 of the
//     scales' product); for each level L = a + b the slice products are summed
//     by the tensor cores in FP32, exactly, because a level of at most 8
//     products over at most 32 terms stays below 2^24 (8 * 32 * 255^2 < 2^24);
//   * the levels are combined exactly in 128-bit integers,
//     T = sum_L A_L 2^(8(9-L)), and T 2^(e + e' - 72) is rounded once to the
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
#include <cstdlib>
#include <type_traits>

#include "blk_pair.cuh"
#include "hz_device.cuh"
#include "hz_kernels.h"

namespace hz {

namespace {

constexpr int NSL = 8;  // slices (64 bits)
constexpr int NLV = 8;  // levels L = 2..9
constexpr int OZ_EOFF = 72;  // 2^-72: the weight of level L = 2 relative to the two scales
constexpr int OZ_CHUNK = 32;  // Gram rows per FP32 level sum

__device__ __forceinline__ int exp_field(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return e ? e : 1;
}

// The 64-bit fixed-point magnitude X of x relative to the scale whose
// exponent field is emax (|x| < 2^(emax - 1022), X = |x| 2^(1086 - emax),
// truncated); eadd is added to x's exponent first (x 2^eadd is taken).
__device__ __forceinline__ unsigned long long fixed64(double x, int emax, int eadd) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int sh = (e ? e + eadd : 1 + eadd) - emax + 11;
  if (sh >= 0) return m << sh;  // sh <= 11: X < 2^64
  return sh > -64 ? (m >> (-sh)) : 0ull;
}

// BF16 pattern of the integer c in [0, 255], with the sign bit sgn: the FP32
// value 2^23 + c minus 2^23 is exactly c, and an integer below 256 has at
// most 8 significant bits, so its FP32 pattern's high half is its BF16
// pattern (c = 0 gives a signed zero, which adds nothing).
__device__ __forceinline__ uint32_t bf16_digit(uint32_t c, uint32_t sgn) {
  const float f = __uint_as_float(0x4B000000u | c) - 8388608.0f;
  return (__float_as_uint(f) >> 16) | sgn;
}

// The eight signed 8-bit digits of x (most significant first) as BF16
// patterns in the low halves of out[]: x = s 2^e sum_a c_a 2^(-8(a+1)) + r.
__device__ __forceinline__ void slice8(double x, int emax, int eadd, uint32_t out[NSL]) {
  const unsigned long long X = fixed64(x, emax, eadd);
  const uint32_t sgn = (uint32_t)((unsigned long long)__double_as_longlong(x) >> 63) << 15;
  const uint32_t h = (uint32_t)(X >> 32), l = (uint32_t)X;
  out[0] = bf16_digit(h >> 24, sgn);
  out[1] = bf16_digit((h >> 16) & 255u, sgn);
  out[2] = bf16_digit((h >> 8) & 255u, sgn);
  out[3] = bf16_digit(h & 255u, sgn);
  out[4] = bf16_digit(l >> 24, sgn);
  out[5] = bf16_digit((l >> 16) & 255u, sgn);
  out[6] = bf16_digit((l >> 8) & 255u, sgn);
  out[7] = bf16_digit(l & 255u, sgn);
}

// An integer-valued FP32 value as a 64-bit integer, with integer operations
// (the FP32 -> 64-bit conversion instruction would use the FP64 pipe).
__device__ __forceinline__ long long float_int_to_ll(float f) {
  const uint32_t b = __float_as_uint(f);
  const int e = (int)((b >> 23) & 255u);
  if (e < 127) return 0;  // |f| < 1: an integer-valued f is 0
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const long long v = e >= 150 ? (m << (e - 150)) : (m >> (150 - e));
  return (b >> 31) ? -v : v;
}

// sum_i x_i 2^(8(7 - i)) 2^e2 rounded to the nearest FP64 value (ties to
// even), with integer operations only.  The sum is formed exactly as
// H 2^32 + L (H signed 64-bit, L unsigned 32-bit); |x_i| < 2^36 is assumed
// (level sums over at most OZ_K_MAX rows are below 8 * 2^16 * 255^2 < 2^35).
// (hi 2^32 + lo) 2^e2: the same, from hi = sum_{i<4} x_i 2^(8(3 - i)) and
// lo = sum_{i>=4} x_i 2^(8(7 - i))
__device__ __forceinline__ double levels_to_double_hl(long long hi, long long lo, int e2) {
  long long H = hi + (lo >> 32);
  uint32_t L = (uint32_t)lo;
  if (H == 0 && L == 0) return 0.0;
  const bool neg = H < 0;
  if (neg) {
    H = -H - (L != 0 ? 1 : 0);
    L = 0u - L;
  }
  unsigned long long W;
  bool sticky;
  int top;
  if (H != 0) {
    const int lz = __clzll(H);
    const unsigned long long Lw = (unsigned long long)L << 32;
    W = ((unsigned long long)H << lz) | (lz ? (Lw >> (64 - lz)) : 0ull);
    sticky = (Lw << lz) != 0ull;
    top = 95 - lz;
  } else {
    const int lz = __clzll((long long)(unsigned long long)L);
    W = (unsigned long long)L << lz;
    sticky = false;
    top = 63 - lz;
  }
  unsigned long long m = W >> 11;
  const uint32_t r = (uint32_t)W & 0x7FFu;
  m += (r > 0x400u || (r == 0x400u && (sticky || (m & 1ull)))) ? 1ull : 0ull;
  int ex = top + e2;
  if (m >> 53) {
    m >>= 1;
    ++ex;
  }
  // outside the normal range: below it the value is flushed to a signed
  // zero (an entry below 2^-1022 is far under the product's error bound);
  // above it, a signed infinity
  const unsigned long long sign = neg ? (1ull << 63) : 0ull;
  if (ex + 1023 <= 0) return __longlong_as_double((long long)sign);
  if (ex + 1023 >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ double levels_to_double(const long long x[NLV], int e2) {
  const long long hi = (x[0] << 24) + (x[1] << 16) + (x[2] << 8) + x[3];
  const long long lo = (x[4] << 24) + (x[5] << 16) + (x[6] << 8) + x[7];
  return levels_to_double_hl(hi, lo, e2);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// level products of one k-step with the A fragments loaded slice by slice
// (fewer live registers): acc[a + b] += A_a B_b for a + b + 2 <= 9
template <class LoadA>
__device__ __forceinline__ void level_mmas_stream(float acc[NLV][4], LoadA load_a, const uint32_t B[NSL][2]) {
#pragma unroll
  for (int a = 0; a < NSL; ++a) {
    uint32_t A[4];
    load_a(a, A);
#pragma unroll
    for (int b = 0; b < NSL; ++b)
      if (a + b + 2 <= NSL + 1) mma_bf16(acc[a + b], A, B[b]);
  }
}

// level products of one k-step: acc[L - 2] += A_a B_b for a + b = L <= 9
__device__ __forceinline__ void level_mmas(float acc[NLV][4], const uint32_t A[NSL][4], const uint32_t B[NSL][2]) {
#pragma unroll
  for (int a = 0; a < NSL; ++a)
#pragma unroll
    for (int b = 0; b < NSL; ++b)
      if (a + b + 2 <= NSL + 1) mma_bf16(acc[a + b], A[a], B[b]);
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
__global__ void __launch_bounds__(32 * oz_gram_warps<V>()) k_gram_oz(BlkDims d, BlkBuffers b, int step,
                                                                        BlkBatch bt) {
  constexpr int NW = oz_gram_warps<V>();
  constexpr int NT = 32 * NW;
  __shared__ __align__(16) uint16_t Ss[NSL][V][GRS];
  __shared__ int s_emax[V];
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
  //    the level products of this warp's tile, then the exact flush.  Item
  //    it is the row pair (r, r + 1) of (real-view, or complex) column
  //    it / 16; the next chunk's values are loaded while this one is used.
  constexpr int ITEMS = (V / E) * (OZ_CHUNK / 2);
  constexpr int PERT = (ITEMS + NT - 1) / NT;
  double pre[PERT][2 * E];
  auto fetch = [&](int c0) {
#pragma unroll
    for (int u = 0; u < PERT; ++u) {
      const int it = threadIdx.x + NT * u;
      const int c = it / (OZ_CHUNK / 2), rp = 2 * (it % (OZ_CHUNK / 2));
#pragma unroll
      for (int q = 0; q < 2 * E; ++q) pre[u][q] = 0.0;
      if (it < ITEMS && c < bb) {
        const double* col = Y + (size_t)pc.gcol(c) * E * ld;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (c0 + rp + h < r1) {
            if constexpr (CPLX) {
              const double2 v = reinterpret_cast<const double2*>(col)[c0 + rp + h];
              pre[u][h] = v.x;
              pre[u][2 + h] = v.y;
            } else {
              pre[u][h] = col[c0 + rp + h];
            }
          }
      }
    }
  };
  if (r0 < r1) fetch(r0);
  for (int c0 = r0; c0 < r1; c0 += OZ_CHUNK) {
#pragma unroll
    for (int u = 0; u < PERT; ++u) {
      const int it = threadIdx.x + NT * u;
      if (it >= ITEMS) continue;
      const int c = it / (OZ_CHUNK / 2), rp = 2 * (it % (OZ_CHUNK / 2));
#pragma unroll
      for (int part = 0; part < E; ++part) {
        // complex column c (< bb) gives real-view columns c (Re) and bb + c
        // (Im); for c >= bb the zero columns 2c and 2c + 1 (they cover the
        // padding [2 bb, V))
        int vc = c;
        if constexpr (CPLX) vc = part == 0 ? (c < bb ? c : 2 * c) : (c < bb ? bb + c : 2 * c + 1);
        const int em = s_emax[vc];
        uint32_t s0[NSL], s1[NSL];
        slice8(pre[u][2 * part], em, 0, s0);
        slice8(pre[u][2 * part + 1], em, 0, s1);
#pragma unroll
        for (int a = 0; a < NSL; ++a) *reinterpret_cast<uint32_t*>(&Ss[a][vc][rp]) = s0[a] | (s1[a] << 16);
      }
    }
    if (c0 + OZ_CHUNK < r1) fetch(c0 + OZ_CHUNK);
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
    long long x[NLV];
#pragma unroll
    for (int L = 0; L < NLV; ++L) x[L] = float_int_to_ll(hi[L][q]) + (long long)__float2int_rn(lo[L][q]);
    const int e2 = (s_emax[i] - 1022) + (s_emax[j] - 1022) - OZ_EOFF;
    out[i * V + j] = levels_to_double(x, e2);
  }
}

// --------------------------------------------------------------- apply ----
// [Y_p Y_q] <- [Y_p Y_q] Z-tilde on a tile of 64 rows (real view, V <= 32):
// eight warps, warp w owns rows 16 (w & 3) + [0, 16) and V / 16 of the V / 8
// column tiles.
constexpr int ATR = 64;

template <int V, bool CPLX>
__global__ void __launch_bounds__(256) k_apply_oz(BlkDims d, BlkBuffers b, int step, int tile0, BlkBatch bt) {
  constexpr int YS = V + 8;  // padded row stride of the Y slices (bf16)
  constexpr int TS = V + 8;  // padded stride of a Z slice column (bf16)
  constexpr int NNW = V / 16;  // column tiles (n8) per warp
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint16_t* Ys = reinterpret_cast<uint16_t*>(smem_raw);  // [NSL][ATR][YS]
  uint16_t* Ts = Ys + NSL * ATR * YS;                    // [NSL][V][TS]
  double* Zd = reinterpret_cast<double*>(Ts + NSL * V * TS);  // [V][V], row k = Z-tilde row
  __shared__ int s_ey[V], s_fz[V];

  int slot;
  if (!batch_item(bt, blockIdx.x, step, d, b, slot)) return;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  if (!b.flags[slot]) return;
  const int tf = (d.mf + ATR - 1) / ATR, tg = (d.mg + ATR - 1) / ATR;
  int tile = tile0 + blockIdx.y;
  if (tile >= tf + tg + (d.n + ATR - 1) / ATR) return;
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
  //    thread x holds row x % 64 of the real-view column pairs
  //    (2 (x / 64 + 4 i), 2 (x / 64 + 4 i) + 1), i = 0 .. V / 8 - 1
  //    (complex: complex column x / 64 + 4 i gives real-view columns
  //    c (Re) and bb + c (Im), or the zero columns 2c, 2c + 1 for c >= bb)
  constexpr int NPR = V / 8;  // column pairs per thread
  for (int idx = threadIdx.x; idx < V * V; idx += 256) Zd[idx] = zt[idx];
  if (threadIdx.x < V) s_ey[threadIdx.x] = 1;
  const int rr = threadIdx.x & (ATR - 1), grp = threadIdx.x >> 6;
  const bool live = r0 + rr < m;
  double y[NPR][2];
  int yc[NPR][2];  // real-view columns of the two values
#pragma unroll
  for (int i = 0; i < NPR; ++i) {
    if constexpr (!CPLX) {
      const int c = 2 * (grp + 4 * i);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        yc[i][h] = c + h;
        y[i][h] = (c + h < bb && live) ? Y[(size_t)pc.gcol(c + h) * ld + r0 + rr] : 0.0;
      }
    } else {
      const int c = grp + 4 * i;
      double2 v = make_double2(0.0, 0.0);
      if (c < bb && live) v = reinterpret_cast<const double2*>(Y)[(size_t)pc.gcol(c) * ld + r0 + rr];
      y[i][0] = v.x;
      y[i][1] = v.y;
      yc[i][0] = c < bb ? c : 2 * c;
      yc[i][1] = c < bb ? bb + c : 2 * c + 1;
    }
  }
  __syncthreads();
  // 2. column exponents of the tile (two warps share a column: 64 rows)
#pragma unroll
  for (int i = 0; i < NPR; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int mx = __reduce_max_sync(FULL, exp_field(y[i][h]));
      if (lane == 0) atomicMax(&s_ey[yc[i][h]], mx);
    }
  __syncthreads();
  // 3. Z' = D Z-tilde (row k scaled by 2^(e_k)), its column exponents, slices
  //    (row pairs (k, k + 1) of a column packed in one word)
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
  for (int it = threadIdx.x; it < V * (V / 2); it += 256) {
    const int j = it % V, k = 2 * (it / V);
    uint32_t s0[NSL], s1[NSL];
    slice8(Zd[k * V + j], s_fz[j], s_ey[k] - 1022, s0);
    slice8(Zd[(k + 1) * V + j], s_fz[j], s_ey[k + 1] - 1022, s1);
#pragma unroll
    for (int a = 0; a < NSL; ++a) *reinterpret_cast<uint32_t*>(&Ts[(a * V + j) * TS + k]) = s0[a] | (s1[a] << 16);
  }
#pragma unroll
  for (int i = 0; i < NPR; ++i) {
    uint32_t s0[NSL], s1[NSL];
    slice8(y[i][0], s_ey[yc[i][0]], 0, s0);
    slice8(y[i][1], s_ey[yc[i][1]], 0, s1);
    if constexpr (!CPLX) {
#pragma unroll
      for (int a = 0; a < NSL; ++a)
        *reinterpret_cast<uint32_t*>(&Ys[(a * ATR + rr) * YS + yc[i][0]]) = s0[a] | (s1[a] << 16);
    } else {
#pragma unroll
      for (int a = 0; a < NSL; ++a) {
        Ys[(a * ATR + rr) * YS + yc[i][0]] = (uint16_t)s0[a];
        Ys[(a * ATR + rr) * YS + yc[i][1]] = (uint16_t)s1[a];
      }
    }
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
      long long x[NLV];
#pragma unroll
      for (int L = 0; L < NLV; ++L) x[L] = __float2int_rn(acc[u][L][q]);
      Ob[j * OS + r] = levels_to_double(x, s_fz[j] - 1022 - OZ_EOFF);
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


// ------------------------------------------------------ general DGEMM ----
// C = alpha op(A) op(B) + beta C (column-major FP64) on the BF16 tensor
// cores with FP64 accuracy, for the large products of the QR shortening.
// Each operand is sliced once into digit planes: for every row r of op(A)
// (every column of op(B)) one scale, the exponent field e[r] of its largest
// |value| over all of K, and S[p][r][k] = BF16 digit p of value (r, k),
// k < Kp = K rounded up to 32 (zero beyond K).  The product kernel then
// runs on 32 x 32 output tiles, K in chunks of 32 (exact FP32 level sums),
// flushed into exact FP32 double-words (TwoSum) and rounded once to FP64.

// rows whose k values are contiguous: value (r, k) = X[r ld + k]; one warp per row
__global__ void __launch_bounds__(256) k_slice_kc(int R, int K, const double* __restrict__ X, long long ld,
                                                  uint16_t* __restrict__ S, long long Kp, long long plane,
                                                  int* __restrict__ e) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * 8 + warp;
  if (r >= R) return;
  const double* row = X + (size_t)r * ld;
  int mx = 1;
  for (int k = lane; k < K; k += 32) mx = max(mx, exp_field(row[k]));
  mx = __reduce_max_sync(FULL, mx);
  if (lane == 0) e[r] = mx;
  uint16_t* out = S + (size_t)r * Kp;
  for (int k = 2 * lane; k < Kp; k += 64) {
    const double x0 = k < K ? row[k] : 0.0, x1 = k + 1 < K ? row[k + 1] : 0.0;
    uint32_t s0[NSL], s1[NSL];
    slice8(x0, mx, 0, s0);
    slice8(x1, mx, 0, s1);
#pragma unroll
    for (int q = 0; q < NSL; ++q) *reinterpret_cast<uint32_t*>(out + q * plane + k) = s0[q] | (s1[q] << 16);
  }
}

// rows that are strided: value (r, k) = X[k ld + r] (the rows of a
// column-major matrix); 32 rows per CTA, transposed through shared memory
__global__ void __launch_bounds__(256) k_slice_tr(int R, int K, const double* __restrict__ X, long long ld,
                                                  uint16_t* __restrict__ S, long long Kp, long long plane,
                                                  int* __restrict__ e) {
  __shared__ double T[32][33];
  __shared__ int s_e[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32, r = r0 + lane;
  const bool live = r < R;
  if (threadIdx.x < 32) s_e[threadIdx.x] = 1;
  int mx = 1;
  if (live)
    for (int k = warp; k < K; k += 8) mx = max(mx, exp_field(X[(size_t)k * ld + r]));
  __syncthreads();
  atomicMax(&s_e[lane], mx);
  __syncthreads();
  if (warp == 0 && live) e[r] = s_e[lane];
  for (int k0 = 0; k0 < Kp; k0 += 32) {
    for (int kk = warp; kk < 32; kk += 8) T[kk][lane] = (live && k0 + kk < K) ? X[(size_t)(k0 + kk) * ld + r] : 0.0;
    __syncthreads();
    for (int rr = warp; rr < 32; rr += 8) {
      if (r0 + rr < R && lane < 16) {
        const int kk = 2 * lane;
        uint32_t s0[NSL], s1[NSL];
        slice8(T[kk][rr], s_e[rr], 0, s0);
        slice8(T[kk + 1][rr], s_e[rr], 0, s1);
        uint16_t* out = S + (size_t)(r0 + rr) * Kp + k0 + kk;
#pragma unroll
        for (int q = 0; q < NSL; ++q) *reinterpret_cast<uint32_t*>(out + q * plane) = s0[q] | (s1[q] << 16);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;  // 0: the 16 bytes are zero-filled, nothing is read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int GT = 32;  // output tile edge of the general product

// one warp per m16 x n8 tile of the 32 x 32 output: rows 16 (w >> 2), columns 8 (w & 3)
__global__ void __launch_bounds__(256, 2) k_gemm_oz(int M, int N, int K, long long Kp, const uint16_t* __restrict__ As,
                                                 long long aplane, const uint16_t* __restrict__ Bs, long long bplane,
                                                 const int* __restrict__ ea, const int* __restrict__ eb, double alpha,
                                                 double beta, double* __restrict__ C, long long ldc, int upper) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [stage][operand][slice][row][GRS]
  uint16_t* sm = reinterpret_cast<uint16_t*>(smem_raw);
  auto at = [&](int st, int op, int q, int row) -> uint16_t* {
    return sm + ((((size_t)st * 2 + op) * NSL + q) * GT + row) * GRS;
  };
  const int m0 = blockIdx.x * GT, n0 = blockIdx.y * GT;
  if (upper && m0 >= n0 + GT) return;  // below the diagonal: not needed
  const int kbeg = upper == 2 ? m0 : 0;
  const int kend = upper == 2 ? min(K, n0 + GT) : K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = warp >> 2, nt = warp & 3, g = lane >> 2, t = lane & 3;
  // copies of one chunk: 2 operands x 7 slices x 32 rows x 4 pieces of 16 bytes
  auto issue = [&](int st, int k0) {
    for (int c = threadIdx.x; c < 2 * NSL * GT * 4; c += 256) {
      const int piece = c & 3, row = (c >> 2) % GT, q = (c >> 2) / GT % NSL, op = c / (NSL * GT * 4);
      const int rr = (op ? n0 : m0) + row;
      const bool valid = rr < (op ? N : M);
      const uint16_t* base = op ? Bs + q * bplane : As + q * aplane;
      const uint16_t* src = valid ? base + (size_t)rr * Kp + k0 + piece * 8 : base;
      cp_async16(at(st, op, q, row) + piece * 8, src, valid);
    }
    cp_async_commit();
  };
  float hi[NLV][4], lo[NLV][4];
#pragma unroll
  for (int L = 0; L < NLV; ++L)
#pragma unroll
    for (int q = 0; q < 4; ++q) hi[L][q] = lo[L][q] = 0.0f;
  int st = 0;
  if (kbeg < kend) issue(0, kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += OZ_CHUNK) {
    if (k0 + OZ_CHUNK < kend) {
      issue(st ^ 1, k0 + OZ_CHUNK);
      cp_async_wait_1();
    } else {
      cp_async_wait_0();
    }
    __syncthreads();
    float acc[NLV][4];
#pragma unroll
    for (int L = 0; L < NLV; ++L)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[L][q] = 0.0f;
#pragma unroll
    for (int kb = 0; kb < OZ_CHUNK; kb += 16) {
      uint32_t B[NSL][2];
#pragma unroll
      for (int q = 0; q < NSL; ++q) {
        const uint16_t* bp = at(st, 1, q, 8 * nt + g);
        B[q][0] = ld32(bp + kb + 2 * t);
        B[q][1] = ld32(bp + kb + 2 * t + 8);
      }
      auto load_a = [&](int q, uint32_t A[4]) {
        const uint16_t* ap = at(st, 0, q, 16 * mt + g);
        A[0] = ld32(ap + kb + 2 * t);
        A[1] = ld32(ap + 8 * GRS + kb + 2 * t);
        A[2] = ld32(ap + kb + 2 * t + 8);
        A[3] = ld32(ap + 8 * GRS + kb + 2 * t + 8);
      };
      level_mmas_stream(acc, load_a, B);
    }
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
    __syncthreads();  // this stage is refilled by the next issue
    st ^= 1;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = m0 + 16 * mt + g + ((q & 2) ? 8 : 0);
    const int j = n0 + 8 * nt + 2 * t + (q & 1);
    if (i >= M || j >= N) continue;
    long long x[NLV];
#pragma unroll
    for (int L = 0; L < NLV; ++L) x[L] = float_int_to_ll(hi[L][q]) + (long long)__float2int_rn(lo[L][q]);
    const double v = levels_to_double(x, (ea[i] - 1022) + (eb[j] - 1022) - OZ_EOFF);
    double* cp = C + (size_t)j * ldc + i;
    *cp = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *cp);
  }
}

template <int V>
size_t apply_oz_smem() {
  const size_t slices = sizeof(uint16_t) * NSL * ((size_t)ATR * (V + 8) + (size_t)V * (V + 8));
  const size_t out = sizeof(double) * V * (ATR + 1);
  return (slices > out ? slices : out) + sizeof(double) * V * V + 16;
}

// --------------------------------------------- apply on tcgen05 / TMEM ----
// The block apply [Y_p Y_q] <- [Y_p Y_q] Z-tilde of a tile of 128 rows on the
// 5th-generation tensor cores: the eight digit planes of the tile (A, 128 x V)
// and of Z-tilde' (B, V x V) are written to shared memory in the canonical
// K-major layout of 8 x 8 core matrices; one thread issues the
// tcgen05.mma.kind::f16 instructions (BF16 operands, FP32 accumulation), one
// accumulator per level L = a + b (V TMEM columns each, 8 levels); after a
// tcgen05.commit to an mbarrier every thread reads its row's level sums with
// tcgen05.ld and recombines them exactly (same arithmetic as k_apply_oz: the
// level sums are integers below 2^24, so the order of the tensor core's
// additions does not matter).
constexpr int TT = 128;  // rows per tile (M of the MMA; TMEM lane = row)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of tcgen05: start address, leading (K)
// and stride (M/N) byte offsets of the 8 x 8 core matrices, version 1, no
// swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// byte offset of element (r, k) of a K-major operand with K = V: core matrix
// (r / 8, k / 8) at (r / 8) 16 V + (k / 8) 128, 16 bytes per core-matrix row
template <int V>
__device__ __forceinline__ int tc_off(int r, int k) {
  return (r >> 3) * (16 * V) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&v)[N]);
template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

template <int V>
constexpr size_t apply_tc_smem() {
  return (size_t)NSL * TT * V * 2 + (size_t)NSL * V * V * 2 + (size_t)V * V * 8 + 1024;
}

template <int V, bool CPLX>
__global__ void __launch_bounds__(256, 2) k_apply_tc(BlkDims d, BlkBuffers b, int step, int tile0, BlkBatch bt) {
  constexpr int H = V / 2;              // real-view columns per thread (two threads per row)
  constexpr int APL = TT * V * 2;       // bytes of an A digit plane
  constexpr int BPL = V * V * 2;        // bytes of a B digit plane
  constexpr uint32_t TCOLS = NSL * V;   // TMEM columns: one V-wide accumulator per level
  extern __shared__ __align__(128) unsigned char tc_smem[];
  unsigned char* As = tc_smem;                                   // [NSL][APL]
  unsigned char* Bs = As + NSL * APL;                            // [NSL][BPL]
  double* Zd = reinterpret_cast<double*>(Bs + NSL * BPL);        // [V][V], row k = Z-tilde row
  __shared__ int s_ey[V], s_fz[V];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_bar;

  int slot;
  if (!batch_item(bt, blockIdx.x, step, d, b, slot)) return;
  PairCols pc;
  if (!load_pair(d, b, step, slot, pc)) return;
  if (!b.flags[slot]) return;
  const int tf = (d.mf + TT - 1) / TT, tg = (d.mg + TT - 1) / TT;
  int tile = tile0 + blockIdx.y;
  if (tile >= tf + tg + (d.n + TT - 1) / TT) return;
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
  const int r0 = tile * TT;
  const int bb = pc.bb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* zt = static_cast<const double*>(b.ztil) + (size_t)slot * V * V;

  // TMEM for the eight level accumulators (warp 0), the mbarrier of the MMAs
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_taddr)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }

  // 1. Z-tilde into shared memory; this thread's H real-view values of row
  //    r = tid % 128: columns h H + [0, H), h = tid / 128 (real view: complex
  //    column c gives Re in column c and Im in column bb + c; zero beyond 2 bb)
  for (int idx = tid; idx < V * V; idx += 256) Zd[idx] = zt[idx];
  if (tid < V) s_ey[tid] = 1;
  const int r = tid & (TT - 1), h = tid >> 7;
  const bool live = r0 + r < m;
  double y[H];
#pragma unroll
  for (int c = 0; c < H; ++c) {
    const int vc = h * H + c;
    double v = 0.0;
    if (live) {
      if constexpr (!CPLX) {
        if (vc < bb) v = Y[(size_t)pc.gcol(vc) * ld + r0 + r];
      } else {
        if (vc < bb) v = Y[2 * ((size_t)pc.gcol(vc) * ld + r0 + r)];
        else if (vc < 2 * bb) v = Y[2 * ((size_t)pc.gcol(vc - bb) * ld + r0 + r) + 1];
      }
    }
    y[c] = v;
  }
  __syncthreads();
  // 2. column exponents of the tile (four warps share a column: 128 rows)
#pragma unroll
  for (int c = 0; c < H; ++c) {
    const int mx = __reduce_max_sync(FULL, exp_field(y[c]));
    if (lane == 0) atomicMax(&s_ey[h * H + c], mx);
  }
  __syncthreads();
  // 3. Z' = D Z-tilde (row k scaled by 2^(e_k)): column exponents, then the
  //    digit planes of B = Z'^T (N = output column j, K = k), eight k per chunk
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
  for (int it = tid; it < V * (V / 2); it += 256) {  // two k per 32-bit word
    const int j = it / (V / 2), k = 2 * (it % (V / 2));
    uint32_t d0[NSL], d1[NSL];
    slice8(Zd[k * V + j], s_fz[j], s_ey[k] - 1022, d0);
    slice8(Zd[(k + 1) * V + j], s_fz[j], s_ey[k + 1] - 1022, d1);
#pragma unroll
    for (int a = 0; a < NSL; ++a) *reinterpret_cast<uint32_t*>(Bs + a * BPL + tc_off<V>(j, k)) = d0[a] | (d1[a] << 16);
  }
  // 4. the digit planes of A = the tile (M = row, K = real-view column)
#pragma unroll
  for (int c = 0; c < H; c += 2) {
    uint32_t d0[NSL], d1[NSL];
    slice8(y[c], s_ey[h * H + c], 0, d0);
    slice8(y[c + 1], s_ey[h * H + c + 1], 0, d1);
#pragma unroll
    for (int a = 0; a < NSL; ++a)
      *reinterpret_cast<uint32_t*>(As + a * APL + tc_off<V>(r, h * H + c)) = d0[a] | (d1[a] << 16);
  }
  // the operands become visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t taddr = s_taddr;

  // 5. the level products, issued by one thread: D_L += A_a B_b^T for
  //    a + b = L, K = V in steps of 16
  if (tid == 0) {
    // kind::f16: FP32 accumulator, BF16 A and B, both K-major, N = V, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(V >> 3) << 17) | ((uint32_t)(TT >> 4) << 24);
#pragma unroll
    for (int L = 0; L < NLV; ++L) {
      bool first = true;
#pragma unroll
      for (int a = 0; a <= L; ++a) {
        const int bq = L - a;
#pragma unroll
        for (int kk = 0; kk < V / 16; ++kk) {
          const uint64_t ad = tc_sdesc(smem_u32(As + a * APL) + kk * 256, 128, 16 * V);
          const uint64_t bd = tc_sdesc(smem_u32(Bs + bq * BPL) + kk * 256, 128, 16 * V);
          const uint32_t acc = first ? 0u : 1u;
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr + (uint32_t)(L * V)),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                       : "memory");
          first = false;
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(&s_bar))
                 : "memory");
  }
  // 6. wait for the products (bounded: on a time-out the tile is left as it
  //    was and the pass is counted as failed, so the solve reports it)
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(smem_u32(&s_bar))
                 : "memory");
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (done) {
    // 7. this thread's row r = 32 (warp % 4) + lane (its TMEM lane) and
    //    columns h H + [0, H): the eight level sums of each output, recombined
    const uint32_t tl = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(h * H);
#pragma unroll 1
    for (int cg = 0; cg < H; cg += 8) {  // eight outputs at a time
      long long hi[8], lo[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) hi[c] = lo[c] = 0;
#pragma unroll
      for (int L = 0; L < NLV; ++L) {
        uint32_t v[8];
        tmem_ld<8>(tl + (uint32_t)(L * V + cg), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        const int sh = 24 - 8 * (L & 3);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const long long x = float_int_to_ll(__uint_as_float(v[c])) << sh;
          if (L < 4) hi[c] += x; else lo[c] += x;
        }
      }
      if (live) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int j = h * H + cg + c;
          if (j >= (CPLX ? 2 : 1) * bb) continue;
          const double out = levels_to_double_hl(hi[c], lo[c], s_fz[j] - 1022 - OZ_EOFF);
          if constexpr (!CPLX) {
            Y[(size_t)pc.gcol(j) * ld + r0 + r] = out;
          } else {
            if (j < bb) Y[2 * ((size_t)pc.gcol(j) * ld + r0 + r)] = out;
            else Y[2 * ((size_t)pc.gcol(j - bb) * ld + r0 + r) + 1] = out;
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicAdd(&b.ctr[2], 1ull);  // reported as a failed pass (the solve returns ENOTPD)
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(TCOLS) : "memory");
}

}  // namespace

bool oz_supported(int V) { return V == 16 || V == 32; }

cudaError_t launch_gram_oz(const BlkDims& d, const BlkBuffers& b, bool cplx, int step, cudaStream_t s,
                           const BlkBatch* bt, int nitems, int grid_y) {
  const int V = blk_vmax(d.w, cplx);
  // a row split is one exact accumulation: at most OZ_K_MAX rows (the batch
  // planner checks every problem of a batch)
  auto per = [](int m, int nsplit) { return ((m + 63) / 64 + nsplit - 1) / nsplit * 64; };
  if (!bt && (per(d.mf, d.rf) > OZ_K_MAX || per(d.mg, d.rg) > OZ_K_MAX)) return cudaErrorInvalidValue;
  const BlkBatch one;
  const BlkBatch& bb = bt ? *bt : one;
  dim3 grid(bt ? nitems : d.nslots, bt ? grid_y : d.rf + d.rg);
  if (V == 16) {
    if (cplx) k_gram_oz<16, true><<<grid, 32 * oz_gram_warps<16>(), 0, s>>>(d, b, step, bb);
    else k_gram_oz<16, false><<<grid, 32 * oz_gram_warps<16>(), 0, s>>>(d, b, step, bb);
  } else if (V == 32) {
    if (cplx) k_gram_oz<32, true><<<grid, 32 * oz_gram_warps<32>(), 0, s>>>(d, b, step, bb);
    else k_gram_oz<32, false><<<grid, 32 * oz_gram_warps<32>(), 0, s>>>(d, b, step, bb);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int V, bool CPLX>
static cudaError_t apply_oz_v(const BlkDims& d, const BlkBuffers& b, int step, cudaStream_t s, const BlkBatch* bt,
                              int nitems, int grid_y) {
  const size_t smem = apply_oz_smem<V>();
  auto kern = k_apply_oz<V, CPLX>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (bt) {  // batched: one launch, grid y = the largest problem's row tiles (the planner keeps it <= 65535)
    kern<<<dim3(nitems, grid_y), 256, smem, s>>>(d, b, step, 0, *bt);
    return cudaGetLastError();
  }
  const BlkBatch one;
  const int tiles = (d.mf + ATR - 1) / ATR + (d.mg + ATR - 1) / ATR + (d.n + ATR - 1) / ATR;
  // tiles of F, G, Z on grid y, in launches of at most 65535 tiles each
  for (int t0 = 0; t0 < tiles; t0 += 65535) {
    dim3 grid(d.nslots, std::min(65535, tiles - t0));
    kern<<<grid, 256, smem, s>>>(d, b, step, t0, one);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int V, bool CPLX>
static cudaError_t apply_tc_v(const BlkDims& d, const BlkBuffers& b, int step, cudaStream_t s, const BlkBatch* bt,
                              int nitems, int grid_y) {
  constexpr size_t smem = apply_tc_smem<V>();
  auto kern = k_apply_tc<V, CPLX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (bt) {  // batched: grid y sized for 64-row tiles; the extra blocks leave at once
    kern<<<dim3(nitems, grid_y), 256, smem, s>>>(d, b, step, 0, *bt);
    return cudaGetLastError();
  }
  const BlkBatch one;
  const int tiles = (d.mf + TT - 1) / TT + (d.mg + TT - 1) / TT + (d.n + TT - 1) / TT;
  for (int t0 = 0; t0 < tiles; t0 += 65535) {
    kern<<<dim3(d.nslots, std::min(65535, tiles - t0)), 256, smem, s>>>(d, b, step, t0, one);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_apply_oz(const BlkDims& d, const BlkBuffers& b, bool cplx, int step, cudaStream_t s, bool tc,
                            const BlkBatch* bt, int nitems, int grid_y) {
  const int V = blk_vmax(d.w, cplx);
  if (tc) {
    if (V == 16)
      return cplx ? apply_tc_v<16, true>(d, b, step, s, bt, nitems, grid_y)
                  : apply_tc_v<16, false>(d, b, step, s, bt, nitems, grid_y);
    if (V == 32)
      return cplx ? apply_tc_v<32, true>(d, b, step, s, bt, nitems, grid_y)
                  : apply_tc_v<32, false>(d, b, step, s, bt, nitems, grid_y);
  }
  if (V == 16)
    return cplx ? apply_oz_v<16, true>(d, b, step, s, bt, nitems, grid_y)
                : apply_oz_v<16, false>(d, b, step, s, bt, nitems, grid_y);
  if (V == 32)
    return cplx ? apply_oz_v<32, true>(d, b, step, s, bt, nitems, grid_y)
                : apply_oz_v<32, false>(d, b, step, s, bt, nitems, grid_y);
  return cudaErrorInvalidValue;
}


static size_t align256z(size_t x) { return (x + 255) & ~size_t(255); }

size_t dgemm_oz_ws_bytes(int M, int N, int K) {
  const size_t Kp = (size_t)(K + 31) / 32 * 32;
  return align256z(sizeof(uint16_t) * NSL * (size_t)M * Kp) + align256z(sizeof(uint16_t) * NSL * (size_t)N * Kp) +
         align256z(sizeof(int) * ((size_t)M + N)) + 256;
}

cudaError_t dgemm_oz(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long long lda,
                     const double* B, long long ldb, double beta, double* C, long long ldc, int upper, void* ws,
                     size_t ws_bytes, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!ws || K <= 0 || K > OZ_K_MAX || ws_bytes < dgemm_oz_ws_bytes(M, N, K)) return cudaErrorInvalidValue;
  const long long Kp = (long long)(K + 31) / 32 * 32;
  unsigned char* w = static_cast<unsigned char*>(ws);
  uint16_t* As = reinterpret_cast<uint16_t*>(w);
  w += align256z(sizeof(uint16_t) * NSL * (size_t)M * Kp);
  uint16_t* Bs = reinterpret_cast<uint16_t*>(w);
  w += align256z(sizeof(uint16_t) * NSL * (size_t)N * Kp);
  int* ea = reinterpret_cast<int*>(w);
  int* eb = ea + M;
  const long long aplane = (long long)M * Kp, bplane = (long long)N * Kp;
  // the Gram op(A) = A^T, op(B) = A slices the same rows once
  const bool same = ta && !tb && A == B && lda == ldb && M == N;
  // rows of op(A): columns of A (ta) or rows of A; columns of op(B): columns of B (!tb) or rows of B
  if (ta)
    k_slice_kc<<<(M + 7) / 8, 256, 0, s>>>(M, K, A, lda, As, Kp, aplane, ea);
  else
    k_slice_tr<<<(M + 31) / 32, 256, 0, s>>>(M, K, A, lda, As, Kp, aplane, ea);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (same) {
    Bs = As;
    eb = ea;
  } else {
    if (!tb)
      k_slice_kc<<<(N + 7) / 8, 256, 0, s>>>(N, K, B, ldb, Bs, Kp, bplane, eb);
    else
      k_slice_tr<<<(N + 31) / 32, 256, 0, s>>>(N, K, B, ldb, Bs, Kp, bplane, eb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = sizeof(uint16_t) * 2 * 2 * NSL * GT * GRS;
  e = cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT);
  k_gemm_oz<<<grid, 256, smem, s>>>(M, N, K, Kp, As, aplane, Bs, same ? aplane : bplane, ea, eb, alpha, beta, C,
                                    ldc, upper);
  return cudaGetLastError();
}

}  // namespace hz
