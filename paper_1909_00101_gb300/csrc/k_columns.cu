// k_columns.cu -- column-wise and dense helper kernels of the sweep engine:
// prescaling (Sec. 2, initFGZ of Sec. 3.3), the between-sweep rescaling of Z
// and the final extraction of U, V, Z, Sigma_F, Sigma_G, Sigma with the sort by
// descending Sigma (Sec. 2.4, Sec. 3.4, Sec. 1), and the conversions and the
// FP64 product F <- F Z_acc of the mixed-precision path.
//
// Column kernels use one warp per column with lane-strided partial sums and a
// fixed xor-butterfly reduction (Appendix C), so every result is bitwise
// reproducible.  They are HBM-bound: each reads (and writes) a column once.
#include <type_traits>

#include "hz_device.cuh"
#include "hz_kernels.h"

namespace hz {

namespace {

constexpr int CW = 8;  // columns (warps) per CTA

template <class T>
__device__ __forceinline__ double col_sumsq(const T* y, int len) {
  double s = 0.0;
  for (int r = (threadIdx.x & 31); r < len; r += 32) {
    const double v = (double)y[r];
    s = fma(v, v, s);
  }
  return warp_sum(s);
}

__global__ void __launch_bounds__(256) k_prescale(int mf, int mg, int n, int E, double* F, long long ldf,
                                                  double* G, long long ldg, double* Z, long long ldz,
                                                  double* zdiag, int* status) {
  const int j = blockIdx.x * CW + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  double* g = G + (size_t)j * E * ldg;
  double* f = F + (size_t)j * E * ldf;
  const double s = col_sumsq(g, E * mg);
  double zj = 1.0;
  if (!(s > 0.0) || !isfinite(s)) {
    if (lane == 0) atomicExch(status, ST_ENOTPD);
  } else {
    zj = 1.0 / sqrt(s);
  }
  for (int r = lane; r < E * mf; r += 32) f[r] *= zj;
  for (int r = lane; r < E * mg; r += 32) g[r] *= zj;
  double* z = Z + (size_t)j * E * ldz;
  for (int r = lane; r < E * n; r += 32) z[r] = (r == E * j) ? zj : 0.0;
  if (lane == 0) zdiag[j] = zj;
}

// Between sweeps (Sec. 2.4): theta_j = (||f_j||^2 + ||g_j||^2)^{-1/2}.  The
// paper scales only z_j, relying on every block visit to leave its columns
// normalised; visits without any transformation are skipped here (Sec. 2.5
// allows skipping identity updates), so f_j and g_j are scaled with z_j: the
// same diagonal congruence on all three keeps F Z = F_k exact.
template <class T>
__global__ void __launch_bounds__(256) k_rescale(int mf, int mg, int n, int E, T* F, long long ldf,
                                                 T* G, long long ldg, T* Z, long long ldz) {
  const int j = blockIdx.x * CW + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  T* f = F + (size_t)j * E * ldf;
  T* g = G + (size_t)j * E * ldg;
  const double sf = col_sumsq(f, E * mf);
  const double sg = col_sumsq(g, E * mg);
  const double th = 1.0 / sqrt(sf + sg);
  if (th != 1.0) {
    T* z = Z + (size_t)j * E * ldz;
    for (int r = lane; r < E * n; r += 32) z[r] = (T)((double)z[r] * th);
    for (int r = lane; r < E * mf; r += 32) f[r] = (T)((double)f[r] * th);
    for (int r = lane; r < E * mg; r += 32) g[r] = (T)((double)g[r] * th);
  }
}

// column norms ||f_j||, ||g_j|| into norms[0..n), norms[n..2n)
__global__ void __launch_bounds__(256) k_norms(int mf, int mg, int n, int E, const double* F, long long ldf,
                                               const double* G, long long ldg, double* norms, int* status) {
  const int j = blockIdx.x * CW + (threadIdx.x >> 5);
  if (j >= n) return;
  const double sf = col_sumsq(F + (size_t)j * E * ldf, E * mf);
  const double sg = col_sumsq(G + (size_t)j * E * ldg, E * mg);
  if ((threadIdx.x & 31) == 0) {
    norms[j] = sqrt(sf);
    norms[n + j] = sqrt(sg);
    if (!isfinite(sf) || !isfinite(sg) || !(sg > 0.0)) atomicExch(status, ST_EOVERFLOW);
  }
}

// stable rank of column j by descending sigma_j = ||f_j|| / ||g_j||
__global__ void k_rank(int n, const double* norms, int* rank) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double sj = norms[j] / norms[n + j];
  int rk = 0;
  for (int k = 0; k < n; ++k) {
    const double sk = norms[k] / norms[n + k];
    rk += (sk > sj) || (sk == sj && k < j);
  }
  rank[j] = rk;
}

// out[:, rank[j]] = in[:, j] * scale_j, where scale_j = 1/norms[off + j]
// (mode 0) or Theta_j (mode 1)
__global__ void __launch_bounds__(256) k_gather(int m, int n, int E, const double* in, long long ldi,
                                                double* out, long long ldo, const double* norms,
                                                const int* rank, int mode, int off) {
  const int j = blockIdx.x * CW + (threadIdx.x >> 5);
  if (j >= n) return;
  double sc;
  if (mode == 0) {
    sc = 1.0 / norms[off + j];
  } else {
    const double nf = norms[j], ng = norms[n + j];
    sc = 1.0 / sqrt(fma(nf, nf, ng * ng));
  }
  const double* src = in + (size_t)j * E * ldi;
  double* dst = out + (size_t)rank[j] * E * ldo;
  for (int r = (threadIdx.x & 31); r < E * m; r += 32) dst[r] = (mode == 0) ? src[r] / norms[off + j] : src[r] * sc;
}

__global__ void k_sigmas(int n, const double* norms, const int* rank, double* sf, double* sg, double* sigma) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double nf = norms[j], ng = norms[n + j];
  const double th = 1.0 / sqrt(fma(nf, nf, ng * ng));
  sf[rank[j]] = nf * th;
  sg[rank[j]] = ng * th;
  sigma[rank[j]] = nf / ng;
}

__global__ void k_copy_cols(int m, int n, int E, const double* in, long long ldi, double* out, long long ldo) {
  const int j = blockIdx.x * CW + (threadIdx.x >> 5);
  if (j >= n) return;
  const double* src = in + (size_t)j * E * ldi;
  double* dst = out + (size_t)j * E * ldo;
  for (int r = (threadIdx.x & 31); r < E * m; r += 32) dst[r] = src[r];
}

__global__ void k_to_f32(int m, int n, int E, const double* src, long long lds, float* dst, long long ldd) {
  const int j = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < E * m; r += gridDim.x * blockDim.x)
    dst[(size_t)j * E * ldd + r] = __double2float_rn(src[(size_t)j * E * lds + r]);
}

template <class T>
__global__ void k_identity(int n, int E, T* Z, long long ldz) {
  const int j = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < E * n; r += gridDim.x * blockDim.x)
    Z[(size_t)j * E * ldz + r] = (r == E * j) ? T(1) : T(0);
}

__global__ void k_rowscale(int n, int E, const double* zdiag, const float* Z32, long long ld32, double* Z,
                           long long ldz) {
  const int j = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < E * n; r += gridDim.x * blockDim.x)
    Z[(size_t)j * E * ldz + r] = zdiag[r / E] * (double)Z32[(size_t)j * E * ld32 + r];
}

__global__ void k_check_finite(int m, int n, int E, const double* A, long long lda, int* flag) {
  const int j = blockIdx.y;
  bool bad = false;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < E * m; r += gridDim.x * blockDim.x)
    bad |= !isfinite(A[(size_t)j * E * lda + r]);
  if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// C (m x n) = A (m x n) * B (n x n) in FP64 on the DMMA pipe, B given in FP32
// (the accumulated transformation of the FP32 sweeps; every FP32 value is
// exact in FP64).  Tiles of 64 x 64 outputs, K in chunks of 32; real only (the
// complex product runs on real views: see launch_gemm_f64_by_f32).
constexpr int GM = 64, GN = 64, GK = 32;
__global__ void __launch_bounds__(256) k_gemm_f64(int m, int n, int kdim, const double* A, long long lda,
                                                  const float* B, long long ldb, double* C, long long ldc) {
  __shared__ double As[GK][GM + 8];  // As[k][r]
  __shared__ double Bs[GK][GN + 8];  // Bs[k][c]
  const int r0 = blockIdx.x * GM, c0 = blockIdx.y * GN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[8][2];
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t][0] = acc[t][1] = 0.0;
  for (int k0 = 0; k0 < kdim; k0 += GK) {
    for (int idx = threadIdx.x; idx < GK * GM; idx += blockDim.x) {
      const int k = idx / GM, r = idx % GM;
      As[k][r] = (r0 + r < m && k0 + k < kdim) ? A[(size_t)(k0 + k) * lda + r0 + r] : 0.0;
    }
    for (int idx = threadIdx.x; idx < GK * GN; idx += blockDim.x) {
      const int c = idx / GK, k = idx % GK;
      Bs[k][c] = (c0 + c < n && k0 + k < kdim) ? (double)B[(size_t)(c0 + c) * ldb + k0 + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk += 4) {
      const double a = As[kk + (lane & 3)][warp * 8 + (lane >> 2)];
#pragma unroll
      for (int t = 0; t < 8; ++t) dmma(acc[t][0], acc[t][1], a, Bs[kk + (lane & 3)][t * 8 + (lane >> 2)]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = r0 + warp * 8 + (lane >> 2), c = c0 + t * 8 + 2 * (lane & 3);
    if (r < m && c < n) C[(size_t)c * ldc + r] = acc[t][0];
    if (r < m && c + 1 < n) C[(size_t)(c + 1) * ldc + r] = acc[t][1];
  }
}

// complex C = A B via real views: A interleaved (re, im) of m x n; Re/Im
// planes of A and B are extracted by strided indexing in the real GEMM:
// Re C = Re A Re B - Im A Im B, Im C = Re A Im B + Im A Re B.
constexpr int GKC = 16;
__global__ void __launch_bounds__(256) k_gemm_c64(int m, int n, const double* A, long long lda,
                                                  const float* B, long long ldb, double* C, long long ldc) {
  __shared__ double Ar[GKC][GM + 8], Ai[GKC][GM + 8];
  __shared__ double Br[GKC][GN + 8], Bi[GKC][GN + 8];
  const int r0 = blockIdx.x * GM, c0 = blockIdx.y * GN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double accr[8][2], acci[8][2];
#pragma unroll
  for (int t = 0; t < 8; ++t) accr[t][0] = accr[t][1] = acci[t][0] = acci[t][1] = 0.0;
  for (int k0 = 0; k0 < n; k0 += GKC) {
    for (int idx = threadIdx.x; idx < GKC * GM; idx += blockDim.x) {
      const int k = idx / GM, r = idx % GM;
      const bool ok = r0 + r < m && k0 + k < n;
      Ar[k][r] = ok ? A[2 * ((size_t)(k0 + k) * lda + r0 + r)] : 0.0;
      Ai[k][r] = ok ? A[2 * ((size_t)(k0 + k) * lda + r0 + r) + 1] : 0.0;
    }
    for (int idx = threadIdx.x; idx < GKC * GN; idx += blockDim.x) {
      const int c = idx / GKC, k = idx % GKC;
      const bool ok = c0 + c < n && k0 + k < n;
      Br[k][c] = ok ? (double)B[2 * ((size_t)(c0 + c) * ldb + k0 + k)] : 0.0;
      Bi[k][c] = ok ? (double)B[2 * ((size_t)(c0 + c) * ldb + k0 + k) + 1] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GKC; kk += 4) {
      const double ar = Ar[kk + (lane & 3)][warp * 8 + (lane >> 2)];
      const double ai = Ai[kk + (lane & 3)][warp * 8 + (lane >> 2)];
      const double nai = -ai;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const double br = Br[kk + (lane & 3)][t * 8 + (lane >> 2)];
        const double bi = Bi[kk + (lane & 3)][t * 8 + (lane >> 2)];
        dmma(accr[t][0], accr[t][1], ar, br);
        dmma(accr[t][0], accr[t][1], nai, bi);
        dmma(acci[t][0], acci[t][1], ar, bi);
        dmma(acci[t][0], acci[t][1], ai, br);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = r0 + warp * 8 + (lane >> 2), c = c0 + t * 8 + 2 * (lane & 3);
    if (r < m && c < n) {
      C[2 * ((size_t)c * ldc + r)] = accr[t][0];
      C[2 * ((size_t)c * ldc + r) + 1] = acci[t][0];
    }
    if (r < m && c + 1 < n) {
      C[2 * ((size_t)(c + 1) * ldc + r)] = accr[t][1];
      C[2 * ((size_t)(c + 1) * ldc + r) + 1] = acci[t][1];
    }
  }
}

inline int cgrid(int n) { return (n + CW - 1) / CW; }

}  // namespace

cudaError_t launch_prescale(int mf, int mg, int n, bool cplx, double* F, long long ldf, double* G, long long ldg,
                            double* Z, long long ldz, double* zdiag, int* status, cudaStream_t s) {
  k_prescale<<<cgrid(n), 32 * CW, 0, s>>>(mf, mg, n, cplx ? 2 : 1, F, ldf, G, ldg, Z, ldz, zdiag, status);
  return cudaGetLastError();
}

cudaError_t launch_rescale(int mf, int mg, int n, bool cplx, bool fp32, void* F, long long ldf, void* G,
                           long long ldg, void* Z, long long ldz, cudaStream_t s) {
  const int E = cplx ? 2 : 1;
  if (fp32)
    k_rescale<float><<<cgrid(n), 32 * CW, 0, s>>>(mf, mg, n, E, (float*)F, ldf, (float*)G, ldg, (float*)Z, ldz);
  else
    k_rescale<double><<<cgrid(n), 32 * CW, 0, s>>>(mf, mg, n, E, (double*)F, ldf, (double*)G, ldg, (double*)Z,
                                                   ldz);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int mf, int mg, int n, bool cplx, double* F, long long ldf, double* G, long long ldg,
                            double* Z, long long ldz, double* sf, double* sg, double* sigma, double* norms,
                            int* rank, double* work, int* status, cudaStream_t s) {
  const int E = cplx ? 2 : 1;
  k_norms<<<cgrid(n), 32 * CW, 0, s>>>(mf, mg, n, E, F, ldf, G, ldg, norms, status);
  k_rank<<<(n + 127) / 128, 128, 0, s>>>(n, norms, rank);
  // U = F Sigma~_F^{-1}, permuted, via the scratch buffer, then copied back
  k_gather<<<cgrid(n), 32 * CW, 0, s>>>(mf, n, E, F, ldf, work, mf, norms, rank, 0, 0);
  k_copy_cols<<<cgrid(n), 32 * CW, 0, s>>>(mf, n, E, work, mf, F, ldf);
  k_gather<<<cgrid(n), 32 * CW, 0, s>>>(mg, n, E, G, ldg, work, mg, norms, rank, 0, n);
  k_copy_cols<<<cgrid(n), 32 * CW, 0, s>>>(mg, n, E, work, mg, G, ldg);
  k_gather<<<cgrid(n), 32 * CW, 0, s>>>(n, n, E, Z, ldz, work, n, norms, rank, 1, 0);
  k_copy_cols<<<cgrid(n), 32 * CW, 0, s>>>(n, n, E, work, n, Z, ldz);
  k_sigmas<<<(n + 127) / 128, 128, 0, s>>>(n, norms, rank, sf, sg, sigma);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(int m, int n, bool cplx, const double* src, long long lds, float* dst, long long ldd,
                          cudaStream_t s) {
  const int E = cplx ? 2 : 1;
  dim3 grid((E * m + 255) / 256, n);
  k_to_f32<<<grid, 256, 0, s>>>(m, n, E, src, lds, dst, ldd);
  return cudaGetLastError();
}

cudaError_t launch_identity(int n, bool cplx, bool fp32, void* Z, long long ldz, cudaStream_t s) {
  const int E = cplx ? 2 : 1;
  dim3 grid((E * n + 255) / 256, n);
  if (fp32)
    k_identity<float><<<grid, 256, 0, s>>>(n, E, (float*)Z, ldz);
  else
    k_identity<double><<<grid, 256, 0, s>>>(n, E, (double*)Z, ldz);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64_by_f32(int m, int n, bool cplx, const double* A, long long lda, const float* B,
                                   long long ldb, double* C, long long ldc, cudaStream_t s) {
  dim3 grid((m + GM - 1) / GM, (n + GN - 1) / GN);
  if (cplx)
    k_gemm_c64<<<grid, 256, 0, s>>>(m, n, A, lda, B, ldb, C, ldc);
  else
    k_gemm_f64<<<grid, 256, 0, s>>>(m, n, n, A, lda, B, ldb, C, ldc);
  return cudaGetLastError();
}

// X(i, j) <- sf_i X(i, j) + sg_i T(i, j)  (n x n, column-major)
// X <- diag(sf) X + diag(sg) T for n x n matrices (E scalars per element;
// ldx, ldt in elements): row i of both scaled by real factors
__global__ void k_rows_combine(int n, int E, double* X, long long ldx, const double* sf, const double* T,
                               long long ldt, const double* sg) {
  const int j = blockIdx.y;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < E * n; q += gridDim.x * blockDim.x) {
    const int i = q / E;
    X[(size_t)j * E * ldx + q] = fma(sf[i], X[(size_t)j * E * ldx + q], sg[i] * T[(size_t)j * E * ldt + q]);
  }
}

cudaError_t launch_rows_combine(int n, bool cplx, double* X, long long ldx, const double* sf, const double* T,
                                long long ldt, const double* sg, cudaStream_t s) {
  const int E = cplx ? 2 : 1;
  dim3 grid((E * n + 255) / 256, n);
  k_rows_combine<<<grid, 256, 0, s>>>(n, E, X, ldx, sf, T, ldt, sg);
  return cudaGetLastError();
}

// C = A^H B for complex A (m x k), B (m x n), C (k x n), interleaved (re, im),
// leading dimensions in complex elements: 16 x 16 output tiles, 16-row
// chunks of A and B staged in shared memory (loaded along the columns), each
// entry summed over the rows in order with FP64 fmas
__global__ void __launch_bounds__(256) k_gemm_ch(int m, int k, int n, const double2* A, long long lda,
                                                 const double2* B, long long ldb, double2* C, long long ldc) {
  __shared__ double2 As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int c0 = blockIdx.x * 16, d0 = blockIdx.y * 16;
  double cr = 0.0, ci = 0.0;
  for (int r0 = 0; r0 < m; r0 += 16) {
    const int r = r0 + tx;  // consecutive threads read consecutive rows of one column
    As[tx][ty] = (r < m && c0 + ty < k) ? A[(size_t)(c0 + ty) * lda + r] : make_double2(0.0, 0.0);
    Bs[tx][ty] = (r < m && d0 + ty < n) ? B[(size_t)(d0 + ty) * ldb + r] : make_double2(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double2 a = As[q][tx], b = Bs[q][ty];
      cr = fma(a.x, b.x, fma(a.y, b.y, cr));    // Re(conj(a) b)
      ci = fma(a.x, b.y, fma(-a.y, b.x, ci));   // Im(conj(a) b)
    }
    __syncthreads();
  }
  if (c0 + tx < k && d0 + ty < n) C[(size_t)(d0 + ty) * ldc + c0 + tx] = make_double2(cr, ci);
}

cudaError_t launch_gemm_ch(int m, int k, int n, const double* A, long long lda, const double* B, long long ldb,
                           double* C, long long ldc, cudaStream_t s) {
  dim3 grid((k + 15) / 16, (n + 15) / 16);
  k_gemm_ch<<<grid, 256, 0, s>>>(m, k, n, reinterpret_cast<const double2*>(A), lda,
                                 reinterpret_cast<const double2*>(B), ldb, reinterpret_cast<double2*>(C), ldc);
  return cudaGetLastError();
}

// A (rows x n) <- deterministic values in [-1, 1): a 64-bit hash of the
// element's index and the seed (SplitMix64's finaliser), the top 53 bits
// taken as a fraction
__global__ void k_fill_hash(int rows, int n, unsigned seed, double* A, long long lda) {
  const int j = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    unsigned long long x = ((unsigned long long)seed << 48) ^ ((unsigned long long)j * rows + r);
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    A[(size_t)j * lda + r] = (double)(x >> 11) * (1.0 / 4503599627370496.0) - 1.0;
  }
}

cudaError_t launch_fill_hash(int rows, int n, unsigned seed, double* A, long long lda, cudaStream_t s) {
  dim3 grid((rows + 255) / 256 < 64 ? (rows + 255) / 256 : 64, n);
  k_fill_hash<<<grid, 256, 0, s>>>(rows, n, seed, A, lda);
  return cudaGetLastError();
}

cudaError_t launch_rowscale(int n, bool cplx, const double* zdiag, const float* Z32, long long ld32, double* Z,
                            long long ldz, cudaStream_t s) {
  const int E = cplx ? 2 : 1;
  dim3 grid((E * n + 255) / 256, n);
  k_rowscale<<<grid, 256, 0, s>>>(n, E, zdiag, Z32, ld32, Z, ldz);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(int m, int n, bool cplx, const double* A, long long lda, int* flag,
                                cudaStream_t s) {
  const int E = cplx ? 2 : 1;
  dim3 grid((E * m + 255) / 256, n);
  k_check_finite<<<grid, 256, 0, s>>>(m, n, E, A, lda, flag);
  return cudaGetLastError();
}

}  // namespace hz
