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

__device__ __forceinline__ void prescale_at(int bx, int by, int mf, int mg, int n, int E, double* F, long long ldf,
                                                  double* G, long long ldg, double* Z, long long ldz,
                                                  double* zdiag, int* status) {
  const int j = bx * CW + (threadIdx.x >> 5);
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

__global__ void __launch_bounds__(256) k_prescale(int mf, int mg, int n, int E, double* F, long long ldf,
                                                  double* G, long long ldg, double* Z, long long ldz,
                                                  double* zdiag, int* status) {
  prescale_at(blockIdx.x, blockIdx.y, mf, mg, n, E, F, ldf, G, ldg, Z, ldz, zdiag, status);
}

// Between sweeps (Sec. 2.4): theta_j = (||f_j||^2 + ||g_j||^2)^{-1/2}.  The
// paper scales only z_j, relying on every block visit to leave its columns
// normalised; visits without any transformation are skipped here (Sec. 2.5
// allows skipping identity updates), so f_j and g_j are scaled with z_j: the
// same diagonal congruence on all three keeps F Z = F_k exact.
template <class T>
__device__ __forceinline__ void rescale_at(int bx, int by, int mf, int mg, int n, int E, T* F, long long ldf,
                                                 T* G, long long ldg, T* Z, long long ldz) {
  const int j = bx * CW + (threadIdx.x >> 5);
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

template <class T>
__global__ void __launch_bounds__(256) k_rescale(int mf, int mg, int n, int E, T* F, long long ldf,
                                                 T* G, long long ldg, T* Z, long long ldz) {
  rescale_at<T>(blockIdx.x, blockIdx.y, mf, mg, n, E, F, ldf, G, ldg, Z, ldz);
}

// column norms ||f_j||, ||g_j|| into norms[0..n), norms[n..2n)
__device__ __forceinline__ void norms_at(int bx, int by, int mf, int mg, int n, int E, const double* F, long long ldf,
                                               const double* G, long long ldg, double* norms, int* status) {
  const int j = bx * CW + (threadIdx.x >> 5);
  if (j >= n) return;
  const double sf = col_sumsq(F + (size_t)j * E * ldf, E * mf);
  const double sg = col_sumsq(G + (size_t)j * E * ldg, E * mg);
  if ((threadIdx.x & 31) == 0) {
    norms[j] = sqrt(sf);
    norms[n + j] = sqrt(sg);
    if (!isfinite(sf) || !isfinite(sg) || !(sg > 0.0)) atomicExch(status, ST_EOVERFLOW);
  }
}

__global__ void __launch_bounds__(256) k_norms(int mf, int mg, int n, int E, const double* F, long long ldf,
                                               const double* G, long long ldg, double* norms, int* status) {
  norms_at(blockIdx.x, blockIdx.y, mf, mg, n, E, F, ldf, G, ldg, norms, status);
}

// stable rank of column j by descending sigma_j = ||f_j|| / ||g_j||
__device__ __forceinline__ void rank_at(int bx, int by, int n, const double* norms, int* rank) {
  const int j = bx * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double sj = norms[j] / norms[n + j];
  int rk = 0;
  for (int k = 0; k < n; ++k) {
    const double sk = norms[k] / norms[n + k];
    rk += (sk > sj) || (sk == sj && k < j);
  }
  rank[j] = rk;
}

__global__ void k_rank(int n, const double* norms, int* rank) {
  rank_at(blockIdx.x, blockIdx.y, n, norms, rank);
}

// out[:, rank[j]] = in[:, j] * scale_j, where scale_j = 1/norms[off + j]
// (mode 0) or Theta_j (mode 1)
__device__ __forceinline__ void gather_at(int bx, int by, int m, int n, int E, const double* in, long long ldi,
                                                double* out, long long ldo, const double* norms,
                                                const int* rank, int mode, int off) {
  const int j = bx * CW + (threadIdx.x >> 5);
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

__global__ void __launch_bounds__(256) k_gather(int m, int n, int E, const double* in, long long ldi,
                                                double* out, long long ldo, const double* norms,
                                                const int* rank, int mode, int off) {
  gather_at(blockIdx.x, blockIdx.y, m, n, E, in, ldi, out, ldo, norms, rank, mode, off);
}

__device__ __forceinline__ void sigmas_at(int bx, int by, int n, const double* norms, const int* rank, double* sf, double* sg, double* sigma) {
  const int j = bx * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double nf = norms[j], ng = norms[n + j];
  const double th = 1.0 / sqrt(fma(nf, nf, ng * ng));
  sf[rank[j]] = nf * th;
  sg[rank[j]] = ng * th;
  sigma[rank[j]] = nf / ng;
}

__global__ void k_sigmas(int n, const double* norms, const int* rank, double* sf, double* sg, double* sigma) {
  sigmas_at(blockIdx.x, blockIdx.y, n, norms, rank, sf, sg, sigma);
}

__device__ __forceinline__ void copy_cols_at(int bx, int by, int m, int n, int E, const double* in, long long ldi, double* out, long long ldo) {
  const int j = bx * CW + (threadIdx.x >> 5);
  if (j >= n) return;
  const double* src = in + (size_t)j * E * ldi;
  double* dst = out + (size_t)j * E * ldo;
  for (int r = (threadIdx.x & 31); r < E * m; r += 32) dst[r] = src[r];
}

__global__ void k_copy_cols(int m, int n, int E, const double* in, long long ldi, double* out, long long ldo) {
  copy_cols_at(blockIdx.x, blockIdx.y, m, n, E, in, ldi, out, ldo);
}

__device__ __forceinline__ void to_f32_at(int bx, int by, int m, int n, int E, const double* src, long long lds, float* dst, long long ldd) {
  const int j = by;
  for (int r = bx * blockDim.x + threadIdx.x; r < E * m; r += gridDim.x * blockDim.x)
    dst[(size_t)j * E * ldd + r] = __double2float_rn(src[(size_t)j * E * lds + r]);
}

__global__ void k_to_f32(int m, int n, int E, const double* src, long long lds, float* dst, long long ldd) {
  to_f32_at(blockIdx.x, blockIdx.y, m, n, E, src, lds, dst, ldd);
}

template <class T>
__device__ __forceinline__ void identity_at(int bx, int by, int n, int E, T* Z, long long ldz) {
  const int j = by;
  for (int r = bx * blockDim.x + threadIdx.x; r < E * n; r += gridDim.x * blockDim.x)
    Z[(size_t)j * E * ldz + r] = (r == E * j) ? T(1) : T(0);
}

template <class T>
__global__ void k_identity(int n, int E, T* Z, long long ldz) {
  identity_at<T>(blockIdx.x, blockIdx.y, n, E, Z, ldz);
}

__device__ __forceinline__ void rowscale_at(int bx, int by, int n, int E, const double* zdiag, const float* Z32, long long ld32, double* Z,
                           long long ldz) {
  const int j = by;
  for (int r = bx * blockDim.x + threadIdx.x; r < E * n; r += gridDim.x * blockDim.x)
    Z[(size_t)j * E * ldz + r] = zdiag[r / E] * (double)Z32[(size_t)j * E * ld32 + r];
}

__global__ void k_rowscale(int n, int E, const double* zdiag, const float* Z32, long long ld32, double* Z,
                           long long ldz) {
  rowscale_at(blockIdx.x, blockIdx.y, n, E, zdiag, Z32, ld32, Z, ldz);
}

__device__ __forceinline__ void check_finite_at(int bx, int by, int m, int n, int E, const double* A, long long lda, int* flag) {
  const int j = by;
  bool bad = false;
  for (int r = bx * blockDim.x + threadIdx.x; r < E * m; r += gridDim.x * blockDim.x)
    bad |= !isfinite(A[(size_t)j * E * lda + r]);
  if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

__global__ void k_check_finite(int m, int n, int E, const double* A, long long lda, int* flag) {
  check_finite_at(blockIdx.x, blockIdx.y, m, n, E, A, lda, flag);
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
__device__ __forceinline__ void gemm_f64_at(int bx, int by, int m, int n, int kdim, const double* A, long long lda,
                                                  const float* B, long long ldb, double* C, long long ldc) {
  __shared__ double As[GK][GM + 8];  // As[k][r]
  __shared__ double Bs[GK][GN + 8];  // Bs[k][c]
  const int r0 = bx * GM, c0 = by * GN;
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

__global__ void __launch_bounds__(256) k_gemm_f64(int m, int n, int kdim, const double* A, long long lda,
                                                  const float* B, long long ldb, double* C, long long ldc) {
  gemm_f64_at(blockIdx.x, blockIdx.y, m, n, kdim, A, lda, B, ldb, C, ldc);
}

// complex C = A B via real views: A interleaved (re, im) of m x n; Re/Im
// planes of A and B are extracted by strided indexing in the real GEMM:
// Re C = Re A Re B - Im A Im B, Im C = Re A Im B + Im A Re B.
constexpr int GKC = 16;
__device__ __forceinline__ void gemm_c64_at(int bx, int by, int m, int n, const double* A, long long lda,
                                                  const float* B, long long ldb, double* C, long long ldc) {
  __shared__ double Ar[GKC][GM + 8], Ai[GKC][GM + 8];
  __shared__ double Br[GKC][GN + 8], Bi[GKC][GN + 8];
  const int r0 = bx * GM, c0 = by * GN;
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

__global__ void __launch_bounds__(256) k_gemm_c64(int m, int n, const double* A, long long lda,
                                                  const float* B, long long ldb, double* C, long long ldc) {
  gemm_c64_at(blockIdx.x, blockIdx.y, m, n, A, lda, B, ldb, C, ldc);
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

// ------------------------------------------------------ batched solves ----
// The column phases of gsvd_solve_batched's blocked problems, one launch each
// for the whole batch: grid z is the problem (grid x, y sized for the largest
// problem; blocks beyond a problem's size leave at once), and the per-problem
// bookkeeping of the sweep loop runs one thread per problem.  Every problem's
// arithmetic is the one-problem kernels' own (the same device functions).
namespace hz {

namespace {

__device__ __forceinline__ int bphase(int state) { return (state & BST_FP32) ? 0 : 1; }

// state and counters of every problem; the non-finite check of F and G;
// the prescale; the FP32 copies and Z_acc = I of the mixed path.  Problems
// with a non-finite entry are marked EINVAL and left untouched.
__global__ void k_b_init(BatchSweep* bs, int count, bool mixed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  BatchSweep z = {};
  z.state = mixed ? BST_FP32 : BST_FP64;
  bs[p] = z;
}
__global__ void k_b_check(const BatchCol* bc, BatchSweep* bs) {
  const BatchCol& q = bc[blockIdx.z];
  const int E = q.cplx ? 2 : 1;
  if ((int)blockIdx.y >= q.n) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && blockIdx.y == 0) {
    q.status[0] = 0;
    q.status[1] = 0;
  }
  __syncthreads();
  check_finite_at(blockIdx.x, blockIdx.y, q.mf, q.n, E, q.F, q.ldf, &bs[blockIdx.z].status);
  check_finite_at(blockIdx.x, blockIdx.y, q.mg, q.n, E, q.G, q.ldg, &bs[blockIdx.z].status);
}
__global__ void k_b_mark_invalid(BatchSweep* bs, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  if (bs[p].status != 0) {  // the check wrote 1: a non-finite entry
    bs[p].status = ST_EINVAL;
    bs[p].state = 0;
  }
}
__global__ void __launch_bounds__(256) k_b_prescale(const BatchCol* bc, const BatchSweep* bs) {
  const BatchCol& q = bc[blockIdx.z];
  if (bs[blockIdx.z].status == ST_EINVAL) return;
  prescale_at(blockIdx.x, 0, q.mf, q.mg, q.n, q.cplx ? 2 : 1, q.F, q.ldf, q.G, q.ldg, q.Z, q.ldz, q.zdiag,
              q.status);
}
__global__ void k_b_to_f32(const BatchCol* bc, const BatchSweep* bs) {
  const BatchCol& q = bc[blockIdx.z];
  if (bs[blockIdx.z].status == ST_EINVAL || (int)blockIdx.y >= q.n) return;
  const int E = q.cplx ? 2 : 1;
  to_f32_at(blockIdx.x, blockIdx.y, q.mf, q.n, E, q.F, q.ldf, q.F32, q.mf);
  to_f32_at(blockIdx.x, blockIdx.y, q.mg, q.n, E, q.G, q.ldg, q.G32, q.mg);
  identity_at<float>(blockIdx.x, blockIdx.y, q.n, E, q.Z32, q.n);
}

// Start of a global sweep: a problem whose last sweep hit the sweep cap
// leaves its phase now (after that sweep's rescale, as in the one-problem
// loop): the FP32 sweeps hand over to the FP64 ones, the FP64 sweeps end
// with ENOCONV; the counters of every sweeping problem are cleared.
__global__ void k_b_sweep_begin(const BatchCol* bc, BatchSweep* bs, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  if (bs[p].state & (BST_FP32 | BST_FP64))
    for (int k = 0; k < 8; ++k) bc[p].ctr[k] = 0ull;
}
// After the rescale: a problem whose sweep hit the sweep cap leaves its
// phase (as the one-problem loop does after that sweep's rescale): the FP32
// sweeps hand over to the FP64 ones, the FP64 sweeps end with ENOCONV.
__global__ void k_b_after_rescale(BatchSweep* bs, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  BatchSweep& t = bs[p];
  t.state &= ~BST_RESCALE;
  if (t.state & BST_CAP) {
    if (t.state & BST_FP32) {
      t.state = BST_RESTART;
    } else {
      t.state = 0;
      t.status = ST_ENOCONV;
    }
  }
}

// End of a global sweep: the convergence test of Sec. 2.5 for every problem
// that swept, with the same rules and order as the one-problem loop.
__global__ void k_b_sweep_end(const BatchCol* bc, BatchSweep* bs, BatchRule rule, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  BatchSweep& t = bs[p];
  if (!(t.state & (BST_FP32 | BST_FP64))) return;
  const unsigned long long* c = bc[p].ctr;
  const int ph = bphase(t.state);
  t.sweeps[ph] += 1;
  t.tall += c[0];
  t.tbig += c[1];
  t.chol_skipped += (int)c[3];
  t.visits += c[4];
  t.visits_applied += c[5];
  if (ph == 0) {
    t.visits32 += c[4];
    t.applied32 += c[5];
  }
  if (c[2]) {  // a pivot pair failed (rank-deficient G): ENOTPD, outputs still finalised
    t.status = ST_ENOTPD;
    t.state = ph == 0 ? BST_RESTART : 0;
    return;
  }
  if (c[1] == 0) {  // no big transformation: this phase has converged
    t.state = ph == 0 ? BST_RESTART : 0;
    return;
  }
  const double b2 = 2.0 * bc[p].w;
  const double examined = (double)c[4] * b2 * (b2 - 1.0) * 0.5 * (double)rule.inner_max32;
  if (ph == 0 && rule.stop_permille > 0 && (double)c[1] * 1000.0 < (double)rule.stop_permille * examined) {
    t.state = BST_RESTART;  // the FP32 sweeps hand over to the FP64 sweeps
    return;
  }
  t.state |= BST_RESCALE;
  if (t.sweeps[ph] >= rule.cap[ph]) t.state |= BST_CAP;
}

template <class T>
__global__ void __launch_bounds__(256) k_b_rescale(const BatchCol* bc, const BatchSweep* bs) {
  const BatchSweep& t = bs[blockIdx.z];
  if (!(t.state & BST_RESCALE)) return;
  const bool f32 = (t.state & BST_FP32) != 0;
  if (f32 != std::is_same<T, float>::value) return;
  const BatchCol& q = bc[blockIdx.z];
  const int E = q.cplx ? 2 : 1;
  if constexpr (std::is_same<T, float>::value)
    rescale_at<float>(blockIdx.x, 0, q.mf, q.mg, q.n, E, q.F32, q.mf, q.G32, q.mg, q.Z32, q.n);
  else
    rescale_at<double>(blockIdx.x, 0, q.mf, q.mg, q.n, E, q.F, q.ldf, q.G, q.ldg, q.Z, q.ldz);
}

// The restart of the mixed path after the FP32 sweeps: F <- F Z_acc,
// G <- G Z_acc (FP64 products into the work buffer, then copied back),
// Z <- Z0 Z_acc.
__global__ void __launch_bounds__(256) k_b_gemm_real(const BatchCol* bc, const BatchSweep* bs, int which) {
  const BatchCol& q = bc[blockIdx.z];
  if (!(bs[blockIdx.z].state & BST_RESTART) || q.cplx) return;
  const int m = which ? q.mg : q.mf;
  if ((int)blockIdx.x * GM >= m || (int)blockIdx.y * GN >= q.n) return;
  gemm_f64_at(blockIdx.x, blockIdx.y, m, q.n, q.n, which ? q.G : q.F, which ? q.ldg : q.ldf, q.Z32, q.n, q.work, m);
}
__global__ void __launch_bounds__(256) k_b_gemm_cplx(const BatchCol* bc, const BatchSweep* bs, int which) {
  const BatchCol& q = bc[blockIdx.z];
  if (!(bs[blockIdx.z].state & BST_RESTART) || !q.cplx) return;
  const int m = which ? q.mg : q.mf;
  if ((int)blockIdx.x * GM >= m || (int)blockIdx.y * GN >= q.n) return;
  gemm_c64_at(blockIdx.x, blockIdx.y, m, q.n, which ? q.G : q.F, which ? q.ldg : q.ldf, q.Z32, q.n, q.work, m);
}
__global__ void __launch_bounds__(256) k_b_copy_back(const BatchCol* bc, const BatchSweep* bs, int which) {
  const BatchCol& q = bc[blockIdx.z];
  if (!(bs[blockIdx.z].state & BST_RESTART)) return;
  const int m = which ? q.mg : q.mf;
  copy_cols_at(blockIdx.x, 0, m, q.n, q.cplx ? 2 : 1, q.work, m, which ? q.G : q.F, which ? q.ldg : q.ldf);
}
__global__ void k_b_restart_z(const BatchCol* bc, BatchSweep* bs) {
  const BatchCol& q = bc[blockIdx.z];
  if (!(bs[blockIdx.z].state & BST_RESTART) || (int)blockIdx.y >= q.n) return;
  rowscale_at(blockIdx.x, blockIdx.y, q.n, q.cplx ? 2 : 1, q.zdiag, q.Z32, q.n, q.Z, q.ldz);
}
__global__ void k_b_restart_done(BatchSweep* bs, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count || !(bs[p].state & BST_RESTART)) return;
  bs[p].state = bs[p].status == 0 ? BST_FP64 : 0;  // a failed or stopped problem skips the FP64 sweeps
}

// a deadline: every problem still sweeping stops with this status (FP32
// sweeps still go through the restart, so that the outputs are FP64 results)
__global__ void k_b_stop(BatchSweep* bs, int count, int status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  BatchSweep& t = bs[p];
  if (!(t.state & (BST_FP32 | BST_FP64 | BST_RESTART))) return;
  if (t.status == 0) t.status = status;
  t.state = (t.state & (BST_FP32 | BST_RESTART)) ? BST_RESTART : 0;
}

// the final rescaling and sort of Sec. 2.4 / Sec. 1 for every problem that
// was not refused (EINVAL), then its final status
__global__ void __launch_bounds__(256) k_b_norms(const BatchCol* bc, const BatchSweep* bs) {
  const BatchCol& q = bc[blockIdx.z];
  if (bs[blockIdx.z].status == ST_EINVAL) return;
  norms_at(blockIdx.x, 0, q.mf, q.mg, q.n, q.cplx ? 2 : 1, q.F, q.ldf, q.G, q.ldg, q.norms, q.status);
}
__global__ void k_b_rank(const BatchCol* bc, const BatchSweep* bs) {
  const BatchCol& q = bc[blockIdx.z];
  if (bs[blockIdx.z].status == ST_EINVAL) return;
  rank_at(blockIdx.x, 0, q.n, q.norms, q.rank);
}
// which: 0 = U from F, 1 = V from G, 2 = Z; gather into the work buffer
__global__ void __launch_bounds__(256) k_b_gather(const BatchCol* bc, const BatchSweep* bs, int which) {
  const BatchCol& q = bc[blockIdx.z];
  if (bs[blockIdx.z].status == ST_EINVAL) return;
  const int E = q.cplx ? 2 : 1;
  if (which == 0) gather_at(blockIdx.x, 0, q.mf, q.n, E, q.F, q.ldf, q.work, q.mf, q.norms, q.rank, 0, 0);
  else if (which == 1) gather_at(blockIdx.x, 0, q.mg, q.n, E, q.G, q.ldg, q.work, q.mg, q.norms, q.rank, 0, q.n);
  else gather_at(blockIdx.x, 0, q.n, q.n, E, q.Z, q.ldz, q.work, q.n, q.norms, q.rank, 1, 0);
}
__global__ void __launch_bounds__(256) k_b_scatter(const BatchCol* bc, const BatchSweep* bs, int which) {
  const BatchCol& q = bc[blockIdx.z];
  if (bs[blockIdx.z].status == ST_EINVAL) return;
  const int E = q.cplx ? 2 : 1;
  if (which == 0) copy_cols_at(blockIdx.x, 0, q.mf, q.n, E, q.work, q.mf, q.F, q.ldf);
  else if (which == 1) copy_cols_at(blockIdx.x, 0, q.mg, q.n, E, q.work, q.mg, q.G, q.ldg);
  else copy_cols_at(blockIdx.x, 0, q.n, q.n, E, q.work, q.n, q.Z, q.ldz);
}
__global__ void k_b_sigmas(const BatchCol* bc, BatchSweep* bs) {
  const BatchCol& q = bc[blockIdx.z];
  if (bs[blockIdx.z].status == ST_EINVAL) return;
  sigmas_at(blockIdx.x, 0, q.n, q.norms, q.rank, q.sf, q.sg, q.sigma);
}
__global__ void k_b_final_status(const BatchCol* bc, BatchSweep* bs, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  if (bs[p].status == 0 && bc[p].status[0] != 0) bs[p].status = bc[p].status[0];
}

inline int pgrid(int count) { return (count + 127) / 128; }

}  // namespace

cudaError_t launch_batch_init(const BatchCol* bc, BatchSweep* bs, int count, int maxm, int maxn, bool mixed,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_b_init<<<pgrid(count), 128, 0, s>>>(bs, count, mixed);
  const int gx = std::min(64, (2 * maxm + 255) / 256);
  k_b_check<<<dim3(gx, maxn, count), 256, 0, s>>>(bc, bs);
  k_b_mark_invalid<<<pgrid(count), 128, 0, s>>>(bs, count);
  k_b_prescale<<<dim3(cgrid(maxn), 1, count), 32 * CW, 0, s>>>(bc, bs);
  if (mixed) k_b_to_f32<<<dim3(gx, maxn, count), 256, 0, s>>>(bc, bs);
  return cudaGetLastError();
}

cudaError_t launch_batch_sweep_begin(const BatchCol* bc, BatchSweep* bs, int count, cudaStream_t s) {
  k_b_sweep_begin<<<pgrid(count), 128, 0, s>>>(bc, bs, count);
  return cudaGetLastError();
}

cudaError_t launch_batch_sweep_end(const BatchCol* bc, BatchSweep* bs, const BatchRule& rule, int count,
                                   cudaStream_t s) {
  k_b_sweep_end<<<pgrid(count), 128, 0, s>>>(bc, bs, rule, count);
  return cudaGetLastError();
}

cudaError_t launch_batch_rescale(const BatchCol* bc, BatchSweep* bs, int count, int maxn, cudaStream_t s) {
  k_b_rescale<float><<<dim3(cgrid(maxn), 1, count), 32 * CW, 0, s>>>(bc, bs);
  k_b_rescale<double><<<dim3(cgrid(maxn), 1, count), 32 * CW, 0, s>>>(bc, bs);
  k_b_after_rescale<<<pgrid(count), 128, 0, s>>>(bs, count);
  return cudaGetLastError();
}

cudaError_t launch_batch_restart(const BatchCol* bc, BatchSweep* bs, int count, int maxm, int maxn, cudaStream_t s) {
  const dim3 gg((maxm + GM - 1) / GM, (maxn + GN - 1) / GN, count);
  for (int which = 0; which < 2; ++which) {
    k_b_gemm_real<<<gg, 256, 0, s>>>(bc, bs, which);
    k_b_gemm_cplx<<<gg, 256, 0, s>>>(bc, bs, which);
    k_b_copy_back<<<dim3(cgrid(maxn), 1, count), 32 * CW, 0, s>>>(bc, bs, which);
  }
  k_b_restart_z<<<dim3((2 * maxn + 255) / 256, maxn, count), 256, 0, s>>>(bc, bs);
  k_b_restart_done<<<pgrid(count), 128, 0, s>>>(bs, count);
  return cudaGetLastError();
}

cudaError_t launch_batch_stop(BatchSweep* bs, int count, int status, cudaStream_t s) {
  k_b_stop<<<pgrid(count), 128, 0, s>>>(bs, count, status);
  return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchCol* bc, BatchSweep* bs, int count, int maxm, int maxn,
                                  cudaStream_t s) {
  (void)maxm;
  const dim3 gc(cgrid(maxn), 1, count);
  k_b_norms<<<gc, 32 * CW, 0, s>>>(bc, bs);
  k_b_rank<<<dim3((maxn + 127) / 128, 1, count), 128, 0, s>>>(bc, bs);
  for (int which = 0; which < 3; ++which) {
    k_b_gather<<<gc, 32 * CW, 0, s>>>(bc, bs, which);
    k_b_scatter<<<gc, 32 * CW, 0, s>>>(bc, bs, which);
  }
  k_b_sigmas<<<dim3((maxn + 127) / 128, 1, count), 128, 0, s>>>(bc, bs);
  k_b_final_status<<<pgrid(count), 128, 0, s>>>(bc, bs, count);
  return cudaGetLastError();
}

}  // namespace hz
