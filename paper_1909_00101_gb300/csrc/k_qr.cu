// k_qr.cu -- the QR shortening of Sec. 2 of arXiv 1909.00101 (F = Q_F R_F,
// G = Q_G R_G; the Hari-Zimmermann sweeps then run on the n x n factors
// (R_F, R_G), which have the same Grams F^T F = R_F^T R_F, G^T G = R_G^T R_G,
// so the iteration is the same while every sweep touches n instead of m rows;
// finally U = Q_F U'', V = Q_G V'').
//
// The QR is CholeskyQR2 (R1 = chol(F^T F), Q1 = F R1^{-1}, R2 = chol(Q1^T Q1),
// Q = Q1 R2^{-1}, R = R2 R1) built from FP64 kernels: a DMMA GEMM, a blocked
// right-looking Cholesky (one-CTA diagonal blocks, row-panel triangular
// solves, GEMM trailing updates) and a blocked right triangular solve with
// row-wise substitution (backward stable per row); the large products run on
// the BF16 tensor cores with FP64 accuracy (k_ozaki.cu) when the caller
// gives a workspace for the digit planes.  It is accurate for
// cond(F) up to about 1e8; the caller skips the shortening when the first
// Cholesky of either Gram fails.  Real data only.
#include <algorithm>

#include "hz_device.cuh"
#include "hz_kernels.h"

namespace hz {

namespace {

constexpr int QB = 32;  // block size of the Cholesky and the triangular solves

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// C (M x N) = alpha op(A) op(B) + beta C, column-major; op(A) is M x K, op(B)
// is K x N.  64 x 64 output tiles, K in chunks of 16, DMMA m8n8k4: warp w owns
// rows [8w, 8w + 8) of the tile.  upper = 1: only tiles that meet the upper
// triangle (the caller uses only C's upper triangle); upper = 2: besides,
// op(A) and op(B) are upper triangular, so tile (r0, c0) sums k in
// [r0, c0 + DN) only.
constexpr int DM = 64, DN = 64, DK = 16;
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double* __restrict__ A,
                                               long long lda, const double* __restrict__ B, long long ldb,
                                               double beta, double* __restrict__ C, long long ldc, int upper) {
  __shared__ double As[DK][DM + 8];  // As[k][i] = op(A)[i][k]
  __shared__ double Bs[DK][DN + 8];  // Bs[k][j] = op(B)[k][j]
  const int r0 = blockIdx.x * DM, c0 = blockIdx.y * DN;
  if (upper && r0 >= c0 + DN) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[8][2];
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t][0] = acc[t][1] = 0.0;
  const int kend = upper == 2 ? min(K, c0 + DN) : K;
  for (int k0 = upper == 2 ? r0 : 0; k0 < kend; k0 += DK) {
    for (int idx = threadIdx.x; idx < DK * DM; idx += blockDim.x) {
      int i, k;
      if (TA) { i = idx / DK; k = idx % DK; } else { k = idx / DM; i = idx % DM; }
      double v = 0.0;
      if (r0 + i < M && k0 + k < K) v = TA ? A[(size_t)(r0 + i) * lda + k0 + k] : A[(size_t)(k0 + k) * lda + r0 + i];
      As[k][i] = v;
    }
    for (int idx = threadIdx.x; idx < DK * DN; idx += blockDim.x) {
      int j, k;
      if (TB) { k = idx / DN; j = idx % DN; } else { j = idx / DK; k = idx % DK; }
      double v = 0.0;
      if (c0 + j < N && k0 + k < K) v = TB ? B[(size_t)(k0 + k) * ldb + c0 + j] : B[(size_t)(c0 + j) * ldb + k0 + k];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DK; kk += 4) {
      const double a = As[kk + (lane & 3)][warp * 8 + (lane >> 2)];
#pragma unroll
      for (int t = 0; t < 8; ++t) dmma(acc[t][0], acc[t][1], a, Bs[kk + (lane & 3)][t * 8 + (lane >> 2)]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = r0 + warp * 8 + (lane >> 2);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = c0 + t * 8 + 2 * (lane & 3) + e;
      if (r < M && c < N) {
        double* p = C + (size_t)c * ldc + r;
        *p = beta == 0.0 ? alpha * acc[t][e] : fma(alpha, acc[t][e], beta * *p);
      }
    }
  }
}

// Cholesky of one nb x nb diagonal block in place (upper R, A = R^T R); a
// non-positive pivot sets *fail.
__global__ void __launch_bounds__(256) k_potrf_diag(int nb, double* A, long long lda, int* fail) {
  __shared__ double S[QB][QB + 1];  // S[j][i] = A(i, j)
  __shared__ double s_inv;
  __shared__ int s_bad;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) S[idx / nb][idx % nb] = A[(size_t)(idx / nb) * lda + idx % nb];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      const double d = S[k][k];
      if (!(d > 0.0) || !isfinite(d)) {
        s_bad = 1;
        s_inv = 0.0;
      } else {
        const double r = sqrt(d);
        S[k][k] = r;
        s_inv = 1.0 / r;
      }
    }
    __syncthreads();
    if (s_bad) break;
    for (int j = k + 1 + threadIdx.x; j < nb; j += blockDim.x) S[j][k] *= s_inv;  // row k of R
    __syncthreads();
    const int rem = nb - k - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      const int j = k + 1 + idx / rem, i = k + 1 + idx % rem;
      if (i <= j) S[j][i] = fma(-S[i][k], S[j][k], S[j][i]);
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicExch(fail, 1);
    return;
  }
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int j = idx / nb, i = idx % nb;
    A[(size_t)j * lda + i] = (i <= j) ? S[j][i] : 0.0;
  }
}

// X = R^{-T} B in place (R nb x nb upper at R, B nb x ncols): R^T x = b per
// column, forward substitution, one thread per column.
__global__ void k_trsm_lt(int nb, int ncols, const double* __restrict__ R, long long ldr, double* B, long long ldb) {
  __shared__ double S[QB][QB + 1];  // S[j][i] = R(i, j)
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) S[idx / nb][idx % nb] = R[(size_t)(idx / nb) * ldr + idx % nb];
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double* b = B + (size_t)c * ldb;
  double x[QB];
  for (int i = 0; i < nb; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s = fma(-S[i][k], x[k], s);  // R(k, i) x_k
    x[i] = s / S[i][i];
  }
  for (int i = 0; i < nb; ++i) b[i] = x[i];
}

// X = B R^{-1} in place (B m x nb, R nb x nb upper): x R = b per row, forward
// substitution along the columns, one thread per row.
__global__ void k_trsm_ru(int m, int nb, const double* __restrict__ R, long long ldr, double* B, long long ldb) {
  __shared__ double S[QB][QB + 1];  // S[j][i] = R(i, j)
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) S[idx / nb][idx % nb] = R[(size_t)(idx / nb) * ldr + idx % nb];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double x[QB];
  for (int j = 0; j < nb; ++j) {
    double s = B[(size_t)j * ldb + r];
    for (int k = 0; k < j; ++k) s = fma(-x[k], S[j][k], s);  // x_k R(k, j)
    x[j] = s / S[j][j];
  }
  for (int j = 0; j < nb; ++j) B[(size_t)j * ldb + r] = x[j];
}

__global__ void k_zero_lower(int n, double* A, long long lda) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (i > j) A[(size_t)j * lda + i] = 0.0;
}

thread_local long long t_launches = 0;  // kernels launched by this thread's QR calls

}  // namespace

long long qr_launch_count() { return t_launches; }

cudaError_t dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long long lda,
                  const double* B, long long ldb, double beta, double* C, long long ldc, int upper,
                  cudaStream_t s, const OzWs* oz) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  // large products on the tensor cores (FP64 accuracy), small ones on DMMA.
  // The sliced product bounds an entry's error by the largest |value| of its
  // row of op(A) times that of its column of op(B); every product here has
  // an op(A) with columns of one scale (Q, or F^T's rows as F's columns),
  // except the triangular R2 R1 (upper = 2), which stays on DMMA.
  if (oz && oz->p && upper != 2 && (double)M * N * K >= OZ_GEMM_MIN &&
      oz->bytes >= dgemm_oz_ws_bytes(M, N, std::min(K, OZ_K_MAX))) {
    // K in pieces of at most OZ_K_MAX (the longest exact level sum); each
    // piece is rounded once and added to C
    for (int k0 = 0; k0 < K; k0 += OZ_K_MAX) {
      const int kc = std::min(OZ_K_MAX, K - k0);
      const double* Ak = A + (ta ? (size_t)k0 : (size_t)k0 * lda);  // op(A)(:, k0 :)
      const double* Bk = B + (tb ? (size_t)k0 * ldb : (size_t)k0);  // op(B)(k0 :, :)
      const bool same = ta && !tb && Ak == Bk && lda == ldb && M == N;
      t_launches += same ? 2 : 3;
      const cudaError_t e = dgemm_oz(ta, tb, M, N, kc, alpha, Ak, lda, Bk, ldb, k0 ? 1.0 : beta, C, ldc, upper,
                                     oz->p, oz->bytes, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  dim3 grid((M + DM - 1) / DM, (N + DN - 1) / DN);
  ++t_launches;
  if (ta && !tb)
    k_dgemm<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, upper);
  else if (!ta && !tb)
    k_dgemm<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, upper);
  else if (!ta && tb)
    k_dgemm<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, upper);
  else
    k_dgemm<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, upper);
  return cudaGetLastError();
}

// Blocked Cholesky A = R^T R in place (upper), strict lower part zeroed.
cudaError_t potrf_upper(int n, double* A, long long lda, int* fail, cudaStream_t s, const OzWs* oz) {
  for (int k0 = 0; k0 < n; k0 += QB) {
    const int nb = std::min(QB, n - k0);
    double* Akk = A + (size_t)k0 * lda + k0;
    k_potrf_diag<<<1, 256, 0, s>>>(nb, Akk, lda, fail);
    ++t_launches;
    const int rest = n - k0 - nb;
    if (rest > 0) {
      ++t_launches;
      double* Akr = A + (size_t)(k0 + nb) * lda + k0;  // nb x rest block right of the diagonal
      k_trsm_lt<<<(rest + 127) / 128, 128, 0, s>>>(nb, rest, Akk, lda, Akr, lda);
      double* Arr = A + (size_t)(k0 + nb) * lda + k0 + nb;
      cudaError_t e = dgemm(true, false, rest, rest, nb, -1.0, Akr, lda, Akr, lda, 1.0, Arr, lda, true, s, oz);
      if (e != cudaSuccess) return e;
    }
  }
  k_zero_lower<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, A, lda);
  ++t_launches;
  return cudaGetLastError();
}

cudaError_t launch_zero_lower(int n, double* A, long long lda, cudaStream_t s) {
  k_zero_lower<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, A, lda);
  ++t_launches;
  return cudaGetLastError();
}

// B (m x n) <- B R^{-1}, R n x n upper: recursive halving (B1 R11^{-1}, then
// B2 -= B1 R12, then B2 R22^{-1}) down to column blocks of QB, which the
// row-wise substitution kernel solves; the bulk of the work is in the GEMMs.
cudaError_t trsm_right_upper(int m, int n, const double* R, long long ldr, double* B, long long ldb, cudaStream_t s,
                             const OzWs* oz) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (n <= QB) {
    k_trsm_ru<<<(m + 127) / 128, 128, 0, s>>>(m, n, R, ldr, B, ldb);
    ++t_launches;
    return cudaGetLastError();
  }
  const int n1 = ((n / 2 + QB - 1) / QB) * QB;
  cudaError_t e = trsm_right_upper(m, n1, R, ldr, B, ldb, s, oz);
  if (e != cudaSuccess) return e;
  double* B2 = B + (size_t)n1 * ldb;
  e = dgemm(false, false, m, n - n1, n1, -1.0, B, ldb, R + (size_t)n1 * ldr, ldr, 1.0, B2, ldb, false, s, oz);
  if (e != cudaSuccess) return e;
  return trsm_right_upper(m, n - n1, R + (size_t)n1 * ldr + n1, ldr, B2, ldb, s, oz);
}

}  // namespace hz
