// hz_kernels.h -- internal interface between the host runtime (gsvd_api.cu)
// and the CUDA kernels.  Not part of the public C ABI (include/gsvd.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace hz {

// ---------------------------------------------------------- pointwise ----
struct PwStats {
  int32_t status;
  int32_t sweeps;
  long long transf_all;
  long long transf_big;
};

struct PwProblem {
  void* F;
  long long ldf;
  void* G;
  long long ldg;
  void* Z;
  long long ldz;
  int mf, mg, n, pad;
  double* sigma_f;
  double* sigma_g;
  double* sigma;
  PwStats* stats;
};

struct PwParams {
  double eps;
  int max_sweeps;
  bool sort;
  bool f32cls;
  bool crit2;
  bool rowcyc;  // row-cyclic wavefront order (else round robin)
  // variants of Sec. 2.6 (Table "Variants"), besides crit2 (C2):
  bool enhanced = false;  // App. A enhanced dot products (variants 1, 3, 5, 7)
  bool dscale = false;    // no prescaling; each pivot pair rescaled by D-hat (variants 2, 3, 6, 7)
};

size_t pointwise_smem_bytes(int mf, int mg, int n, bool cplx, bool fp32, int slots);
// largest dynamic shared memory of a pointwise launch: the 227 KB one CTA may
// use, less room for the kernel's static shared arrays (512 B in the real one)
constexpr size_t POINTWISE_SMEM_MAX = 227 * 1024 - 1024;
// slots: the largest number of pairs per step over the batch (shared-memory layout)
cudaError_t launch_pointwise(const PwProblem* d_probs, int count, int slots, bool cplx, bool fp32, size_t smem,
                             const PwParams& prm, cudaStream_t stream);

// ------------------------------------------------------------ blocked ----
// One solve (or one member of a batch) on the blocked path.  Matrices are
// column-major; complex data interleaved (re, im).  T is double (FP64 sweeps)
// or float (FP32 bulk sweeps of the mixed-precision path).
struct BlkDims {
  int mf, mg, n;
  int w;        // block width; block k covers columns [k w, min((k+1) w, n))
  int nblk;     // N = ceil(n / w)
  int nslots;   // pairs per outer step = N_eff / 2 (N_eff = N rounded up to even)
  int rf, rg;   // row splits of the Gram over F and G
  int trows;    // rows per Gram row split are a multiple of this
};

struct BlkBuffers {
  void* F;
  long long ldf;
  void* G;
  long long ldg;
  void* Z;
  long long ldz;
  void* partial;              // [nslots][rf+rg][V][V] of T
  void* ztil;                 // [nslots][V][V] of T (real view of Z-tilde)
  int* flags;                 // [nslots]: 1 = apply needed
  unsigned long long* ctr;    // [0] all, [1] big, [2] failures (ENOTPD), [3] chol failures skipped,
                              // [4] visits, [5] visits applied
  const uint16_t* table;      // outer table [N_eff - 1][nslots][2]
};

struct InnerParams {
  double eps;          // unit roundoff of the sweep's data type
  double tol;          // > 0: skip-test threshold to use instead of eps * sqrt(columns)
  int inner_max;       // inner sweeps cap (30 = FB, 1 = BO)
  bool sort;
  bool f32cls;         // classify small/big at FP32 resolution
  bool crit2;
  bool chol_skip;      // Cholesky failure: skip the visit (FP32 bulk) instead of failing
  bool par32;          // FP32 bulk sweeps: 2x2 parameters in FP32 (else FP64)
  bool enhanced = false;  // FP64 sweeps, variants +1: the enhanced dot products of App. A
  bool dscale = false;    // FP64 sweeps, variants +2: no inner prescale, each pivot pair rescaled by D-hat
};

// Batched sweeps (gsvd_solve_batched): many blocked problems advance one
// outer step per launch.  Grid x enumerates (problem, pair slot) items of all
// problems of a group (same data type and real-view width V); each CTA loads
// its problem's dimensions, buffers and pivot-step parameters from the device
// table and leaves at once when its problem is not sweeping in this phase or
// has fewer outer steps per sweep than the step being run.  Every problem's
// arithmetic is the one-problem kernels' own.
// Progress of one problem of a batched solve (device, read by the host after
// every global sweep).  State bits: sweeping in the FP32 bulk or the FP64
// phase, waiting for the restart of the mixed path (F <- F Z_acc ...), a
// rescale due before the next sweep, the sweep cap reached.
enum : int { BST_FP32 = 1, BST_FP64 = 2, BST_RESTART = 4, BST_RESCALE = 8, BST_CAP = 16 };
struct BatchSweep {
  int state;                   // BST_* bits; 0 = finished
  int status;
  int sweeps[2];               // FP32 bulk and FP64 sweeps done
  int chol_skipped, pad;
  unsigned long long tall, tbig, visits, visits_applied, visits32, applied32;
};
struct BlkProb {
  BlkDims d[2];         // [0] FP32 bulk sweeps, [1] FP64 sweeps
  BlkBuffers b[2];
  InnerParams ip[2];
  int steps;            // outer steps per sweep
  int tiles;            // row tiles of the apply over F, G and Z
};
struct BlkBatch {
  const BlkProb* probs = nullptr;  // device table; nullptr: one problem, given by value
  const int2* items = nullptr;     // device: (problem, slot) of each grid-x index
  const BatchSweep* sweep = nullptr;  // device: per problem, bit `phase` of its state set while it sweeps in that phase
  int phase = 0;                   // 0 = FP32 bulk sweeps, 1 = FP64 sweeps
};

// Column data of one problem of a batched solve (device table): the caller's
// FP64 data and outputs, the FP32 copies of the mixed-precision path and the
// problem's workspace.
struct BatchCol {
  int mf, mg, n, cplx, w;
  double* F;
  long long ldf;
  double* G;
  long long ldg;
  double* Z;
  long long ldz;
  double *sf, *sg, *sigma;
  float *F32, *G32, *Z32;      // mixed precision (ld = mf, mg, n)
  double* zdiag;
  double* norms;
  int* rank;
  double* work;
  int* status;                 // [0]: device-side status of the solve, [1]: non-finite input
  unsigned long long* ctr;     // the sweep counters of the blocked kernels
};
// Rules of a batched solve (the handle's configuration).
struct BatchRule {
  int cap[2];                  // sweep caps of the FP32 bulk and the FP64 sweeps
  int stop_permille;           // FP32 -> FP64 hand-over threshold (0 = off)
  int inner_max32;             // inner sweeps per visit in the FP32 sweeps
};
// One launch each; grid z (or one thread) per problem of the batch.
cudaError_t launch_batch_init(const BatchCol* bc, BatchSweep* bs, int count, int maxm, int maxn, bool mixed,
                              cudaStream_t s);
cudaError_t launch_batch_sweep_begin(const BatchCol* bc, BatchSweep* bs, int count, cudaStream_t s);
cudaError_t launch_batch_sweep_end(const BatchCol* bc, BatchSweep* bs, const BatchRule& rule, int count,
                                   cudaStream_t s);
cudaError_t launch_batch_rescale(const BatchCol* bc, BatchSweep* bs, int count, int maxn, cudaStream_t s);
cudaError_t launch_batch_restart(const BatchCol* bc, BatchSweep* bs, int count, int maxm, int maxn, cudaStream_t s);
cudaError_t launch_batch_stop(BatchSweep* bs, int count, int status, cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchCol* bc, BatchSweep* bs, int count, int maxm, int maxn,
                                  cudaStream_t s);

int blk_vmax(int w, bool cplx);  // real-view width V of the kernels for this w
// the variants of Sec. 2.6 run in the FP64 pivot step of width V (the two-CTA kernel)
bool inner_variants_supported(int V);
cudaError_t launch_gram(const BlkDims& d, const BlkBuffers& b, bool cplx, bool fp32, int step,
                        cudaStream_t s, const BlkBatch* bt = nullptr, int nitems = 0, int grid_y = 0);
cudaError_t launch_inner(const BlkDims& d, const BlkBuffers& b, bool cplx, bool fp32, int step,
                         const InnerParams& p, cudaStream_t s, const BlkBatch* bt = nullptr, int nitems = 0);
cudaError_t launch_apply(const BlkDims& d, const BlkBuffers& b, bool cplx, bool fp32, int step,
                         cudaStream_t s, const BlkBatch* bt = nullptr, int nitems = 0, int grid_y = 0);
// FP64 Gram and apply on the BF16 tensor cores with FP64 accuracy (sliced
// operands, exact level sums); real-view widths V = 16 and 32
bool oz_supported(int V);
cudaError_t launch_gram_oz(const BlkDims& d, const BlkBuffers& b, bool cplx, int step, cudaStream_t s,
                           const BlkBatch* bt = nullptr, int nitems = 0, int grid_y = 0);
// tc: issue the level products as tcgen05.mma with TMEM accumulators (else mma.sync)
cudaError_t launch_apply_oz(const BlkDims& d, const BlkBuffers& b, bool cplx, int step, cudaStream_t s, bool tc,
                            const BlkBatch* bt = nullptr, int nitems = 0, int grid_y = 0);

// -------------------------------------------------- column operations ----
// prescale: z_j = 1/||g_j||, F <- F Z0, G <- G Z0, Z <- Z0 (FP64, in place)
cudaError_t launch_prescale(int mf, int mg, int n, bool cplx, double* F, long long ldf, double* G,
                            long long ldg, double* Z, long long ldz, double* zdiag, int* status,
                            cudaStream_t s);
// between sweeps: f_j, g_j, z_j *= (||f_j||^2 + ||g_j||^2)^{-1/2} (T = double or float)
cudaError_t launch_rescale(int mf, int mg, int n, bool cplx, bool fp32, void* F, long long ldf, void* G,
                           long long ldg, void* Z, long long ldz, cudaStream_t s);
// final: norms, Theta, Sigma, rank sort, gather into U, V, Z (work: scratch of
// max(mf, mg, n) * n elements), sigma vectors.
cudaError_t launch_finalize(int mf, int mg, int n, bool cplx, double* F, long long ldf, double* G,
                            long long ldg, double* Z, long long ldz, double* sf, double* sg,
                            double* sigma, double* norms, int* rank, double* work, int* status,
                            cudaStream_t s);
// conversions for the mixed-precision path
cudaError_t launch_to_f32(int m, int n, bool cplx, const double* src, long long lds, float* dst,
                          long long ldd, cudaStream_t s);
cudaError_t launch_identity(int n, bool cplx, bool fp32, void* Z, long long ldz, cudaStream_t s);
// C (m x n) = A (m x n, FP64) * B (n x n, FP32 widened to FP64), dst may not alias A.
cudaError_t launch_gemm_f64_by_f32(int m, int n, bool cplx, const double* A, long long lda,
                                   const float* B, long long ldb, double* C, long long ldc,
                                   cudaStream_t s);
// A (rows x n, column-major) <- deterministic pseudo-random values in [-1, 1)
cudaError_t launch_fill_hash(int rows, int n, unsigned seed, double* A, long long lda, cudaStream_t s);
// X(i, j) <- sf_i X(i, j) + sg_i T(i, j) (n x n): the right vectors from
// U^T F (in X) and V^T G (in T)
cudaError_t launch_rows_combine(int n, bool cplx, double* X, long long ldx, const double* sf, const double* T,
                                long long ldt, const double* sg, cudaStream_t s);
// C = A^H B, complex interleaved (right vectors of complex problems)
cudaError_t launch_gemm_ch(int m, int k, int n, const double* A, long long lda, const double* B, long long ldb,
                           double* C, long long ldc, cudaStream_t s);
// Z64 = diag(zdiag) * Z32 (rows scaled), FP64 result
cudaError_t launch_rowscale(int n, bool cplx, const double* zdiag, const float* Z32, long long ld32,
                            double* Z, long long ldz, cudaStream_t s);
// workspace of the tensor-core products (digit planes); products with
// M N K >= OZ_GEMM_MIN run there when it is large enough
struct OzWs {
  void* p;
  size_t bytes;
};
constexpr double OZ_GEMM_MIN = 1073741824.0;  // 2^30
// Longest sum of slice products (rows of a Gram, K of a product) that one
// accumulation may cover.  A level of seven digit products adds below
// 7 * 2^16 per row; after K rows the FP32 high word holds below 7 * 2^16 K
// and the low word, which collects a TwoSum error below 2^-24 of the high
// word every 32 rows, below 7 K^2 / 2^13.  K <= 2^16 keeps the low word
// under 2^22, so both words stay exact integers.
constexpr int OZ_K_MAX = 65536;
// FP64 GEMM: C = alpha op(A) op(B) + beta C (column-major); upper = 1:
// only tiles meeting C's upper triangle are computed; upper = 2: also op(A)
// and op(B) are upper triangular (square), so each tile sums its k range only
cudaError_t dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long long lda,
                  const double* B, long long ldb, double beta, double* C, long long ldc, int upper,
                  cudaStream_t s, const OzWs* oz = nullptr);
// kernels launched so far by the calling thread's dgemm/potrf/trsm calls
long long qr_launch_count();
// the same product on the BF16 tensor cores with FP64 accuracy (operands
// sliced once into digit planes in ws); cudaErrorInvalidValue if ws is
// smaller than dgemm_oz_ws_bytes(M, N, K) or K > OZ_K_MAX (dgemm cuts a
// longer K into pieces)
size_t dgemm_oz_ws_bytes(int M, int N, int K);
cudaError_t dgemm_oz(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long long lda,
                     const double* B, long long ldb, double beta, double* C, long long ldc, int upper, void* ws,
                     size_t ws_bytes, cudaStream_t s);
// zero the strict lower triangle of an n x n matrix
cudaError_t launch_zero_lower(int n, double* A, long long lda, cudaStream_t s);
// blocked Cholesky A = R^T R in place (upper), *fail = 1 on a non-positive pivot
cudaError_t potrf_upper(int n, double* A, long long lda, int* fail, cudaStream_t s, const OzWs* oz = nullptr);
// B (m x n) <- B R^{-1} for upper triangular R (n x n)
cudaError_t trsm_right_upper(int m, int n, const double* R, long long ldr, double* B, long long ldb, cudaStream_t s,
                             const OzWs* oz = nullptr);
// non-finite check of a column-major matrix: sets *flag = 1 on NaN/Inf
cudaError_t launch_check_finite(int m, int n, bool cplx, const double* A, long long lda, int* flag,
                                cudaStream_t s);

}  // namespace hz
