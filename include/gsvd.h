/*
 * gsvd.h -- C ABI of the GB300 implicit Hari-Zimmermann GSVD engine.
 *
 * Computes the generalized singular value decomposition of a full-column-rank
 * pair (F, G), F of m_F x n and G of m_G x n, real or complex, by the one-sided
 * implicit Hari-Zimmermann method (Novakovic & Singer, "Implicit
 * Hari-Zimmermann algorithm for the generalized SVD on the GPUs",
 * arXiv 1909.00101):
 *
 *     F Z = U Sigma_F,   G Z = V Sigma_G,   U^* U = V^* V = I,
 *     Sigma_F^2 + Sigma_G^2 = I,   Sigma = Sigma_G^{-1} Sigma_F sorted descending
 *
 * (Sec. 1 of the paper; the sweep loop of Sec. 2.2-2.5 runs on one GPU).
 *
 * Memory: every matrix is column-major with a leading dimension (in elements).
 * Real data is double; complex data is interleaved (re, im) doubles, the layout
 * of C99 double _Complex and of numpy/torch complex128.  F is overwritten by U
 * and G by V (in place, as in Sec. 3.1.1); Z (n x n) and the three length-n
 * vectors are outputs.  Pointers may be device pointers of the current device
 * (the solve runs in place) or host pointers (pageable or pinned: the library
 * copies in and out through its own device buffers); one problem must not mix
 * the two, and memory of another device is GSVD_EINVAL.
 *
 * Ownership: the caller owns every buffer passed in a gsvd_problem; the
 * library owns the handle, its stream use, device workspace and the serving
 * thread.  Buffers given to gsvd_submit must stay valid and untouched until
 * gsvd_poll returns a terminal status for that ticket.
 *
 * Errors: every function returns an int status (GSVD_OK = 0, negative =
 * error, GSVD_EAGAIN = 1 is "not yet").  Argument errors are detected before
 * any launch and leave the buffers untouched.  GSVD_ENOCONV still writes the
 * outputs of the last sweep.  Device-side failures (GSVD_ENOTPD,
 * GSVD_EOVERFLOW) are per problem; one failed problem of a batch does not
 * affect the others.
 */
#ifndef GSVD_GB300_H
#define GSVD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GSVD_OK = 0,
  GSVD_EAGAIN = 1,     /* poll: not finished; submit: queue full */
  GSVD_EINVAL = -1,    /* bad argument, non-finite input, m < n, n < 1, ld < m */
  GSVD_ENOMEM = -2,    /* device allocation failed */
  GSVD_ENOCONV = -3,   /* sweep cap reached; outputs written */
  GSVD_ENOTPD = -4,    /* non-positive Cholesky pivot or 1 - x^2 <= 0 (rank-deficient G) */
  GSVD_EOVERFLOW = -5, /* non-finite column norm */
  GSVD_ETIMEOUT = -6,  /* the deadline timeout_ms passed; outputs finalised from the last sweep */
  GSVD_ECUDA = -7,     /* a CUDA runtime call failed */
  GSVD_ETOOBIG = -8    /* one request exceeds the memory budget */
};

enum { GSVD_R64 = 0, GSVD_C128 = 1 };
enum { GSVD_PREC_FP64 = 0, GSVD_PREC_MIXED = 1 };
enum { GSVD_PATH_AUTO = 0, GSVD_PATH_POINTWISE = 1, GSVD_PATH_BLOCKED = 2 };
enum { GSVD_ORDER_ROUND_ROBIN = 0, GSVD_ORDER_ROW_CYCLIC = 1 };

typedef struct gsvd_ctx *gsvd_handle;

/* Solver configuration (gsvd_config_default fills the defaults below). */
typedef struct {
  int32_t precision;        /* GSVD_PREC_FP64 (default) or GSVD_PREC_MIXED: FP32 bulk sweeps with
                               FP64 2x2 parameters, then FP64 refinement sweeps */
  int32_t block_w;          /* block width w of Sec. 2.3 (pair width 2w); 0 = choose by size */
  int32_t max_sweeps;       /* outer sweep cap (default 30, Alg. cpu1) */
  int32_t inner_max_sweeps; /* inner sweep cap: 30 = full block (FB), 1 = block-oriented (BO) */
  int32_t criterion;        /* small-transformation criterion of Sec. 2.5: 1 = C1, 2 = C2 */
  int32_t sort;             /* 1 = per-step column sorting (Sec. 2.1) */
  int32_t path;             /* GSVD_PATH_*: pointwise in-shared-memory or blocked */
  int32_t order;            /* pointwise pivot order: GSVD_ORDER_* */
  int32_t fp32_max_sweeps;  /* mixed precision: cap of the FP32 bulk sweeps (default 30) */
  int32_t timeout_ms;       /* deadline of one blocked solve, counted from its start (the call for
                               gsvd_solve, the start on a worker for gsvd_submit); 0 = none (default).
                               Checked after every outer sweep: once it has passed no further sweep
                               is issued, the outputs are finalised from that sweep's state (a valid
                               decomposition, as after the sweep cap) and the status is
                               GSVD_ETIMEOUT.  A host wait therefore ends at most one sweep and the
                               finalisation after the deadline; the device is idle for that solve
                               when the call returns.  The pointwise kernel (one launch) ignores it */
  uint64_t hbm_budget_bytes;/* serving: device memory admitted at once (default 60 GiB): the
                               workspaces of the requests on the GPU, which come from the handle's
                               stream-ordered pool and return to it when a request ends */
  int32_t max_inflight;     /* serving: requests on the GPU at once (default 16) */
  int32_t profile;          /* 1 = time every Gram / inner / apply launch with CUDA events on the
                               solve's stream (gsvd_info.t_kernel_us); 0 = off (default) */
  int32_t inner_max_sweeps_fp32; /* inner sweep cap of the FP32 bulk sweeps (default 1 = BO;
                               0 = same as inner_max_sweeps) */
  int32_t shorten;          /* QR shortening of Sec. 2 (F = Q_F R_F, G = Q_G R_G, sweeps on the n x n
                               factors): 0 = never, 1 = when m_F + m_G >= 2.6 n on the blocked real path
                               (default), 2 = whenever possible.  Skipped (and reported) when a Gram of
                               F or G is too ill-conditioned for CholeskyQR2 */
  int32_t fp32_params;      /* mixed precision: 1 = the pivot-pair step of the FP32 bulk sweeps (partial
                               Gram sums, the two Choleskys, the 2x2 parameters) in FP32, whose inputs
                               are FP32 dot products anyway (default); 0 = those in FP64 */
  int32_t fp64_gemm;        /* blocked FP64 sweeps: pivot Grams and block applies 1 = on the BF16 tensor
                               cores with FP64 accuracy (operands split into eight 8-bit integer
                               slices, exact level sums, one rounding; mma.sync; default, block widths
                               with 2w <= 32 real / 4w <= 32 complex), 2 = the same with the block
                               apply issued as tcgen05.mma with its level sums in tensor memory,
                               0 = FP64 DMMA */
  int32_t fp32_stop_permille; /* mixed precision: the FP32 bulk sweeps stop (and the FP64 sweeps take
                               over) after a sweep in which big transformations number fewer than
                               this many per mille of the pivot pairs examined (default 50); 0 = run
                               them to their own convergence (or fp32_max_sweeps) */
  int32_t variant;          /* variants of Sec. 2.6 (Table "Variants") besides the criterion: +1 = the
                               enhanced dot products of App. A, +2 = no prescaling, each pivot pair
                               rescaled by D-hat (Z-hat = D-hat Z-hat'); with criterion = 2 these are
                               variants 4-7.  Default 0.  Variants 1-3 run on the pointwise kernel
                               only: a problem that takes the blocked path is GSVD_EINVAL */
} gsvd_config;

/* One problem.  dtype = GSVD_R64 or GSVD_C128.
 * Sizes: 1 <= n <= 32768 and n <= m_f, m_g <= 2^30.  n < 4 always runs on the
 * pointwise kernel, which holds the whole problem in one CTA's shared memory
 * ((m_f + m_g + n) n doubles, twice that complex, plus its tables, within
 * 227 KB); a larger problem with n < 4 is GSVD_EINVAL. */
typedef struct {
  int32_t dtype;
  int32_t reserved;
  int64_t m_f, m_g, n;
  void *F;                  /* in: F (m_f x n);  out: U */
  int64_t ldf;
  void *G;                  /* in: G (m_g x n);  out: V */
  int64_t ldg;
  void *Z;                  /* out: Z (n x n) */
  int64_t ldz;
  double *sigma_f;          /* out: diag(Sigma_F), length n, sorted by descending Sigma */
  double *sigma_g;          /* out: diag(Sigma_G) */
  double *sigma;            /* out: Sigma = Sigma_F / Sigma_G */
  void *X;                  /* optional out (NULL = not wanted): the right generalized singular vectors
                               X = Z^-1 (n x n, the problem's dtype), gsvd_solve and gsvd_submit (Sec. 1:
                               X may be computed from Z).  Computed from the identity X = Sigma_F U^* F +
                               Sigma_G V^* G, which holds because [U Sigma_F; V Sigma_G] has orthonormal
                               columns; the library keeps copies of F and G for it ((m_f + m_g) n
                               elements of device memory during the solve).  The GEVD of (F^* F, G^* G)
                               is Z with Lambda = Sigma^2 */
  int64_t ldx;
} gsvd_problem;

/* Per-solve report. */
typedef struct {
  int32_t status;           /* GSVD_* of this problem */
  int32_t sweeps_fp32;      /* FP32 bulk sweeps (mixed precision) */
  int32_t sweeps_fp64;      /* FP64 sweeps (outer sweeps of the blocked path; sweeps of the pointwise path) */
  int32_t path;             /* GSVD_PATH_POINTWISE or GSVD_PATH_BLOCKED */
  uint64_t transf_all;      /* transformations applied (all classes) */
  uint64_t transf_big;      /* big transformations (Sec. 2.5) */
  double t_total_us;        /* wall time of the solve on the device */
  double t_fp32_us;         /* time of the FP32 bulk sweeps */
  double t_refine_us;       /* time of the FP64 sweeps after the FP32 ones */
  int32_t block_w;          /* block width used (0 = pointwise) */
  int32_t chol_skipped;     /* FP32 pivot blocks skipped for a failed Cholesky */
  uint64_t visits;          /* block pair visits (blocked path) */
  uint64_t visits_applied;  /* visits whose Z-tilde was applied (the others had no transformation) */
  double t_kernel_us[6];    /* with profile = 1: summed launch times of Gram FP64, inner FP64, apply
                               FP64, Gram FP32, inner FP32, apply FP32 */
  int32_t n_kernel[6];      /* launch counts of the same kernels */
  uint64_t visits_fp32;     /* of visits: those in FP32 bulk sweeps */
  uint64_t visits_applied_fp32; /* of visits_applied: those in FP32 bulk sweeps */
  int32_t shortened;        /* 1: the sweeps ran on the QR factors (R_F, R_G) */
  int32_t shorten_skipped;  /* 1: shortening was wanted but a Gram was too ill-conditioned */
  double t_qr_us;           /* time of the QR shortening and of U = Q_F U'', V = Q_G V'' */
  int32_t qr_launches;      /* kernel launches of the QR shortening (CholeskyQR2 and the products) */
  int32_t reserved2;
} gsvd_info;

/* Fill cfg with the defaults. */
void gsvd_config_default(gsvd_config *cfg);

/* Create a handle.  cfg may be NULL (defaults).  cuda_stream: a cudaStream_t,
 * NULL = the legacy default stream.  One handle per host thread/stream. */
int gsvd_create(gsvd_handle *h, const gsvd_config *cfg, void *cuda_stream);

/* Destroy a handle: waits for its serving threads and frees its workspace
 * pool.  Workspaces of a handle come from a stream-ordered device memory pool
 * of the current device, created at the handle's first solve; memory freed
 * into it stays reserved for later workspaces until the handle is destroyed,
 * so repeated solves allocate nothing new and never synchronize the device
 * for an allocation. */
int gsvd_destroy(gsvd_handle h);

/* Solve one problem; blocks until the outputs are written.  info may be NULL.
 * Returns the problem's status. */
int gsvd_solve(gsvd_handle h, const gsvd_problem *p, gsvd_info *info);

/* Solve count independent problems; problems small enough for shared memory
 * run in one launch of the pointwise kernel (one CTA each), the others on the
 * blocked path.  infos (may be NULL) receives one report per problem.
 * Returns GSVD_OK if every problem succeeded, else the first failing status. */
int gsvd_solve_batched(gsvd_handle h, const gsvd_problem *ps, int32_t count, gsvd_info *infos);

/* Serving: enqueue a problem (device pointers only) for the handle's
 * scheduler thread, which admits requests while the memory budget and the
 * in-flight limit allow and runs them concurrently on their own streams.
 * The library reads the buffers on its own streams: writes to them pending
 * on any other stream must be complete before the call.
 * Returns GSVD_OK with *ticket set, GSVD_ETOOBIG if the request alone exceeds
 * the budget, GSVD_EINVAL for a bad problem. */
int gsvd_submit(gsvd_handle h, const gsvd_problem *p, uint64_t *ticket);

/* Serving: GSVD_EAGAIN while the ticket is queued or running; otherwise the
 * request's final status (info filled, the ticket released). */
int gsvd_poll(gsvd_handle h, uint64_t ticket, gsvd_info *info);

/* Block-width autotuner: times one sweep of each candidate block width (real
 * 8, 16, 32; complex 4, 8, 16; widths with 2w > n are skipped) on a synthetic
 * pair of this shape (deterministic values in [-1, 1)) with the handle's
 * configuration, and records the fastest for the problem's class (data type,
 * precision, shortened or not, n rounded up to a power of two).  Later solves
 * of that class through this handle (gsvd_solve, gsvd_solve_batched,
 * gsvd_submit) use the recorded width when the configuration's block_w is 0.
 * *block_w receives the width, or 0 when there is nothing to choose (the
 * class runs on the pointwise kernel, or the configuration fixes block_w).
 * Blocks until done; allocates the synthetic pair for the duration of the
 * call. */
int gsvd_autotune(gsvd_handle h, int32_t dtype, int64_t m_f, int64_t m_g, int64_t n, int32_t *block_w);

/* Device bytes a solve of this shape needs beyond the caller's buffers; 0 for
 * a shape the library does not take (see gsvd_problem). */
uint64_t gsvd_workspace_bytes(const gsvd_config *cfg, int32_t dtype, int64_t m_f, int64_t m_g, int64_t n);

/* Static text of a status code. */
const char *gsvd_strerror(int status);

/* ---- allocation-free batch of small problems --------------------------------
 * The paper has no counterpart of this entry point; it exists for callers that
 * must not allocate device memory: code whose device memory is owned by its own
 * pool allocator, latency-critical loops in which cudaMalloc/cudaFree would
 * synchronize the device, host callbacks that may not enter the allocator.
 *
 * Solves count independent problems on the pointwise kernel (one CTA per
 * problem) exactly as gsvd_solve_batched does for small problems, but without
 * any device or pinned allocation: the kernel's scratch (the descriptor table
 * it reads and the status records it writes) is a fixed array of about 480 KiB
 * compiled into the library, which every GPU that loads the library keeps until
 * the process exits.  Limits: count <= GSVD_NOALLOC_MAX_PROBLEMS and n <= 64
 * with F, G, Z fitting in shared memory (else GSVD_ETOOBIG); m_F, m_G <= 2^30
 * as for gsvd_solve; every pointer of every problem must be memory of the
 * current device or managed memory (else GSVD_EINVAL).  cfg may be NULL
 * (defaults; precision, path and block width are ignored: FP64 pointwise;
 * criterion, sort, order, max_sweeps and variant apply).
 * cuda_stream: a cudaStream_t of the current device, NULL = legacy stream.
 *
 * The first call on a device (with that device current) looks up the array's
 * device address; make that first call before any stream capture.  The call
 * is synchronous: it returns after its work on cuda_stream has finished.
 * Every call reuses the same array, and the array keeps the last call's
 * contents (the status records are cleared at the start of each call); calls
 * are serialized inside the library, and two calls on the same device whose
 * work overlapped on the GPU would race on the array.
 * Returns GSVD_OK if every problem succeeded, else the first failing status;
 * infos (may be NULL) receives one report per problem.  An argument rejection
 * (GSVD_EINVAL or GSVD_ETOOBIG before any launch) leaves infos unwritten. */
#define GSVD_NOALLOC_MAX_PROBLEMS 4096
int gsvd_solve_small_noalloc(const gsvd_problem *ps, int32_t count, const gsvd_config *cfg,
                             void *cuda_stream, gsvd_info *infos);

#ifdef __cplusplus
}
#endif

#endif /* GSVD_GB300_H */
