// gsvd_api.cu -- host runtime behind the C ABI of include/gsvd.h: validation,
// planning (path, block width, row splits, pivot tables), workspace, the
// sweep loop of Alg. cpu1 (Sec. 3.6) with the convergence test of Sec. 2.5,
// the mixed-precision driver, batched solves and the serving scheduler.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gsvd.h"
#include "hz_kernels.h"

using namespace hz;

namespace {
// a named host range around one phase of a solve, for profilers that record
// NVTX ranges (a no-op when none is attached)
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace

namespace {

constexpr double EPS64 = 1.1102230246251565e-16;  // 2^-53
constexpr double EPS32 = 5.9604644775390625e-08;  // 2^-24
constexpr int POINTWISE_MAX_N = 64;  // at most 32 pairs per step: one lane each
constexpr int NCTR = 8;

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Round-robin ("circle method") table for M (even) players: M-1 steps of M/2
// disjoint pairs; every pair once per sweep (a cyclic parallel strategy,
// Sec. 2.2).  Players >= nreal are dummies (their pairs are skipped).
std::vector<uint16_t> round_robin_table(int M) {
  std::vector<uint16_t> t((size_t)(M - 1) * (M / 2) * 2);
  for (int s = 0; s < M - 1; ++s)
    for (int k = 0; k < M / 2; ++k) {
      int a, b;
      if (k == 0) {
        a = M - 1;
        b = s;
      } else {
        a = (s + k) % (M - 1);
        b = (s - k + (M - 1)) % (M - 1);
      }
      t[((size_t)s * (M / 2) + k) * 2] = (uint16_t)std::min(a, b);
      t[((size_t)s * (M / 2) + k) * 2 + 1] = (uint16_t)std::max(a, b);
    }
  return t;
}

// Wavefront of the row-cyclic order: step s holds the pairs (i, j), i < j,
// i + j = s + 1.  Any order consistent with the row-cyclic dependencies gives
// the same transformations, so this parallel table reproduces the sequential
// row-cyclic strategy exactly.  Unused slots hold (0xffff, 0xffff).
std::vector<uint16_t> row_cyclic_table(int n, int* steps, int* slots) {
  *steps = std::max(1, 2 * n - 3);
  *slots = std::max(1, n / 2);
  std::vector<uint16_t> t((size_t)(*steps) * (*slots) * 2, 0xffff);
  for (int s = 0; s < *steps; ++s) {
    const int sum = s + 1;
    int k = 0;
    for (int i = std::max(0, sum - (n - 1)); 2 * i < sum; ++i) {
      const int j = sum - i;
      if (j <= i || j >= n) continue;
      t[((size_t)s * (*slots) + k) * 2] = (uint16_t)i;
      t[((size_t)s * (*slots) + k) * 2 + 1] = (uint16_t)j;
      ++k;
    }
  }
  return t;
}

// Per-thread state of the call being served: the handle's stream-ordered
// memory pool (workspaces come from it with cudaMallocFromPoolAsync and go
// back with cudaFreeAsync, so no allocation or free synchronizes the device
// once the pool holds the memory) and the solve's deadline (timeout_ms).
struct CallState {
  cudaMemPool_t pool = nullptr;
  bool has_deadline = false;
  std::chrono::steady_clock::time_point deadline;
};
thread_local CallState tl_call;

struct CallScope {
  CallState saved;
  CallScope(cudaMemPool_t pool, int timeout_ms) : saved(tl_call) {
    tl_call.pool = pool;
    tl_call.has_deadline = timeout_ms > 0;
    if (timeout_ms > 0)
      tl_call.deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  }
  ~CallScope() { tl_call = saved; }
  CallScope(const CallScope&) = delete;
  CallScope& operator=(const CallScope&) = delete;
};

bool deadline_passed() {
  return tl_call.has_deadline && std::chrono::steady_clock::now() >= tl_call.deadline;
}

// Device buffer from the calling thread's pool (stream-ordered on the stream
// of its allocation), or cudaMalloc'ed when no pool is set.
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  cudaMemPool_t pool = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      if (pool)
        cudaFreeAsync(p, s);
      else
        cudaFree(p);
    }
    p = nullptr;
    n = 0;
  }
  cudaError_t ensure(size_t bytes, cudaStream_t st) {
    if (bytes <= n && st == s) return cudaSuccess;
    release();
    pool = tl_call.pool;
    s = st;
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMalloc(&p, bytes);
    if (e == cudaSuccess)
      n = bytes;
    else
      p = nullptr;
    return e;
  }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

struct Plan {
  bool cplx;
  int E;
  int mf, mg, n;
  int path;  // GSVD_PATH_POINTWISE / BLOCKED
  // blocked
  int w = 0, nblk = 0, neff = 0, nslots = 0, steps = 0, rf = 1, rg = 1, rf32 = 1, rg32 = 1, V = 0;
  // workspace layout (bytes)
  size_t off_partial = 0, off_ztil = 0, off_flags = 0, off_ctr = 0, off_zdiag = 0, off_norms = 0,
         off_rank = 0, off_status = 0, off_work = 0, off_f32 = 0, off_g32 = 0, off_z32 = 0, off_table = 0,
         total = 0;
  size_t table_bytes = 0;
  // pointwise
  int pw_steps = 0, pw_slots = 0;
  size_t pw_smem = 0;
};

int choose_w(const gsvd_config& c, bool cplx, int n) {
  if (c.block_w > 0) return c.block_w;
  if (cplx) return n >= 256 ? 16 : 8;
  return n >= 512 ? 16 : 8;
}

bool make_plan(const gsvd_config& cfg, int dtype, int64_t mf, int64_t mg, int64_t n, Plan& P) {
  P.cplx = dtype == GSVD_C128;
  P.E = P.cplx ? 2 : 1;
  P.mf = (int)mf;
  P.mg = (int)mg;
  P.n = (int)n;
  const int slots_rr = (int)((n + 1) / 2);
  size_t pw_smem = pointwise_smem_bytes((int)mf, (int)mg, (int)n, P.cplx, false,
                                        cfg.order == GSVD_ORDER_ROW_CYCLIC ? std::max<int64_t>(1, n / 2) : slots_rr);
  bool pw_ok = n <= POINTWISE_MAX_N && pw_smem <= POINTWISE_SMEM_MAX;
  if (cfg.path == GSVD_PATH_POINTWISE && !pw_ok) return false;
  if (cfg.path == GSVD_PATH_POINTWISE || (cfg.path == GSVD_PATH_AUTO && pw_ok) || n < 4) {
    if (!pw_ok) return false;
    P.path = GSVD_PATH_POINTWISE;
    if (cfg.order == GSVD_ORDER_ROW_CYCLIC) {
      row_cyclic_table((int)n, &P.pw_steps, &P.pw_slots);
    } else {
      const int M = (int)(n + (n & 1));
      P.pw_steps = std::max(1, M - 1);
      P.pw_slots = std::max(1, M / 2);
    }
    P.pw_smem = pointwise_smem_bytes((int)mf, (int)mg, (int)n, P.cplx, false, P.pw_slots);
    P.table_bytes = (size_t)P.pw_steps * P.pw_slots * 4;
    P.off_table = 0;
    P.off_status = align256(P.table_bytes);
    P.total = P.off_status + 256;
    return true;
  }
  P.path = GSVD_PATH_BLOCKED;
  P.w = choose_w(cfg, P.cplx, (int)n);
  P.V = blk_vmax(P.w, P.cplx);
  if (P.V == 0) return false;
  P.nblk = (int)((n + P.w - 1) / P.w);
  if (P.nblk < 2) {
    // too narrow for two blocks: halve the width
    P.w = std::max(1, (int)((n + 1) / 2));
    P.V = blk_vmax(P.w, P.cplx);
    P.nblk = (int)((n + P.w - 1) / P.w);
  }
  // variants 1-3 (Sec. 2.6) run in the FP64 pivot step of the two-CTA kernel
  if (cfg.variant != 0 && !inner_variants_supported(P.V)) return false;
  P.neff = P.nblk + (P.nblk & 1);
  P.nslots = P.neff / 2;
  P.steps = P.neff - 1;
  // row splits of the Gram, whole 64-row tiles per split, no empty split.
  // FP64 (DMMA, pipe-bound): about twelve CTAs per SM in total, so the uneven
  // last wave costs little.  FP32 (latency-bound, short CTAs): about four per
  // SM, so that each CTA streams several tiles and the pivot kernel sums
  // fewer partials.
  // The FP32 splits also serve the tensor-core FP64 Gram, whose split is
  // one exact accumulation of at most OZ_K_MAX rows.
  auto splits = [&](int per_sm, int max_tiles, int& rf, int& rg) {
    const int target = per_sm * 152;
    const int s = std::max(2, (target + P.nslots - 1) / P.nslots);
    const int tf = (int)((mf + 63) / 64), tg = (int)((mg + 63) / 64);
    const int sf = std::max(1, (int)std::lround((double)s * tf / (double)(tf + tg)));
    const int sg = std::max(1, s - sf);
    const int pf = std::min(max_tiles, (tf + sf - 1) / sf), pg = std::min(max_tiles, (tg + sg - 1) / sg);
    rf = (tf + pf - 1) / pf;  // tiles per split pf, pg
    rg = (tg + pg - 1) / pg;
  };
  splits(12, INT_MAX, P.rf, P.rg);
  splits(4, OZ_K_MAX / 64, P.rf32, P.rg32);
  const size_t V2 = (size_t)P.V * P.V;
  size_t o = 0;
  P.off_partial = o; o = align256(o + (size_t)P.nslots * std::max(P.rf + P.rg, P.rf32 + P.rg32) * V2 * 8);
  P.off_ztil = o; o = align256(o + (size_t)P.nslots * V2 * 8);
  P.off_flags = o; o = align256(o + (size_t)P.nslots * 4);
  P.off_ctr = o; o = align256(o + NCTR * 8);
  P.off_zdiag = o; o = align256(o + (size_t)n * 8);
  P.off_norms = o; o = align256(o + (size_t)2 * n * 8);
  P.off_rank = o; o = align256(o + (size_t)n * 4);
  P.off_status = o; o = align256(o + 16);
  P.off_work = o; o = align256(o + (size_t)std::max({mf, mg, n}) * n * P.E * 8);
  P.table_bytes = (size_t)P.steps * P.nslots * 4;
  P.off_table = o; o = align256(o + P.table_bytes);
  if (cfg.precision == GSVD_PREC_MIXED) {
    P.off_f32 = o; o = align256(o + (size_t)mf * n * P.E * 4);
    P.off_g32 = o; o = align256(o + (size_t)mg * n * P.E * 4);
    P.off_z32 = o; o = align256(o + (size_t)n * n * P.E * 4);
  }
  P.total = o;
  return true;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? GSVD_OK : (e == cudaErrorMemoryAllocation ? GSVD_ENOMEM : GSVD_ECUDA); }

#define CK(x)                               \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

// Where a caller pointer lives: 1 = device memory of the current device (or
// managed memory), 0 = host memory, -1 = device memory of another device.
// The kernels run on the current device, so -1 is refused by every entry
// point (a peer pointer would fault on the GPU instead of returning a status).
int ptr_loc(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeManaged) return 1;
  if (a.type != cudaMemoryTypeDevice) return 0;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return a.device == dev ? 1 : -1;
}

bool is_device_ptr(const void* p) { return ptr_loc(p) == 1; }

// the shapes the library takes: 1 <= n <= 32768, n <= m_F, m_G <= 2^30
bool shape_ok(int32_t dtype, int64_t mf, int64_t mg, int64_t n) {
  if (dtype != GSVD_R64 && dtype != GSVD_C128) return false;
  if (n < 1 || mf < n || mg < n) return false;
  return n <= 32768 && mf <= (int64_t)1 << 30 && mg <= (int64_t)1 << 30;
}

int validate(const gsvd_problem* p) {
  if (!p) return GSVD_EINVAL;
  if (!shape_ok(p->dtype, p->m_f, p->m_g, p->n)) return GSVD_EINVAL;
  if (p->ldf < p->m_f || p->ldg < p->m_g || p->ldz < p->n) return GSVD_EINVAL;
  if (!p->F || !p->G || !p->Z || !p->sigma_f || !p->sigma_g || !p->sigma) return GSVD_EINVAL;
  if (p->X && p->ldx < p->n) return GSVD_EINVAL;
  return GSVD_OK;
}

}  // namespace

// ------------------------------------------------------------------ ctx ----
struct Request {
  gsvd_problem prob;
  gsvd_info info;
  uint64_t bytes;
  int state;  // 0 queued, 1 running, 2 done
};

struct gsvd_ctx {
  gsvd_config cfg;
  cudaStream_t stream;
  cudaMemPool_t pool = nullptr;         // stream-ordered workspace pool of the handle
  DevBuf ws;
  unsigned long long* h_ctr = nullptr;  // pinned counters (NCTR)
  // serving
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  uint64_t used_bytes = 0;
  int inflight = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  // autotuned block widths by problem class (gsvd_autotune)
  std::mutex tune_mu;
  std::map<uint32_t, int> tuned;
};

namespace {

// problem class of the autotuner: data type, precision, whether the pair is
// shortened, and n rounded up to a power of two
uint32_t tune_key(const gsvd_config& cfg, int dtype, int64_t mf, int64_t mg, int64_t n) {
  int lg = 0;
  while (((int64_t)1 << lg) < n && lg < 31) ++lg;
  const bool sh = dtype == GSVD_R64 &&
                  (cfg.shorten == 2 || (cfg.shorten == 1 && (double)(mf + mg) >= 2.6 * (double)n));
  return (uint32_t)lg | ((uint32_t)(dtype == GSVD_C128) << 8) | ((uint32_t)(cfg.precision == GSVD_PREC_MIXED) << 9) |
         ((uint32_t)sh << 10);
}

// the handle's configuration for one problem: the autotuned block width of
// its class when the configuration leaves the width open
gsvd_config cfg_for(gsvd_ctx* h, const gsvd_problem* p) {
  gsvd_config c = h->cfg;
  if (c.block_w == 0) {
    std::lock_guard<std::mutex> lk(h->tune_mu);
    auto it = h->tuned.find(tune_key(c, p->dtype, p->m_f, p->m_g, p->n));
    if (it != h->tuned.end()) c.block_w = it->second;
  }
  return c;
}

}  // namespace

namespace {

// The blocked sweep loop on (F, G, Z) of type T: Alg. cpu1 with the outer
// stopping rule "no big transformation in a sweep" (Sec. 2.5).
struct KTimer {
  // per-launch CUDA events on the solve's stream (profile mode)
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  void mark(int k, cudaStream_t s) {
    cudaEvent_t a;
    cudaEventCreate(&a);
    cudaEventRecord(a, s);
    ev.push_back(a);
    kind.push_back(k);
  }
  void flush(gsvd_info* info) {
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      info->t_kernel_us[kind[i]] += ms * 1e3;
      info->n_kernel[kind[i]] += 1;
    }
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
    kind.clear();
  }
  KTimer() = default;
  KTimer(const KTimer&) = delete;
  KTimer& operator=(const KTimer&) = delete;
  ~KTimer() {
    for (auto e : ev) cudaEventDestroy(e);  // events of a solve that ended early
  }
};

// the three timing events of one solve, destroyed on every return path
struct SolveEvents {
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  SolveEvents() {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
  }
  ~SolveEvents() {
    for (cudaEvent_t e : {e0, e1, e2})
      if (e) cudaEventDestroy(e);
  }
  SolveEvents(const SolveEvents&) = delete;
  SolveEvents& operator=(const SolveEvents&) = delete;
};

int run_sweeps(const Plan& P, const gsvd_config& cfg, bool fp32, void* F, long long ldf, void* G, long long ldg,
               void* Z, long long ldz, unsigned char* ws, unsigned long long* h_ctr, int max_sweeps,
               cudaStream_t s, int* sweeps_out, uint64_t* tall, uint64_t* tbig, int* chol_skipped,
               gsvd_info* info) {
  TraceRange phase(fp32 ? "gsvd sweeps fp32" : "gsvd sweeps fp64");
  BlkDims d;
  d.mf = P.mf; d.mg = P.mg; d.n = P.n; d.w = P.w; d.nblk = P.nblk; d.nslots = P.nslots;
  // FP64 sweeps: Gram and apply on the tensor cores (sliced operands) or on
  // the FP64 pipe (DMMA)
  const bool oz = !fp32 && cfg.fp64_gemm >= 1 && oz_supported(P.V);
  const bool tc = cfg.fp64_gemm == 2;  // the apply on tcgen05
  d.rf = (fp32 || oz) ? P.rf32 : P.rf;
  d.rg = (fp32 || oz) ? P.rg32 : P.rg;
  d.trows = 64;
  BlkBuffers b;
  b.F = F; b.ldf = ldf; b.G = G; b.ldg = ldg; b.Z = Z; b.ldz = ldz;
  b.partial = ws + P.off_partial;
  b.ztil = ws + P.off_ztil;
  b.flags = reinterpret_cast<int*>(ws + P.off_flags);
  b.ctr = reinterpret_cast<unsigned long long*>(ws + P.off_ctr);
  b.table = reinterpret_cast<const uint16_t*>(ws + P.off_table);
  InnerParams ip;
  ip.eps = fp32 ? EPS32 : EPS64;
  // FP32 bulk sweeps: the pivot Grams carry FP32 rounding noise of about
  // eps32 * sqrt(m) relative (the expected error of a dot product of length m,
  // the argument the paper's threshold rests on); pairs below that level are
  // left to the FP64 sweeps.  FP64 sweeps use the paper's eps * sqrt(b).
  ip.tol = fp32 ? EPS32 * std::sqrt((double)std::max(P.mf, P.mg)) : 0.0;
  ip.inner_max = fp32 && cfg.inner_max_sweeps_fp32 > 0 ? cfg.inner_max_sweeps_fp32 : cfg.inner_max_sweeps;
  ip.sort = cfg.sort != 0;
  ip.f32cls = fp32;
  ip.crit2 = cfg.criterion == 2;
  ip.chol_skip = fp32;
  ip.par32 = fp32 && cfg.fp32_params != 0;
  ip.enhanced = !fp32 && (cfg.variant & 1) != 0;  // the variants act in the FP64 sweeps
  ip.dscale = !fp32 && (cfg.variant & 2) != 0;
  int sw = 0;
  bool converged = false;
  const bool prof = cfg.profile != 0;
  const int kb = fp32 ? 3 : 0;
  KTimer kt;
  static const bool trace = std::getenv("GSVD_TRACE") != nullptr;
  auto t_sweep = std::chrono::steady_clock::now();
  while (sw < max_sweeps) {
    CK(cudaMemsetAsync(b.ctr, 0, NCTR * sizeof(unsigned long long), s));
    for (int k = 0; k < P.steps; ++k) {
      if (prof) kt.mark(kb + 0, s);
      CK(oz ? launch_gram_oz(d, b, P.cplx, k, s) : launch_gram(d, b, P.cplx, fp32, k, s));
      if (prof) { kt.mark(kb + 0, s); kt.mark(kb + 1, s); }
      CK(launch_inner(d, b, P.cplx, fp32, k, ip, s));
      if (prof) { kt.mark(kb + 1, s); kt.mark(kb + 2, s); }
      CK(oz ? launch_apply_oz(d, b, P.cplx, k, s, tc) : launch_apply(d, b, P.cplx, fp32, k, s));
      if (prof) kt.mark(kb + 2, s);
    }
    CK(cudaMemcpyAsync(h_ctr, b.ctr, NCTR * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (prof) kt.flush(info);
    ++sw;
    *tall += h_ctr[0];
    *tbig += h_ctr[1];
    *chol_skipped += (int)h_ctr[3];
    info->visits += h_ctr[4];
    info->visits_applied += h_ctr[5];
    if (fp32) {
      info->visits_fp32 += h_ctr[4];
      info->visits_applied_fp32 += h_ctr[5];
    }
    if (trace) {
      const auto now = std::chrono::steady_clock::now();
      std::fprintf(stderr, "gsvd %s sweep %d: transf %llu big %llu visits %llu applied %llu fail %llu skip %llu  %.2f ms\n",
                   fp32 ? "fp32" : "fp64", sw, h_ctr[0], h_ctr[1], h_ctr[4], h_ctr[5], h_ctr[2], h_ctr[3],
                   std::chrono::duration<double, std::milli>(now - t_sweep).count());
      t_sweep = now;
    }
    if (h_ctr[2]) {
      *sweeps_out = sw;
      return GSVD_ENOTPD;
    }
    if (h_ctr[1] == 0) {
      converged = true;
      break;
    }
    if (deadline_passed()) {
      // timeout_ms: no further sweep is issued; the outputs are finalised
      // from this sweep's state, as after the sweep cap
      *sweeps_out = sw;
      return GSVD_ETIMEOUT;
    }
    // FP32 bulk sweeps hand over to the FP64 sweeps once few of their
    // transformations are big: the FP64 sweep count no longer falls after
    // that point, while every further FP32 sweep costs a full sweep
    // (pairs examined in the sweep: pair visits x b (b - 1) / 2 x inner sweeps)
    const double examined = (double)h_ctr[4] * (2.0 * P.w) * (2.0 * P.w - 1.0) * 0.5 * (double)ip.inner_max;
    if (fp32 && cfg.fp32_stop_permille > 0 &&
        (double)h_ctr[1] * 1000.0 < (double)cfg.fp32_stop_permille * examined) {
      converged = true;
      break;
    }
    CK(launch_rescale(P.mf, P.mg, P.n, P.cplx, fp32, F, ldf, G, ldg, Z, ldz, s));
  }
  *sweeps_out = sw;
  return converged ? GSVD_OK : GSVD_ENOCONV;
}

int solve_pointwise(const gsvd_config& cfg, const gsvd_problem* ps, const int* idx, int count, cudaStream_t s,
                    gsvd_info* infos) {
  // pivot pairs are generated per problem from its own n; the launch only
  // needs the largest step width of the batch for the shared-memory layout
  const bool rowcyc = cfg.order == GSVD_ORDER_ROW_CYCLIC;
  int slots = 1;
  for (int k = 0; k < count; ++k) {
    const int n = (int)ps[idx[k]].n;
    slots = std::max(slots, rowcyc ? std::max(1, n / 2) : std::max(1, (n + (n & 1)) / 2));
  }
  const size_t pb = align256(sizeof(PwProblem) * count);
  SolveEvents ev;  // the launch's time is every problem's (they run together)
  cudaEventRecord(ev.e0, s);
  DevBuf tmp;
  CK(tmp.ensure(2 * pb + sizeof(PwStats) * count, s));
  unsigned char* base = static_cast<unsigned char*>(tmp.p);
  PwStats* d_stats = reinterpret_cast<PwStats*>(base + 2 * pb);
  CK(cudaMemsetAsync(d_stats, 0, sizeof(PwStats) * count, s));
  PwParams prm;
  prm.eps = EPS64;
  prm.max_sweeps = cfg.max_sweeps;
  prm.sort = cfg.sort != 0;
  prm.f32cls = false;
  prm.crit2 = cfg.criterion == 2;
  prm.rowcyc = rowcyc;
  prm.enhanced = (cfg.variant & 1) != 0;
  prm.dscale = (cfg.variant & 2) != 0;
  // real and complex problems run in separate launches (one kernel each)
  size_t off = 0;
  std::vector<int> pos(count);
  for (int kind = 0; kind < 2; ++kind) {
    std::vector<PwProblem> sub;
    size_t smem = 0;
    for (int k = 0; k < count; ++k) {
      const gsvd_problem& p = ps[idx[k]];
      if ((p.dtype == GSVD_C128) != (kind == 1)) continue;
      PwProblem q;
      q.F = p.F; q.ldf = p.ldf; q.G = p.G; q.ldg = p.ldg; q.Z = p.Z; q.ldz = p.ldz;
      q.mf = (int)p.m_f; q.mg = (int)p.m_g; q.n = (int)p.n; q.pad = 0;
      q.sigma_f = p.sigma_f; q.sigma_g = p.sigma_g; q.sigma = p.sigma;
      q.stats = d_stats + k;
      sub.push_back(q);
      smem = std::max(smem, pointwise_smem_bytes(q.mf, q.mg, q.n, kind == 1, false, slots));
    }
    if (sub.empty()) continue;
    PwProblem* d_probs = reinterpret_cast<PwProblem*>(base + off);
    off += pb;
    CK(cudaMemcpyAsync(d_probs, sub.data(), sizeof(PwProblem) * sub.size(), cudaMemcpyHostToDevice, s));
    CK(launch_pointwise(d_probs, (int)sub.size(), slots, kind == 1, false, smem, prm, s));
  }
  std::vector<PwStats> hs(count);
  cudaEventRecord(ev.e1, s);
  CK(cudaMemcpyAsync(hs.data(), d_stats, sizeof(PwStats) * count, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.e0, ev.e1);
  for (int k = 0; k < count; ++k) {
    gsvd_info& in = infos[idx[k]];
    in.t_total_us = ms * 1e3;
    in.status = hs[k].status;
    in.sweeps_fp64 = hs[k].sweeps;
    in.sweeps_fp32 = 0;
    in.transf_all = (uint64_t)hs[k].transf_all;
    in.transf_big = (uint64_t)hs[k].transf_big;
    in.path = GSVD_PATH_POINTWISE;
    in.block_w = 0;
  }
  return GSVD_OK;
}

// QR shortening applies to real blocked problems that are tall enough
bool shorten_applies(const gsvd_config& cfg, const Plan& P, int64_t mf, int64_t mg, int64_t n) {
  return P.path == GSVD_PATH_BLOCKED && !P.cplx && n >= 2 &&
         (cfg.shorten == 2 || (cfg.shorten == 1 && (double)(mf + mg) >= 2.6 * (double)n));
}

// workspace of a shortened solve: the n x n sub-problem's plan, then
// R_F, R_G, R1_F, R1_G (n x n each), a max(m_F, m_G) x n product buffer and
// two flags
size_t shortened_offset(const gsvd_config& cfg, int64_t n) {
  Plan S;
  make_plan(cfg, GSVD_R64, n, n, n, S);
  return (S.total + 255) & ~size_t(255);
}
// digit planes of the tensor-core products (fp64_gemm = 1): the largest of
// the Grams F^T F (n x n over one piece of at most OZ_K_MAX of the m rows)
// and the products m x n x n
size_t shortened_oz_bytes(const gsvd_config& cfg, int64_t mf, int64_t mg, int64_t n) {
  if (cfg.fp64_gemm == 0) return 0;
  const int m = (int)std::max(mf, mg);
  return std::max(dgemm_oz_ws_bytes((int)n, (int)n, std::min(m, OZ_K_MAX)), dgemm_oz_ws_bytes(m, (int)n, (int)n));
}
size_t shortened_total(const gsvd_config& cfg, int64_t mf, int64_t mg, int64_t n) {
  return shortened_offset(cfg, n) + sizeof(double) * (4 * (size_t)n * n + (size_t)std::max(mf, mg) * n) + 256 +
         shortened_oz_bytes(cfg, mf, mg, n);
}

// device bytes one solve needs
size_t solve_bytes(const gsvd_config& cfg, const Plan& P, int64_t mf, int64_t mg, int64_t n) {
  if (shorten_applies(cfg, P, mf, mg, n)) return std::max(P.total, shortened_total(cfg, mf, mg, n));
  return P.total;
}

// one problem with device pointers on stream s, workspace ws (>= P.total)
int solve_plain(const gsvd_config& cfg, const gsvd_problem* p, gsvd_info* info, DevBuf& ws,
                unsigned long long* h_ctr, cudaStream_t s) {
  Plan P;
  if (!make_plan(cfg, p->dtype, p->m_f, p->m_g, p->n, P)) return GSVD_EINVAL;
  CK(ws.ensure(P.total, s));
  unsigned char* w = static_cast<unsigned char*>(ws.p);
  SolveEvents ev;
  cudaEvent_t e0 = ev.e0, e1 = ev.e1, e2 = ev.e2;
  cudaEventRecord(e0, s);
  int* d_status = reinterpret_cast<int*>(w + P.off_status);
  CK(cudaMemsetAsync(d_status, 0, 16, s));
  // non-finite input check
  CK(launch_check_finite(P.mf, P.n, P.cplx, (const double*)p->F, p->ldf, d_status + 1, s));
  CK(launch_check_finite(P.mg, P.n, P.cplx, (const double*)p->G, p->ldg, d_status + 1, s));
  int hst[4];
  CK(cudaMemcpyAsync(hst, d_status, 16, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hst[1]) {
    info->status = GSVD_EINVAL;
    return GSVD_EINVAL;
  }
  int status = GSVD_OK;
  info->path = P.path;
  info->block_w = P.path == GSVD_PATH_BLOCKED ? P.w : 0;
  if (P.path == GSVD_PATH_POINTWISE) {
    int idx0 = 0;
    status = solve_pointwise(cfg, p, &idx0, 1, s, info);
    if (status == GSVD_OK) status = info->status;
  } else {
    double* F = (double*)p->F;
    double* G = (double*)p->G;
    double* Z = (double*)p->Z;
    double* zdiag = reinterpret_cast<double*>(w + P.off_zdiag);
    std::vector<uint16_t> table = round_robin_table(P.neff);
    CK(cudaMemcpyAsync(w + P.off_table, table.data(), table.size() * 2, cudaMemcpyHostToDevice, s));
    CK(launch_prescale(P.mf, P.mg, P.n, P.cplx, F, p->ldf, G, p->ldg, Z, p->ldz, zdiag, d_status, s));
    uint64_t tall = 0, tbig = 0;
    int chol = 0, sw32 = 0, sw64 = 0;
    if (cfg.precision == GSVD_PREC_MIXED) {
      float* F32 = reinterpret_cast<float*>(w + P.off_f32);
      float* G32 = reinterpret_cast<float*>(w + P.off_g32);
      float* Z32 = reinterpret_cast<float*>(w + P.off_z32);
      CK(launch_to_f32(P.mf, P.n, P.cplx, F, p->ldf, F32, P.mf, s));
      CK(launch_to_f32(P.mg, P.n, P.cplx, G, p->ldg, G32, P.mg, s));
      CK(launch_identity(P.n, P.cplx, true, Z32, P.n, s));
      int st32 = run_sweeps(P, cfg, true, F32, P.mf, G32, P.mg, Z32, P.n, w, h_ctr, cfg.fp32_max_sweeps, s, &sw32,
                            &tall, &tbig, &chol, info);
      if (st32 != GSVD_OK && st32 != GSVD_ENOCONV) status = st32;
      cudaEventRecord(e1, s);
      // F <- F Z_acc, G <- G Z_acc (FP64), Z <- Z0 Z_acc
      double* work = reinterpret_cast<double*>(w + P.off_work);
      CK(launch_gemm_f64_by_f32(P.mf, P.n, P.cplx, F, p->ldf, Z32, P.n, work, P.mf, s));
      CK(cudaMemcpy2DAsync(F, p->ldf * 8 * P.E, work, (size_t)P.mf * 8 * P.E, (size_t)P.mf * 8 * P.E, P.n,
                           cudaMemcpyDeviceToDevice, s));
      CK(launch_gemm_f64_by_f32(P.mg, P.n, P.cplx, G, p->ldg, Z32, P.n, work, P.mg, s));
      CK(cudaMemcpy2DAsync(G, p->ldg * 8 * P.E, work, (size_t)P.mg * 8 * P.E, (size_t)P.mg * 8 * P.E, P.n,
                           cudaMemcpyDeviceToDevice, s));
      CK(launch_rowscale(P.n, P.cplx, zdiag, Z32, P.n, Z, p->ldz, s));
    } else {
      cudaEventRecord(e1, s);
    }
    if (status == GSVD_OK) {
      status = run_sweeps(P, cfg, false, F, p->ldf, G, p->ldg, Z, p->ldz, w, h_ctr, cfg.max_sweeps, s, &sw64,
                          &tall, &tbig, &chol, info);
    }
    TraceRange phase_fin("gsvd finalize");
    CK(launch_finalize(P.mf, P.mg, P.n, P.cplx, F, p->ldf, G, p->ldg, Z, p->ldz, p->sigma_f, p->sigma_g, p->sigma,
                       reinterpret_cast<double*>(w + P.off_norms), reinterpret_cast<int*>(w + P.off_rank),
                       reinterpret_cast<double*>(w + P.off_work), d_status, s));
    CK(cudaMemcpyAsync(hst, d_status, 16, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (status == GSVD_OK && hst[0] != 0) status = hst[0];
    info->sweeps_fp32 = sw32;
    info->sweeps_fp64 = sw64;
    info->transf_all = tall;
    info->transf_big = tbig;
    info->chol_skipped = chol;
  }
  cudaEventRecord(e2, s);
  cudaEventSynchronize(e2);
  float ms_all = 0, ms_32 = 0, ms_64 = 0;
  cudaEventElapsedTime(&ms_all, e0, e2);
  if (P.path == GSVD_PATH_BLOCKED) {
    cudaEventElapsedTime(&ms_32, e0, e1);
    cudaEventElapsedTime(&ms_64, e1, e2);
  }
  info->t_total_us = ms_all * 1e3;
  info->t_fp32_us = cfg.precision == GSVD_PREC_MIXED ? ms_32 * 1e3 : 0.0;
  info->t_refine_us = cfg.precision == GSVD_PREC_MIXED ? ms_64 * 1e3 : 0.0;
  info->status = status;
  return status;
}

constexpr int SHORT_SKIP = 100;

// QR shortening (Sec. 2): F = Q_F R_F, G = Q_G R_G by CholeskyQR2, the sweeps
// on (R_F, R_G) (n x n), then U = Q_F U'', V = Q_G V''.  Returns SHORT_SKIP,
// with F and G untouched, when a first Cholesky fails (too ill-conditioned).
int solve_shortened(const gsvd_config& cfg, const gsvd_problem* p, gsvd_info* info, DevBuf& ws,
                    unsigned long long* h_ctr, cudaStream_t s) {
  TraceRange phase("gsvd shortened solve");
  const int n = (int)p->n, mf = (int)p->m_f, mg = (int)p->m_g;
  double* F = (double*)p->F;
  double* G = (double*)p->G;
  const size_t nn = (size_t)n * n;
  const size_t tmp = (size_t)std::max(mf, mg) * n;
  CK(ws.ensure(shortened_total(cfg, mf, mg, n), s));
  double* RF = reinterpret_cast<double*>(static_cast<unsigned char*>(ws.p) + shortened_offset(cfg, n));
  double* RG = RF + nn;
  double* R1F = RG + nn;
  double* R1G = R1F + nn;
  double* T = R1G + nn;
  int* flag = reinterpret_cast<int*>(T + tmp);
  OzWs ozw;
  ozw.bytes = shortened_oz_bytes(cfg, mf, mg, n);
  ozw.p = ozw.bytes ? reinterpret_cast<unsigned char*>(flag) + 256 : nullptr;
  const OzWs* oz = ozw.bytes ? &ozw : nullptr;
  int hflag[2];
  const long long l0 = qr_launch_count();
  CK(cudaMemsetAsync(flag, 0, 8, s));
  CK(launch_check_finite(mf, n, false, F, p->ldf, flag + 1, s));
  CK(launch_check_finite(mg, n, false, G, p->ldg, flag + 1, s));
  // first pass: Grams and Choleskys; F and G are not modified yet
  CK(dgemm(true, false, n, n, mf, 1.0, F, p->ldf, F, p->ldf, 0.0, R1F, n, true, s, oz));
  CK(potrf_upper(n, R1F, n, flag, s, oz));
  CK(dgemm(true, false, n, n, mg, 1.0, G, p->ldg, G, p->ldg, 0.0, R1G, n, true, s, oz));
  CK(potrf_upper(n, R1G, n, flag, s, oz));
  CK(cudaMemcpyAsync(hflag, flag, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hflag[1]) return GSVD_EINVAL;
  if (hflag[0]) {
    info->shorten_skipped = 1;
    return SHORT_SKIP;
  }
  // Q1 = F R1^{-1}; second pass R2 = chol(Q1^T Q1), Q = Q1 R2^{-1}
  CK(trsm_right_upper(mf, n, R1F, n, F, p->ldf, s, oz));
  CK(trsm_right_upper(mg, n, R1G, n, G, p->ldg, s, oz));
  CK(dgemm(true, false, n, n, mf, 1.0, F, p->ldf, F, p->ldf, 0.0, RF, n, true, s, oz));
  CK(potrf_upper(n, RF, n, flag, s, oz));
  CK(dgemm(true, false, n, n, mg, 1.0, G, p->ldg, G, p->ldg, 0.0, RG, n, true, s, oz));
  CK(potrf_upper(n, RG, n, flag, s, oz));
  CK(cudaMemcpyAsync(hflag, flag, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hflag[0]) {
    // Q1^T Q1 not numerically positive definite: undo (F = Q1 R1) and skip
    CK(dgemm(false, false, mf, n, n, 1.0, F, p->ldf, R1F, n, 0.0, T, mf, false, s, oz));
    CK(cudaMemcpy2DAsync(F, p->ldf * 8, T, (size_t)mf * 8, (size_t)mf * 8, n, cudaMemcpyDeviceToDevice, s));
    CK(dgemm(false, false, mg, n, n, 1.0, G, p->ldg, R1G, n, 0.0, T, mg, false, s, oz));
    CK(cudaMemcpy2DAsync(G, p->ldg * 8, T, (size_t)mg * 8, (size_t)mg * 8, n, cudaMemcpyDeviceToDevice, s));
    info->shorten_skipped = 1;
    return SHORT_SKIP;
  }
  CK(trsm_right_upper(mf, n, RF, n, F, p->ldf, s, oz));
  CK(trsm_right_upper(mg, n, RG, n, G, p->ldg, s, oz));
  // R = R2 R1 (both upper triangular)
  CK(dgemm(false, false, n, n, n, 1.0, RF, n, R1F, n, 0.0, T, n, 2, s, oz));
  CK(launch_zero_lower(n, T, n, s));
  CK(cudaMemcpyAsync(RF, T, nn * 8, cudaMemcpyDeviceToDevice, s));
  CK(dgemm(false, false, n, n, n, 1.0, RG, n, R1G, n, 0.0, T, n, 2, s, oz));
  CK(launch_zero_lower(n, T, n, s));
  CK(cudaMemcpyAsync(RG, T, nn * 8, cudaMemcpyDeviceToDevice, s));
  // the sweeps on the shortened pair
  gsvd_problem sub = *p;
  sub.m_f = n;
  sub.m_g = n;
  sub.F = RF;
  sub.ldf = n;
  sub.G = RG;
  sub.ldg = n;
  gsvd_config c2 = cfg;
  c2.shorten = 0;
  const int st = solve_plain(c2, &sub, info, ws, h_ctr, s);
  if (st == GSVD_EINVAL || st == GSVD_ECUDA || st == GSVD_ENOMEM) return st;
  // U = Q_F U'', V = Q_G V''
  CK(dgemm(false, false, mf, n, n, 1.0, F, p->ldf, RF, n, 0.0, T, mf, false, s, oz));
  CK(cudaMemcpy2DAsync(F, p->ldf * 8, T, (size_t)mf * 8, (size_t)mf * 8, n, cudaMemcpyDeviceToDevice, s));
  CK(dgemm(false, false, mg, n, n, 1.0, G, p->ldg, RG, n, 0.0, T, mg, false, s, oz));
  CK(cudaMemcpy2DAsync(G, p->ldg * 8, T, (size_t)mg * 8, (size_t)mg * 8, n, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  info->shortened = 1;
  info->qr_launches = (int32_t)(qr_launch_count() - l0 + 2);  // + the two finiteness checks
  return st;
}

int solve_device_core(const gsvd_config& cfg, const gsvd_problem* p, gsvd_info* info, DevBuf& ws,
                      unsigned long long* h_ctr, cudaStream_t s) {
  TraceRange phase("gsvd solve");
  Plan P;
  if (!make_plan(cfg, p->dtype, p->m_f, p->m_g, p->n, P)) return GSVD_EINVAL;
  if (shorten_applies(cfg, P, p->m_f, p->m_g, p->n)) {
    const auto t0 = std::chrono::steady_clock::now();
    const int st = solve_shortened(cfg, p, info, ws, h_ctr, s);
    if (st != SHORT_SKIP) {
      const double us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
      info->t_qr_us = us - info->t_total_us;
      info->t_total_us = us;
      info->status = st;
      return st;
    }
  }
  return solve_plain(cfg, p, info, ws, h_ctr, s);
}

// one problem with device pointers; with p->X also the right vectors
// X = Z^-1 = Sigma_F U^T F + Sigma_G V^T G (the columns of [U Sigma_F;
// V Sigma_G] are orthonormal, so it is the left inverse of Z applied to
// [F; G] = [U Sigma_F; V Sigma_G] Z^-1), from copies of the inputs
int solve_device(const gsvd_config& cfg, const gsvd_problem* p, gsvd_info* info, DevBuf& ws,
                 unsigned long long* h_ctr, cudaStream_t s) {
  if (!p->X) return solve_device_core(cfg, p, info, ws, h_ctr, s);
  const int n = (int)p->n, mf = (int)p->m_f, mg = (int)p->m_g;
  const bool cplx = p->dtype == GSVD_C128;
  const size_t E = cplx ? 2 : 1;
  DevBuf keep;
  CK(keep.ensure(sizeof(double) * E * (((size_t)mf + mg) * n + (size_t)n * n) + 256, s));
  double* F0 = static_cast<double*>(keep.p);
  double* G0 = F0 + E * mf * n;
  double* T = G0 + E * mg * n;
  CK(cudaMemcpy2DAsync(F0, E * mf * 8, p->F, p->ldf * 8 * E, E * mf * 8, n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpy2DAsync(G0, E * mg * 8, p->G, p->ldg * 8 * E, E * mg * 8, n, cudaMemcpyDeviceToDevice, s));
  const int st = solve_device_core(cfg, p, info, ws, h_ctr, s);
  if (st != GSVD_OK && st != GSVD_ENOCONV && st != GSVD_ETIMEOUT) return st;
  double* X = static_cast<double*>(p->X);
  if (cplx) {
    // X = Sigma_F U^H F + Sigma_G V^H G ([U Sigma_F; V Sigma_G] has orthonormal columns)
    CK(launch_gemm_ch(mf, n, n, (const double*)p->F, p->ldf, F0, mf, X, p->ldx, s));
    CK(launch_gemm_ch(mg, n, n, (const double*)p->G, p->ldg, G0, mg, T, n, s));
  } else {
    CK(dgemm(true, false, n, n, mf, 1.0, (const double*)p->F, p->ldf, F0, mf, 0.0, X, p->ldx, 0, s));
    CK(dgemm(true, false, n, n, mg, 1.0, (const double*)p->G, p->ldg, G0, mg, 0.0, T, n, 0, s));
  }
  CK(launch_rows_combine(n, cplx, X, p->ldx, p->sigma_f, T, n, p->sigma_g, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

// host pointers: stage through device buffers (pinned or pageable host memory)
int solve_host(const gsvd_config& cfg, const gsvd_problem* p, gsvd_info* info, DevBuf& ws, unsigned long long* h_ctr,
               cudaStream_t s) {
  const int E = p->dtype == GSVD_C128 ? 2 : 1;
  const size_t es = 8 * E;
  const size_t bF = align256((size_t)p->m_f * p->n * es), bG = align256((size_t)p->m_g * p->n * es),
               bZ = align256((size_t)p->n * p->n * es), bv = align256((size_t)p->n * 8);
  DevBuf stage;
  const size_t bX = p->X ? align256((size_t)p->n * p->n * es) : 0;
  CK(stage.ensure(bF + bG + bZ + 3 * bv + bX, s));
  unsigned char* b = static_cast<unsigned char*>(stage.p);
  gsvd_problem d = *p;
  d.F = b; d.ldf = p->m_f;
  d.G = b + bF; d.ldg = p->m_g;
  d.Z = b + bF + bG; d.ldz = p->n;
  d.sigma_f = reinterpret_cast<double*>(b + bF + bG + bZ);
  d.sigma_g = reinterpret_cast<double*>(b + bF + bG + bZ + bv);
  d.sigma = reinterpret_cast<double*>(b + bF + bG + bZ + 2 * bv);
  if (p->X) {
    d.X = b + bF + bG + bZ + 3 * bv;
    d.ldx = p->n;
  }
  CK(cudaMemcpy2DAsync(d.F, p->m_f * es, p->F, p->ldf * es, p->m_f * es, p->n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpy2DAsync(d.G, p->m_g * es, p->G, p->ldg * es, p->m_g * es, p->n, cudaMemcpyHostToDevice, s));
  int st = solve_device(cfg, &d, info, ws, h_ctr, s);
  if (st == GSVD_EINVAL && info->status == GSVD_EINVAL) return st;
  CK(cudaMemcpy2DAsync(p->F, p->ldf * es, d.F, p->m_f * es, p->m_f * es, p->n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpy2DAsync(p->G, p->ldg * es, d.G, p->m_g * es, p->m_g * es, p->n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpy2DAsync(p->Z, p->ldz * es, d.Z, p->n * es, p->n * es, p->n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(p->sigma_f, d.sigma_f, p->n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(p->sigma_g, d.sigma_g, p->n * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(p->sigma, d.sigma, p->n * 8, cudaMemcpyDeviceToHost, s));
  if (p->X)
    CK(cudaMemcpy2DAsync(p->X, p->ldx * es, d.X, p->n * es, p->n * es, p->n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

int solve_any(const gsvd_config& cfg, const gsvd_problem* p, gsvd_info* info, DevBuf& ws, unsigned long long* h_ctr,
              cudaStream_t s) {
  int v = validate(p);
  if (v != GSVD_OK) {
    info->status = v;
    return v;
  }
  const int dev = ptr_loc(p->F);
  if (dev < 0 || dev != ptr_loc(p->G) || dev != ptr_loc(p->Z) || dev != ptr_loc(p->sigma) ||
      dev != ptr_loc(p->sigma_f) || dev != ptr_loc(p->sigma_g) || (p->X && dev != ptr_loc(p->X))) {
    info->status = GSVD_EINVAL;
    return GSVD_EINVAL;
  }
  return dev ? solve_device(cfg, p, info, ws, h_ctr, s) : solve_host(cfg, p, info, ws, h_ctr, s);
}

// The blocked problems of a gsvd_solve_batched call, all advancing together
// (north of the one-problem loop of Alg. cpu1): a global sweep runs, for every
// group of problems with the same data type and real-view width V, the outer
// steps k = 0, 1, ... as one Gram, one pivot-step and one apply launch each
// over all (problem, pair) items of the group -- a problem with fewer steps
// per sweep, or one not sweeping in that precision, has its CTAs leave at
// once -- then one launch for every problem's convergence test, one for the
// rescales, and one copy of the problems' states to the host.  The launches
// of a global sweep do not depend on the problem count; from the second
// sweep on they replay as one captured CUDA graph.  Mixed precision: every
// problem runs its FP32 bulk sweeps, the restart F <- F Z_acc (one batched
// launch sequence for the problems that reach it in the same sweep), and its
// FP64 sweeps, with the same rules as a single solve.  Every problem's
// arithmetic is the single-solve kernels' own, so a problem gets the same
// bits as gsvd_solve of it with shortening off.  The batched path does not
// shorten (the QR shortening of Sec. 2 is a per-problem phase).
struct BatchGroup {
  bool cplx = false;
  int V = 0, w = 0;
  int steps = 0;                 // most outer steps per sweep in the group
  int gy_gram[2] = {0, 0};       // grid y of the Gram per phase
  int gy_apply = 0;              // grid y of the apply
  int item0 = 0, nitems = 0;     // (problem, slot) items of the group
  InnerParams ip[2];
  bool oz = false;               // FP64 Gram and apply on the tensor cores
};

// A stream owned for the duration of a call, ordered after the work already
// queued on another stream (the handle's, which may be the legacy stream,
// where no graph can be captured).
struct OwnStream {
  cudaStream_t s = nullptr;
  explicit OwnStream(cudaStream_t after) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s = nullptr;
      return;
    }
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(e, after);
      cudaStreamWaitEvent(s, e, 0);
      cudaEventDestroy(e);
    }
  }
  ~OwnStream() {
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
  OwnStream(const OwnStream&) = delete;
  OwnStream& operator=(const OwnStream&) = delete;
};

int solve_blocked_batch(gsvd_ctx* h, const gsvd_problem* ps, const std::vector<int>& idx, gsvd_info* infos,
                        cudaStream_t hs_stream) {
  TraceRange phase("gsvd batched sweeps");
  const int P = (int)idx.size();
  if (P == 0) return GSVD_OK;
  OwnStream own(hs_stream);
  if (!own.s) return GSVD_ECUDA;
  const cudaStream_t s = own.s;
  const bool mixed = h->cfg.precision == GSVD_PREC_MIXED;
  std::vector<Plan> plans(P);
  std::vector<gsvd_config> cfgs(P);
  std::vector<size_t> woff(P);
  size_t wtotal = 0;
  int maxm = 1, maxn = 1;
  for (int k = 0; k < P; ++k) {
    const gsvd_problem& p = ps[idx[k]];
    cfgs[k] = cfg_for(h, &p);
    cfgs[k].shorten = 0;
    if (!make_plan(cfgs[k], p.dtype, p.m_f, p.m_g, p.n, plans[k])) return GSVD_EINVAL;
    woff[k] = wtotal;
    wtotal += align256(plans[k].total);
    maxm = std::max({maxm, (int)p.m_f, (int)p.m_g});
    maxn = std::max(maxn, (int)p.n);
  }
  // groups by (data type, V)
  std::map<std::pair<int, int>, std::vector<int>> gmap;
  for (int k = 0; k < P; ++k) gmap[{plans[k].cplx ? 1 : 0, plans[k].V}].push_back(k);
  std::vector<BatchGroup> groups;
  std::vector<int2> items;
  for (auto& kv : gmap) {
    BatchGroup g;
    g.cplx = kv.first.first != 0;
    g.V = kv.first.second;
    g.w = plans[kv.second[0]].w;
    g.oz = h->cfg.fp64_gemm >= 1 && oz_supported(g.V);
    g.item0 = (int)items.size();
    for (int k : kv.second) {
      const Plan& Pk = plans[k];
      g.steps = std::max(g.steps, Pk.steps);
      g.gy_gram[0] = std::max(g.gy_gram[0], Pk.rf32 + Pk.rg32);
      g.gy_gram[1] = std::max(g.gy_gram[1], g.oz ? Pk.rf32 + Pk.rg32 : Pk.rf + Pk.rg);
      g.gy_apply = std::max(g.gy_apply, (Pk.mf + 63) / 64 + (Pk.mg + 63) / 64 + (Pk.n + 63) / 64);
      for (int sl = 0; sl < Pk.nslots; ++sl) items.push_back(make_int2(k, sl));
    }
    g.nitems = (int)items.size() - g.item0;
    if (g.gy_apply > 65535) return GSVD_ETOOBIG;
    groups.push_back(g);
  }
  // the tables: problems, column data, items, round-robin tables, states
  const size_t o_prob = 0;
  const size_t o_col = o_prob + align256(sizeof(BlkProb) * P);
  const size_t o_item = o_col + align256(sizeof(BatchCol) * P);
  const size_t o_sw = o_item + align256(sizeof(int2) * items.size());
  size_t o_tab = o_sw + align256(sizeof(BatchSweep) * P);
  std::vector<size_t> toff(P);
  size_t tb = 0;
  std::vector<std::vector<uint16_t>> tabs(P);
  for (int k = 0; k < P; ++k) {
    tabs[k] = round_robin_table(plans[k].neff);
    toff[k] = tb;
    tb += align256(tabs[k].size() * 2);
  }
  const size_t tbytes = o_tab + tb;
  DevBuf buf;
  CK(buf.ensure(tbytes + wtotal, s));
  unsigned char* base = static_cast<unsigned char*>(buf.p);
  unsigned char* wbase = base + tbytes;
  std::vector<unsigned char> host(o_sw);
  BlkProb* hp = reinterpret_cast<BlkProb*>(host.data() + o_prob);
  BatchCol* hc = reinterpret_cast<BatchCol*>(host.data() + o_col);
  std::memcpy(host.data() + o_item, items.data(), sizeof(int2) * items.size());
  for (int k = 0; k < P; ++k) {
    const gsvd_problem& p = ps[idx[k]];
    const Plan& Pk = plans[k];
    const gsvd_config& c = cfgs[k];
    unsigned char* w = wbase + woff[k];
    BlkProb bp{};
    for (int ph = 0; ph < 2; ++ph) {
      const bool fp32 = ph == 0;
      BlkDims& d = bp.d[ph];
      d.mf = Pk.mf; d.mg = Pk.mg; d.n = Pk.n; d.w = Pk.w; d.nblk = Pk.nblk; d.nslots = Pk.nslots;
      const bool oz = !fp32 && c.fp64_gemm >= 1 && oz_supported(Pk.V);
      d.rf = (fp32 || oz) ? Pk.rf32 : Pk.rf;
      d.rg = (fp32 || oz) ? Pk.rg32 : Pk.rg;
      d.trows = 64;
      BlkBuffers& b = bp.b[ph];
      if (fp32) {
        b.F = w + Pk.off_f32; b.ldf = Pk.mf;
        b.G = w + Pk.off_g32; b.ldg = Pk.mg;
        b.Z = w + Pk.off_z32; b.ldz = Pk.n;
      } else {
        b.F = p.F; b.ldf = p.ldf; b.G = p.G; b.ldg = p.ldg; b.Z = p.Z; b.ldz = p.ldz;
      }
      b.partial = w + Pk.off_partial;
      b.ztil = w + Pk.off_ztil;
      b.flags = reinterpret_cast<int*>(w + Pk.off_flags);
      b.ctr = reinterpret_cast<unsigned long long*>(w + Pk.off_ctr);
      b.table = reinterpret_cast<const uint16_t*>(base + o_tab + toff[k]);
      InnerParams& ip = bp.ip[ph];
      ip.eps = fp32 ? EPS32 : EPS64;
      ip.tol = fp32 ? EPS32 * std::sqrt((double)std::max(Pk.mf, Pk.mg)) : 0.0;
      ip.inner_max = fp32 && c.inner_max_sweeps_fp32 > 0 ? c.inner_max_sweeps_fp32 : c.inner_max_sweeps;
      ip.sort = c.sort != 0;
      ip.f32cls = fp32;
      ip.crit2 = c.criterion == 2;
      ip.chol_skip = fp32;
      ip.par32 = fp32 && c.fp32_params != 0;
      ip.enhanced = !fp32 && (c.variant & 1) != 0;
      ip.dscale = !fp32 && (c.variant & 2) != 0;
    }
    bp.steps = Pk.steps;
    bp.tiles = (Pk.mf + 63) / 64 + (Pk.mg + 63) / 64 + (Pk.n + 63) / 64;
    hp[k] = bp;
    BatchCol bc;
    std::memset(&bc, 0, sizeof bc);
    bc.mf = Pk.mf; bc.mg = Pk.mg; bc.n = Pk.n; bc.cplx = Pk.cplx ? 1 : 0; bc.w = Pk.w;
    bc.F = (double*)p.F; bc.ldf = p.ldf; bc.G = (double*)p.G; bc.ldg = p.ldg; bc.Z = (double*)p.Z; bc.ldz = p.ldz;
    bc.sf = p.sigma_f; bc.sg = p.sigma_g; bc.sigma = p.sigma;
    if (mixed) {
      bc.F32 = reinterpret_cast<float*>(w + Pk.off_f32);
      bc.G32 = reinterpret_cast<float*>(w + Pk.off_g32);
      bc.Z32 = reinterpret_cast<float*>(w + Pk.off_z32);
    }
    bc.zdiag = reinterpret_cast<double*>(w + Pk.off_zdiag);
    bc.norms = reinterpret_cast<double*>(w + Pk.off_norms);
    bc.rank = reinterpret_cast<int*>(w + Pk.off_rank);
    bc.work = reinterpret_cast<double*>(w + Pk.off_work);
    bc.status = reinterpret_cast<int*>(w + Pk.off_status);
    bc.ctr = reinterpret_cast<unsigned long long*>(w + Pk.off_ctr);
    hc[k] = bc;
  }
  for (auto& g : groups) {
    const int k0 = items[g.item0].x;
    g.ip[0] = hp[k0].ip[0];
    g.ip[1] = hp[k0].ip[1];
  }
  std::vector<uint16_t> htab(tb / 2, 0);
  for (int k = 0; k < P; ++k) std::memcpy(htab.data() + toff[k] / 2, tabs[k].data(), tabs[k].size() * 2);
  CK(cudaMemcpyAsync(base, host.data(), o_sw, cudaMemcpyHostToDevice, s));
  if (tb) CK(cudaMemcpyAsync(base + o_tab, htab.data(), tb, cudaMemcpyHostToDevice, s));
  const BlkProb* d_prob = reinterpret_cast<const BlkProb*>(base + o_prob);
  const BatchCol* d_col = reinterpret_cast<const BatchCol*>(base + o_col);
  const int2* d_item = reinterpret_cast<const int2*>(base + o_item);
  BatchSweep* d_sw = reinterpret_cast<BatchSweep*>(base + o_sw);
  BatchRule rule;
  rule.cap[0] = h->cfg.fp32_max_sweeps;
  rule.cap[1] = h->cfg.max_sweeps;
  rule.stop_permille = h->cfg.fp32_stop_permille;
  rule.inner_max32 = h->cfg.inner_max_sweeps_fp32 > 0 ? h->cfg.inner_max_sweeps_fp32 : h->cfg.inner_max_sweeps;
  SolveEvents ev;
  cudaEventRecord(ev.e0, s);
  CK(launch_batch_init(d_col, d_sw, P, maxm, maxn, mixed, s));
  if (mixed && rule.cap[0] <= 0) CK(launch_batch_stop(d_sw, P, GSVD_OK, s));  // no FP32 sweeps: straight to the restart

  // one global sweep: every group's outer steps in both precisions, then the
  // convergence tests and the rescales
  auto sweep = [&]() -> cudaError_t {
    cudaError_t e = launch_batch_sweep_begin(d_col, d_sw, P, s);
    for (int ph = mixed ? 0 : 1; ph < 2 && e == cudaSuccess; ++ph) {
      const bool fp32 = ph == 0;
      for (const BatchGroup& g : groups) {
        BlkBatch bt;
        bt.probs = d_prob;
        bt.items = d_item + g.item0;
        bt.sweep = d_sw;
        bt.phase = ph;
        BlkDims dd;
        std::memset(&dd, 0, sizeof dd);
        dd.w = g.w;
        BlkBuffers bb;
        std::memset(&bb, 0, sizeof bb);
        const bool oz = !fp32 && g.oz;
        for (int k = 0; k < g.steps && e == cudaSuccess; ++k) {
          e = oz ? launch_gram_oz(dd, bb, g.cplx, k, s, &bt, g.nitems, g.gy_gram[ph])
                 : launch_gram(dd, bb, g.cplx, fp32, k, s, &bt, g.nitems, g.gy_gram[ph]);
          if (e == cudaSuccess) e = launch_inner(dd, bb, g.cplx, fp32, k, g.ip[ph], s, &bt, g.nitems);
          if (e == cudaSuccess)
            e = oz ? launch_apply_oz(dd, bb, g.cplx, k, s, h->cfg.fp64_gemm == 2, &bt, g.nitems, g.gy_apply)
                   : launch_apply(dd, bb, g.cplx, fp32, k, s, &bt, g.nitems, g.gy_apply);
        }
      }
    }
    if (e == cudaSuccess) e = launch_batch_sweep_end(d_col, d_sw, rule, P, s);
    if (e == cudaSuccess) e = launch_batch_rescale(d_col, d_sw, P, maxn, s);
    return e;
  };
  std::vector<BatchSweep> hs(P);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  struct GraphGuard {
    cudaGraph_t& g;
    cudaGraphExec_t& x;
    ~GraphGuard() {
      if (x) cudaGraphExecDestroy(x);
      if (g) cudaGraphDestroy(g);
    }
  } gguard{graph, gexec};
  bool use_graph = std::getenv("GSVD_BATCH_GRAPH") == nullptr || std::getenv("GSVD_BATCH_GRAPH")[0] != '0';
  int nsweeps = 0;
  for (;;) {
    if (nsweeps == 1 && use_graph) {
      // the launches of a global sweep never change: capture them once
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const cudaError_t e = sweep();
        const cudaError_t ec = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess || ec != cudaSuccess || cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
          cudaGetLastError();
          if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
          if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
          use_graph = false;
        }
      } else {
        cudaGetLastError();
        use_graph = false;
      }
    }
    if (gexec) {
      CK(cudaGraphLaunch(gexec, s));
    } else {
      CK(sweep());
    }
    ++nsweeps;
    CK(cudaMemcpyAsync(hs.data(), d_sw, sizeof(BatchSweep) * P, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (deadline_passed()) {
      CK(launch_batch_stop(d_sw, P, GSVD_ETIMEOUT, s));
      CK(cudaMemcpyAsync(hs.data(), d_sw, sizeof(BatchSweep) * P, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    bool restart = false, active = false;
    for (const BatchSweep& t : hs) {
      restart = restart || (t.state & BST_RESTART);
      active = active || (t.state & (BST_FP32 | BST_FP64));
    }
    if (restart) CK(launch_batch_restart(d_col, d_sw, P, maxm, maxn, s));
    if (!active && !restart) break;
    if (!active) {  // restarts only: they may start FP64 sweeps
      CK(cudaMemcpyAsync(hs.data(), d_sw, sizeof(BatchSweep) * P, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      bool any = false;
      for (const BatchSweep& t : hs) any = any || (t.state & (BST_FP32 | BST_FP64));
      if (!any) break;
    }
  }
  TraceRange phase_fin("gsvd finalize");
  CK(launch_batch_finalize(d_col, d_sw, P, maxm, maxn, s));
  cudaEventRecord(ev.e2, s);
  CK(cudaMemcpyAsync(hs.data(), d_sw, sizeof(BatchSweep) * P, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.e0, ev.e2);
  for (int k = 0; k < P; ++k) {
    gsvd_info& in = infos[idx[k]];
    const BatchSweep& t = hs[k];
    in.status = t.status;
    in.sweeps_fp32 = t.sweeps[0];
    in.sweeps_fp64 = t.sweeps[1];
    in.transf_all = t.tall;
    in.transf_big = t.tbig;
    in.visits = t.visits;
    in.visits_applied = t.visits_applied;
    in.visits_fp32 = t.visits32;
    in.visits_applied_fp32 = t.applied32;
    in.chol_skipped = t.chol_skipped;
    in.path = GSVD_PATH_BLOCKED;
    in.block_w = plans[k].w;
    in.t_total_us = ms * 1e3;  // the whole batched solve: its problems run together
  }
  return GSVD_OK;
}

void worker_loop(gsvd_ctx* h) {
  cudaStream_t s;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  unsigned long long* h_ctr = nullptr;
  cudaMallocHost(&h_ctr, NCTR * sizeof(unsigned long long));
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(h->mu);
      // continuous admission: the oldest queued request starts as soon as the
      // memory budget (and this free worker) allow it
      h->cv.wait(lk, [&] {
        if (h->stop) return true;
        if (h->queue.empty()) return false;
        Request* q = h->reqs[h->queue.front()].get();
        return h->used_bytes + q->bytes <= h->cfg.hbm_budget_bytes || h->inflight == 0;
      });
      if (h->stop && h->queue.empty()) break;
      if (h->queue.empty()) continue;
      const uint64_t t = h->queue.front();
      h->queue.pop_front();
      r = h->reqs[t].get();
      r->state = 1;
      h->used_bytes += r->bytes;
      ++h->inflight;
    }
    gsvd_info info;
    std::memset(&info, 0, sizeof info);
    {
      // the request's workspace comes from the handle's pool and goes back to
      // it when the request ends (stream-ordered: no device-wide
      // synchronisation), so the memory held by the handle stays within the
      // budget that admission counts
      CallScope call(h->pool, h->cfg.timeout_ms);
      DevBuf ws;
      const int st = solve_device(cfg_for(h, &r->prob), &r->prob, &info, ws, h_ctr, s);
      if (st != GSVD_OK && info.status == GSVD_OK) info.status = st;
      ws.release();
      cudaStreamSynchronize(s);
    }
    {
      std::lock_guard<std::mutex> lk(h->mu);
      r->info = info;
      r->state = 2;
      h->used_bytes -= r->bytes;
      --h->inflight;
    }
    h->cv.notify_all();
  }
  cudaFreeHost(h_ctr);
  cudaStreamDestroy(s);
}

}  // namespace

// ------------------------------------------------------------------- ABI ----
extern "C" {

void gsvd_config_default(gsvd_config* c) {
  std::memset(c, 0, sizeof *c);
  c->precision = GSVD_PREC_FP64;
  c->block_w = 0;
  c->max_sweeps = 30;
  c->inner_max_sweeps = 30;
  c->criterion = 1;
  c->sort = 1;
  c->path = GSVD_PATH_AUTO;
  c->order = GSVD_ORDER_ROUND_ROBIN;
  c->fp32_max_sweeps = 30;
  c->timeout_ms = 0;
  c->hbm_budget_bytes = 60ull << 30;
  c->max_inflight = 16;
  c->profile = 0;
  c->inner_max_sweeps_fp32 = 1;
  c->shorten = 1;
  c->fp32_params = 1;
  c->fp64_gemm = 1;
  c->fp32_stop_permille = 50;
  c->variant = 0;
}

int gsvd_create(gsvd_handle* h, const gsvd_config* cfg, void* stream) {
  if (!h) return GSVD_EINVAL;
  gsvd_ctx* c = new (std::nothrow) gsvd_ctx;
  if (!c) return GSVD_ENOMEM;
  if (cfg)
    c->cfg = *cfg;
  else
    gsvd_config_default(&c->cfg);
  if (c->cfg.max_sweeps < 1 || c->cfg.inner_max_sweeps < 1 || c->cfg.fp32_max_sweeps < 0 || c->cfg.timeout_ms < 0 ||
      (c->cfg.criterion != 1 && c->cfg.criterion != 2) || c->cfg.max_inflight < 1 ||
      c->cfg.fp64_gemm < 0 || c->cfg.fp64_gemm > 2 ||
      c->cfg.variant < 0 || c->cfg.variant > 3 ||
      (c->cfg.precision != GSVD_PREC_FP64 && c->cfg.precision != GSVD_PREC_MIXED)) {
    delete c;
    return GSVD_EINVAL;
  }
  c->stream = static_cast<cudaStream_t>(stream);
  *h = c;
  return GSVD_OK;
}

int gsvd_destroy(gsvd_handle h) {
  if (!h) return GSVD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    h->stop = true;
  }
  h->cv.notify_all();
  for (auto& t : h->workers) t.join();
  h->ws.release();
  if (h->pool) {
    cudaStreamSynchronize(h->stream);
    cudaMemPoolDestroy(h->pool);
  }
  if (h->h_ctr) cudaFreeHost(h->h_ctr);
  delete h;
  return GSVD_OK;
}

// First use of a handle on its device: pinned counters and the workspace pool
// (device memory of the current device; memory freed into it stays reserved
// for the next workspace until the handle is destroyed).
static int ensure_pinned(gsvd_handle h) {
  std::lock_guard<std::mutex> lk(h->mu);
  if (!h->h_ctr && cudaMallocHost(&h->h_ctr, NCTR * sizeof(unsigned long long)) != cudaSuccess) return GSVD_ECUDA;
  if (!h->pool) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GSVD_ECUDA;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&h->pool, &props) != cudaSuccess) {
      h->pool = nullptr;
      return GSVD_ECUDA;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  return GSVD_OK;
}

int gsvd_solve(gsvd_handle h, const gsvd_problem* p, gsvd_info* info) {
  if (!h) return GSVD_EINVAL;
  gsvd_info tmp;
  std::memset(&tmp, 0, sizeof tmp);
  int v = validate(p);
  if (v != GSVD_OK) {
    if (info) { *info = tmp; info->status = v; }
    return v;
  }
  int pe = ensure_pinned(h);
  if (pe != GSVD_OK) return pe;
  CallScope call(h->pool, h->cfg.timeout_ms);
  int st = solve_any(cfg_for(h, p), p, &tmp, h->ws, h->h_ctr, h->stream);
  if (st != GSVD_OK && tmp.status == GSVD_OK) tmp.status = st;  // the report carries the returned status
  if (info) *info = tmp;
  return st;
}

int gsvd_solve_batched(gsvd_handle h, const gsvd_problem* ps, int32_t count, gsvd_info* infos) {
  if (!h || count < 0 || (count > 0 && !ps)) return GSVD_EINVAL;
  if (count == 0) return GSVD_OK;
  int pe = ensure_pinned(h);
  if (pe != GSVD_OK) return pe;
  std::vector<gsvd_info> loc(count);
  std::memset(loc.data(), 0, sizeof(gsvd_info) * count);
  std::vector<int> pw, blk;
  for (int k = 0; k < count; ++k) {
    int v = validate(&ps[k]);
    if (v == GSVD_OK && !(is_device_ptr(ps[k].F) && is_device_ptr(ps[k].G) && is_device_ptr(ps[k].Z) &&
                          is_device_ptr(ps[k].sigma_f) && is_device_ptr(ps[k].sigma_g) && is_device_ptr(ps[k].sigma)))
      v = GSVD_EINVAL;
    if (v == GSVD_OK && ps[k].X) v = GSVD_EINVAL;  // right vectors: gsvd_solve and gsvd_submit only
    if (v != GSVD_OK) {
      loc[k].status = v;
      continue;
    }
    Plan P;
    if (!make_plan(h->cfg, ps[k].dtype, ps[k].m_f, ps[k].m_g, ps[k].n, P)) {
      loc[k].status = GSVD_EINVAL;
      continue;
    }
    (P.path == GSVD_PATH_POINTWISE ? pw : blk).push_back(k);
  }
  int first = GSVD_OK;
  // the blocked problems advance together (solve_blocked_batch) on the
  // handle's stream; the pointwise ones run meanwhile in one launch on a
  // stream of their own
  CallScope call(h->pool, h->cfg.timeout_ms);
  std::thread pw_thread;
  if (!pw.empty()) {
    // the pointwise launch on a stream of its own, from a host thread, so that
    // it overlaps the blocked sweeps; it starts after the work already queued
    // on the handle's stream
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess) cudaEventRecord(ready, h->stream);
    int dev = 0;
    cudaGetDevice(&dev);
    pw_thread = std::thread([&, ready, dev]() {
      cudaSetDevice(dev);
      CallScope pcall(h->pool, 0);
      cudaStream_t ps_stream = nullptr;
      int st = GSVD_ECUDA;
      if (cudaStreamCreateWithFlags(&ps_stream, cudaStreamNonBlocking) == cudaSuccess) {
        if (ready) cudaStreamWaitEvent(ps_stream, ready, 0);
        st = solve_pointwise(h->cfg, ps, pw.data(), (int)pw.size(), ps_stream, loc.data());
        cudaStreamSynchronize(ps_stream);
        cudaStreamDestroy(ps_stream);
      }
      if (st != GSVD_OK)
        for (int k : pw) loc[k].status = st;
    });
    if (!blk.empty()) {
      const int st = solve_blocked_batch(h, ps, blk, loc.data(), h->stream);
      if (st != GSVD_OK)
        for (int k : blk)
          if (loc[k].status == GSVD_OK) loc[k].status = st;
    }
    pw_thread.join();
    if (ready) cudaEventDestroy(ready);
  } else if (!blk.empty()) {
    const int st = solve_blocked_batch(h, ps, blk, loc.data(), h->stream);
    if (st != GSVD_OK)
      for (int k : blk)
        if (loc[k].status == GSVD_OK) loc[k].status = st;
  }
  for (int k = 0; k < count; ++k)
    if (loc[k].status != GSVD_OK && first == GSVD_OK) first = loc[k].status;
  if (infos) std::memcpy(infos, loc.data(), sizeof(gsvd_info) * count);
  return first;
}

int gsvd_autotune(gsvd_handle h, int32_t dtype, int64_t m_f, int64_t m_g, int64_t n, int32_t* block_w) {
  if (!h || !block_w || (dtype != GSVD_R64 && dtype != GSVD_C128) || n < 1 || m_f < n || m_g < n ||
      n > 32768 || m_f > (int64_t)1 << 30 || m_g > (int64_t)1 << 30)
    return GSVD_EINVAL;
  *block_w = 0;
  Plan P0;
  if (!make_plan(h->cfg, dtype, m_f, m_g, n, P0)) return GSVD_EINVAL;
  if (P0.path != GSVD_PATH_BLOCKED || h->cfg.block_w != 0) return GSVD_OK;  // nothing to choose
  int pe = ensure_pinned(h);
  if (pe != GSVD_OK) return pe;
  CallScope call(h->pool, 0);
  const bool cplx = dtype == GSVD_C128;
  const int E = cplx ? 2 : 1;
  // a synthetic pair of this shape (hash-based values in [-1, 1))
  DevBuf buf;
  const size_t nF = (size_t)m_f * n * E, nG = (size_t)m_g * n * E, nZ = (size_t)n * n * E;
  CK(buf.ensure(sizeof(double) * (nF + nG + nZ + 3 * (size_t)n) + 256, h->stream));
  double* F = static_cast<double*>(buf.p);
  double* G = F + nF;
  double* Z = G + nG;
  double* v = Z + nZ;
  gsvd_problem p;
  std::memset(&p, 0, sizeof p);
  p.dtype = dtype;
  p.m_f = m_f; p.m_g = m_g; p.n = n;
  p.F = F; p.ldf = m_f; p.G = G; p.ldg = m_g; p.Z = Z; p.ldz = n;
  p.sigma_f = v; p.sigma_g = v + n; p.sigma = v + 2 * n;
  const int cands_r[3] = {8, 16, 32}, cands_c[3] = {4, 8, 16};
  double best_t = 1e300;
  int best_w = 0;
  for (int c = 0; c < 3; ++c) {
    const int w = cplx ? cands_c[c] : cands_r[c];
    if (2 * w > n || blk_vmax(w, cplx) == 0) continue;
    gsvd_config cfg = h->cfg;
    cfg.block_w = w;
    cfg.path = GSVD_PATH_BLOCKED;
    cfg.max_sweeps = 1;
    cfg.fp32_max_sweeps = 1;
    cfg.profile = 0;
    double t = 0.0;
    for (int rep = 0; rep < 2; ++rep) {  // the first run includes one-time set-up
      CK(launch_fill_hash(E * m_f, n, 1u, F, E * m_f, h->stream));
      CK(launch_fill_hash(E * m_g, n, 2u, G, E * m_g, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      gsvd_info info;
      std::memset(&info, 0, sizeof info);
      const auto t0 = std::chrono::steady_clock::now();
      const int st = solve_device(cfg, &p, &info, h->ws, h->h_ctr, h->stream);
      CK(cudaStreamSynchronize(h->stream));
      t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (st != GSVD_OK && st != GSVD_ENOCONV) return st;
    }
    if (t < best_t) {
      best_t = t;
      best_w = w;
    }
  }
  if (best_w == 0) return GSVD_OK;
  {
    std::lock_guard<std::mutex> lk(h->tune_mu);
    h->tuned[tune_key(h->cfg, dtype, m_f, m_g, n)] = best_w;
  }
  *block_w = best_w;
  return GSVD_OK;
}

uint64_t gsvd_workspace_bytes(const gsvd_config* cfg, int32_t dtype, int64_t mf, int64_t mg, int64_t n) {
  gsvd_config c;
  if (cfg)
    c = *cfg;
  else
    gsvd_config_default(&c);
  Plan P;
  if (!shape_ok(dtype, mf, mg, n) || !make_plan(c, dtype, mf, mg, n, P)) return 0;
  return solve_bytes(c, P, mf, mg, n);
}

int gsvd_submit(gsvd_handle h, const gsvd_problem* p, uint64_t* ticket) {
  if (!h || !ticket) return GSVD_EINVAL;
  int v = validate(p);
  if (v != GSVD_OK) return v;
  if (!(is_device_ptr(p->F) && is_device_ptr(p->G) && is_device_ptr(p->Z) && is_device_ptr(p->sigma_f) &&
        is_device_ptr(p->sigma_g) && is_device_ptr(p->sigma)))
    return GSVD_EINVAL;
  Plan P;
  const gsvd_config pc = cfg_for(h, p);
  if (!make_plan(pc, p->dtype, p->m_f, p->m_g, p->n, P)) return GSVD_EINVAL;
  uint64_t bytes = solve_bytes(pc, P, p->m_f, p->m_g, p->n);
  if (p->X)
    bytes += sizeof(double) * (p->dtype == GSVD_C128 ? 2 : 1) *
                 ((uint64_t)(p->m_f + p->m_g) * p->n + (uint64_t)p->n * p->n) + 256;
  if (bytes > h->cfg.hbm_budget_bytes) return GSVD_ETOOBIG;
  int pe = ensure_pinned(h);
  if (pe != GSVD_OK) return pe;
  std::unique_ptr<Request> r(new Request);
  r->prob = *p;
  std::memset(&r->info, 0, sizeof r->info);
  r->bytes = bytes;
  r->state = 0;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    if (h->workers.empty())
      for (int k = 0; k < h->cfg.max_inflight; ++k) h->workers.emplace_back(worker_loop, h);
    *ticket = h->next_ticket++;
    h->reqs[*ticket] = std::move(r);
    h->queue.push_back(*ticket);
  }
  h->cv.notify_all();
  return GSVD_OK;
}

int gsvd_poll(gsvd_handle h, uint64_t ticket, gsvd_info* info) {
  if (!h) return GSVD_EINVAL;
  std::lock_guard<std::mutex> lk(h->mu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return GSVD_EINVAL;
  if (it->second->state != 2) return GSVD_EAGAIN;
  const int st = it->second->info.status;
  if (info) *info = it->second->info;
  h->reqs.erase(it);
  return st;
}

const char* gsvd_strerror(int s) {
  switch (s) {
    case GSVD_OK: return "ok";
    case GSVD_EAGAIN: return "not finished";
    case GSVD_EINVAL: return "invalid argument";
    case GSVD_ENOMEM: return "out of device memory";
    case GSVD_ENOCONV: return "sweep cap reached without convergence";
    case GSVD_ENOTPD: return "pivot block not positive definite (G rank deficient)";
    case GSVD_EOVERFLOW: return "non-finite column norm";
    case GSVD_ETIMEOUT: return "timed out";
    case GSVD_ECUDA: return "CUDA runtime error";
    case GSVD_ETOOBIG: return "request exceeds the memory budget";
    default: return "unknown status";
  }
}

}  // extern "C"
