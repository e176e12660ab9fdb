// gsvd_noalloc.cu -- an entry point for callers that must not allocate device
// memory: a batch of small GSVDs on the pointwise kernel whose scratch (the
// per-problem descriptor table the kernel reads and the per-problem status
// records it writes) lives in a fixed array compiled into the library instead
// of a cudaMalloc'ed buffer.
//
// Who needs it: code that runs where a device allocation is not allowed or
// not wanted -- a framework that owns all device memory through its own pool,
// a latency-critical loop where cudaMalloc/cudaFree may synchronize the device,
// or a host callback that must not call into the allocator.  The caller still
// provides every input and output buffer (device memory), as for gsvd_solve.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/gsvd.h"
#include "hz_kernels.h"

using namespace hz;

namespace {

constexpr int kNoAllocMaxProblems = GSVD_NOALLOC_MAX_PROBLEMS;
constexpr size_t kDescBytes = sizeof(PwProblem) * kNoAllocMaxProblems;
constexpr size_t kStatBytes = sizeof(PwStats) * kNoAllocMaxProblems;
constexpr size_t kScratchBytes = kDescBytes + kStatBytes;
static_assert(kDescBytes % 256 == 0, "descriptor region keeps 256-byte alignment");

// The scratch: descriptors first, then the status records.  Every GPU that
// loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;                          // one call at a time (shared scratch)
void* g_dev_scratch[kMaxDevices] = {};    // device address of the array, per device
PwProblem g_host_desc[kNoAllocMaxProblems];
PwStats g_host_stat[kNoAllocMaxProblems];

// device memory of the device dev (the current one), or managed memory: the
// kernel runs on dev, so a pointer into another GPU's memory is refused
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int gsvd_solve_small_noalloc(const gsvd_problem* ps, int32_t count, const gsvd_config* cfg,
                                        void* cuda_stream, gsvd_info* infos) {
  if (count < 0 || (count > 0 && !ps)) return GSVD_EINVAL;
  if (count > kNoAllocMaxProblems) return GSVD_ETOOBIG;
  if (count == 0) return GSVD_OK;
  gsvd_config c;
  if (cfg)
    c = *cfg;
  else
    gsvd_config_default(&c);
  if (c.max_sweeps < 1 || (c.criterion != 1 && c.criterion != 2) || c.variant < 0 || c.variant > 3)
    return GSVD_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSVD_ECUDA;
  // every problem must be a valid device problem that fits the pointwise kernel
  // (the shape limits of gsvd_solve come first, so that no row count is
  // narrowed to int before it is known to fit)
  const bool rowcyc = c.order == GSVD_ORDER_ROW_CYCLIC;
  const int64_t kMaxRows = (int64_t)1 << 30;
  int slots = 1;
  for (int k = 0; k < count; ++k) {
    const gsvd_problem& p = ps[k];
    if ((p.dtype != GSVD_R64 && p.dtype != GSVD_C128) || p.n < 1 || p.m_f < p.n || p.m_g < p.n ||
        p.m_f > kMaxRows || p.m_g > kMaxRows || p.ldf < p.m_f || p.ldg < p.m_g || p.ldz < p.n || !p.F || !p.G ||
        !p.Z || !p.sigma_f || !p.sigma_g || !p.sigma || p.X)
      return GSVD_EINVAL;
    if (p.n > 64) return GSVD_ETOOBIG;
    if (!on_device(p.F, dev) || !on_device(p.G, dev) || !on_device(p.Z, dev) || !on_device(p.sigma_f, dev) ||
        !on_device(p.sigma_g, dev) || !on_device(p.sigma, dev))
      return GSVD_EINVAL;
    const int n = (int)p.n;
    slots = std::max(slots, rowcyc ? std::max(1, n / 2) : std::max(1, (n + (n & 1)) / 2));
  }
  for (int k = 0; k < count; ++k) {
    const gsvd_problem& p = ps[k];
    if (pointwise_smem_bytes((int)p.m_f, (int)p.m_g, (int)p.n, p.dtype == GSVD_C128, false, slots) > POINTWISE_SMEM_MAX)
      return GSVD_ETOOBIG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  std::lock_guard<std::mutex> lk(g_mu);
  // set-up, once per device (this device is current): the device address of
  // the array.  Host code must not pass &g_noalloc_scratch to a kernel: on the
  // host that name is a stand-in, not a device address.
  if (!g_dev_scratch[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return GSVD_ECUDA;
    }
    g_dev_scratch[dev] = ptr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_dev_scratch[dev]);
  PwProblem* d_desc = reinterpret_cast<PwProblem*>(base);
  PwStats* d_stat = reinterpret_cast<PwStats*>(base + kDescBytes);
  PwParams prm;
  prm.eps = 1.1102230246251565e-16;
  prm.max_sweeps = c.max_sweeps;
  prm.sort = c.sort != 0;
  prm.f32cls = false;
  prm.crit2 = c.criterion == 2;
  prm.rowcyc = rowcyc;
  prm.enhanced = (c.variant & 1) != 0;
  prm.dscale = (c.variant & 2) != 0;
  // descriptors: real problems first, then complex (one launch per kind);
  // status records start at zero on every call (the array keeps old contents)
  int nreal = 0;
  for (int kind = 0, pos = 0; kind < 2; ++kind)
    for (int k = 0; k < count; ++k) {
      const gsvd_problem& p = ps[k];
      if ((p.dtype == GSVD_C128) != (kind == 1)) continue;
      PwProblem& q = g_host_desc[pos];
      q.F = p.F; q.ldf = p.ldf; q.G = p.G; q.ldg = p.ldg; q.Z = p.Z; q.ldz = p.ldz;
      q.mf = (int)p.m_f; q.mg = (int)p.m_g; q.n = (int)p.n; q.pad = k;
      q.sigma_f = p.sigma_f; q.sigma_g = p.sigma_g; q.sigma = p.sigma;
      q.stats = d_stat + k;
      ++pos;
      if (kind == 0) ++nreal;
    }
  if (cudaMemsetAsync(d_stat, 0, sizeof(PwStats) * count, s) != cudaSuccess ||
      cudaMemcpyAsync(d_desc, g_host_desc, sizeof(PwProblem) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GSVD_ECUDA;
  for (int kind = 0; kind < 2; ++kind) {
    const int first = kind ? nreal : 0, num = kind ? count - nreal : nreal;
    if (num == 0) continue;
    size_t smem = 0;
    for (int k = first; k < first + num; ++k)
      smem = std::max(smem, pointwise_smem_bytes(g_host_desc[k].mf, g_host_desc[k].mg, g_host_desc[k].n, kind == 1,
                                                 false, slots));
    if (launch_pointwise(d_desc + first, num, slots, kind == 1, false, smem, prm, s) != cudaSuccess) return GSVD_ECUDA;
  }
  if (cudaMemcpyAsync(g_host_stat, d_stat, sizeof(PwStats) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GSVD_ECUDA;
  int first_bad = GSVD_OK;
  for (int k = 0; k < count; ++k) {
    if (infos) {
      std::memset(&infos[k], 0, sizeof(gsvd_info));
      infos[k].status = g_host_stat[k].status;
      infos[k].sweeps_fp64 = g_host_stat[k].sweeps;
      infos[k].transf_all = (uint64_t)g_host_stat[k].transf_all;
      infos[k].transf_big = (uint64_t)g_host_stat[k].transf_big;
      infos[k].path = GSVD_PATH_POINTWISE;
    }
    if (g_host_stat[k].status != GSVD_OK && first_bad == GSVD_OK) first_bad = g_host_stat[k].status;
  }
  return first_bad;
}
