// blk_pair.cuh -- the pair of column blocks that one CTA of the blocked
// sweep kernels works on (shared by the FP32/FP64 and the tensor-core
// emulated kernels).
#pragma once
#include <cstdint>

#include "hz_kernels.h"

namespace hz {

// Columns of the pair (p, q): block p covers [cp, cp + wp), block q covers
// [cq, cq + wq); pair column c < wp is column cp + c, else cq + c - wp.
struct PairCols {
  int cp, wp, cq, wq, bb;
  __device__ __forceinline__ int gcol(int c) const { return c < wp ? cp + c : cq + (c - wp); }
};

// The pair of this step's slot from the ordering table; false for the idle
// slot of an odd block count.
__device__ __forceinline__ bool load_pair(const BlkDims& d, const BlkBuffers& b, int step, int slot,
                                          PairCols& pc) {
  const uint16_t* pr = b.table + ((size_t)step * d.nslots + slot) * 2;
  const int p = pr[0], q = pr[1];
  if (p >= d.nblk || q >= d.nblk) return false;
  pc.cp = p * d.w;
  pc.wp = min(d.w, d.n - pc.cp);
  pc.cq = q * d.w;
  pc.wq = min(d.w, d.n - pc.cq);
  pc.bb = pc.wp + pc.wq;
  return true;
}

// The CTA's problem and pair slot: in a one-problem launch the slot is the
// grid-x index and d, b (and prm) are the kernel's own; in a batched launch
// they come from the item's problem.  False: nothing to do in this launch.
__device__ __forceinline__ bool batch_item(const BlkBatch& bt, int xi, int step, BlkDims& d, BlkBuffers& b,
                                           int& slot, InnerParams* prm = nullptr) {
  if (!bt.probs) {
    slot = xi;
    return true;
  }
  const int2 it = bt.items[xi];
  if (!(bt.sweep[it.x].state & (1 << bt.phase))) return false;
  const BlkProb& P = bt.probs[it.x];
  if (step >= P.steps) return false;
  d = P.d[bt.phase];
  b = P.b[bt.phase];
  if (prm) *prm = P.ip[bt.phase];
  slot = it.y;
  return true;
}

}  // namespace hz
