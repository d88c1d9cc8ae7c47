// Merged launches over many independent problem instances.
//
// A merged launch runs one level operation (an operator apply, the star products, a
// transfer, a GMRES step, the coarse solve) for every instance of a batch at once.
// Its grid is the concatenation of the instances' own grids, a flattened
// (instance, tile) work list: instance i owns blocks start[i] .. start[i+1]-1, and each
// of those blocks runs the single-instance kernel body with its index inside the range
// and the range's length in place of blockIdx.x and gridDim.x.  Kernels that are
// persistent for one instance (grid-stride loops over star groups) stay persistent
// within their instance's share, and the shares are sized so that the whole launch
// fills the GPU once.  The per-instance arguments travel in the kernel's parameter
// space (__grid_constant__, up to kBatchMax instances per launch); a block finds its
// instance by a binary search over the offsets, which sit in the constant bank.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "pdl.cuh"

namespace als {

constexpr int kBatchMax = 64;   // instances per merged launch (more are split into several)

template <typename A>
struct BatchTab {
  int count;
  unsigned start[kBatchMax + 1];
  A a[kBatchMax];
};

// the instance owning block b: the largest i with start[i] <= b
template <typename A>
__device__ __forceinline__ int batch_slot(const BatchTab<A>& t, unsigned b) {
  int lo = 0, hi = t.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One merged launch per group of at most kBatchMax items: items[i] gets blocks[i]
// blocks (items with none are left out).  Returns the number of launches.
template <typename A>
int launch_batch(void (*kernel)(BatchTab<A>), const std::vector<A>& items, const std::vector<unsigned>& blocks,
                 unsigned threads, size_t smem, cudaStream_t s) {
  static_assert(sizeof(BatchTab<A>) <= 32000, "merged-launch table exceeds the kernel parameter space");
  int launches = 0;
  BatchTab<A>* t = new BatchTab<A>();
  size_t i = 0;
  while (i < items.size()) {
    t->count = 0;
    unsigned total = 0;
    for (; i < items.size() && t->count < kBatchMax; ++i) {
      if (blocks[i] == 0) continue;
      t->start[t->count] = total;
      t->a[t->count] = items[i];
      total += blocks[i];
      ++t->count;
    }
    t->start[t->count] = total;
    if (t->count == 0) continue;
    launch_pdl(kernel, total, threads, smem, s, *t);
    ++launches;
  }
  delete t;
  return launches;
}

// Shares of a persistent merged launch: instance i has work[i] units (star groups)
// and may use at most cap_i = min(work[i], per_instance_cap) blocks; the launch aims
// at `capacity` blocks in all (the resident CTAs of the GPU), split in proportion to
// the work, at least one block per instance with work.
inline std::vector<unsigned> persistent_shares(const std::vector<long long>& work, long long capacity,
                                               long long per_instance_cap) {
  long long W = 0;
  for (long long w : work) W += w;
  std::vector<unsigned> out(work.size(), 0u);
  if (W <= 0) return out;
  for (size_t i = 0; i < work.size(); ++i) {
    if (work[i] <= 0) continue;
    long long b = (capacity * work[i] + W - 1) / W;
    if (b < 1) b = 1;
    if (b > work[i]) b = work[i];
    if (b > per_instance_cap) b = per_instance_cap;
    out[i] = (unsigned)b;
  }
  return out;
}

}  // namespace als
