// sched.cuh -- work items and the persistent-kernel scheduling loop.
//
// The paper balances the element loop across MPI ranks at run time (DLB,
// Sec. 4) because the cost of an element is not known beforehand.  On one GPU
// the same problem appears between CTAs: a persistent grid works through a
// list of work items (runs of `chunk` consecutive elements of one type of one
// type group), either taking the next item from a global counter (dynamic
// work stealing) or following per-CTA queues packed on the host from
// predicted costs.  Every item records how long its CTA spent on it
// (%globaltimer, ns), the measurement a learned cost model trains on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fea_gb300.h"

namespace fea {

// one work item: elements [first, first + count) of parameter-table entry `entry`
struct WorkItem {
  int32_t entry;
  int32_t first;
  int32_t count;
  int32_t pad;
};

struct SchedArgs {
  const WorkItem* items;
  int32_t n_items;
  int32_t mode;           // FEA_SCHED_STEAL or FEA_SCHED_QUEUES
  int32_t* counter;       // STEAL: next item (zeroed before the launch)
  const int32_t* queue;   // QUEUES: item ids
  const int64_t* queue_off;
  uint64_t* item_ns;      // optional per-item duration
  int32_t* item_cta;      // optional per-item CTA
  // batches of meshes (entry = 4 * mesh + type): items left per mesh, the
  // %globaltimer at which each mesh's last item finished, and the launch start
  int32_t* mesh_left;
  uint64_t* mesh_done_ns;
  unsigned long long* start_ns;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The next item of this CTA (-1: done).  Every thread of the CTA calls it; k
// is the CTA's position in its own queue.  s_item is a shared slot.
__device__ __forceinline__ int sched_next(const SchedArgs& S, int& k, int* s_item) {
  if (threadIdx.x == 0) {
    int item = -1;
    if (S.mode == FEA_SCHED_STEAL) {
      const int v = atomicAdd(S.counter, 1);
      item = v < S.n_items ? v : -1;
    } else {
      const int64_t pos = S.queue_off[blockIdx.x] + k;
      if (pos < S.queue_off[blockIdx.x + 1]) {
        const int v = S.queue[pos];
        item = (v >= 0 && v < S.n_items) ? v : -1;
      }
    }
    *s_item = item;
  }
  __syncthreads();
  const int item = *s_item;
  __syncthreads();
  ++k;
  return item;
}

// Called by every thread after the item's work (and a barrier).
__device__ __forceinline__ void sched_record(const SchedArgs& S, int item, int entry, uint64_t t0) {
  if (threadIdx.x == 0) {
    const uint64_t t1 = global_ns();
    if (S.item_ns) S.item_ns[item] = t1 - t0;
    if (S.item_cta) S.item_cta[item] = (int32_t)blockIdx.x;
    if (S.mesh_left) {
      __threadfence();
      if (atomicSub(&S.mesh_left[entry >> 2], 1) == 1 && S.mesh_done_ns) S.mesh_done_ns[entry >> 2] = t1;
    }
  }
}

// launch start of a batch: the earliest CTA start
__device__ __forceinline__ void sched_start(const SchedArgs& S) {
  if (threadIdx.x == 0 && S.start_ns) atomicMin(S.start_ns, (unsigned long long)global_ns());
}

}  // namespace fea
