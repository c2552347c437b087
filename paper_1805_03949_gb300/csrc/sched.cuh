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
  int32_t mode;           // FEA_SCHED_STEAL, FEA_SCHED_QUEUES or FEA_SCHED_QUEUES_STEAL
  int32_t* counter;       // STEAL: next item (zeroed before the launch)
  const int32_t* queue;   // QUEUES*: item ids
  const int64_t* queue_off;
  int32_t* heads;         // QUEUES_STEAL: next position of every queue (zeroed before the launch)
  int32_t n_queues;       // QUEUES_STEAL: number of queues (= grid)
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
//  STEAL          next position of a global counter, into the item list or,
//                 when queue is set (and queue_off is not), into that order
//  QUEUES         position k of the CTA's own queue
//  QUEUES_STEAL   the own queue first; when it is empty, the CTA's threads
//                 read the heads of all queues at once and claim an item of the
//                 first queue (after the own one, in turn) that still has one
__device__ __forceinline__ int sched_next(const SchedArgs& S, int& k, int* s_item) {
  if (S.mode == FEA_SCHED_QUEUES_STEAL) {
    if (threadIdx.x == 0) {
      int item = -1;
      const int q = blockIdx.x;
      const int64_t len = S.queue_off[q + 1] - S.queue_off[q];
      if (*((volatile int32_t*)&S.heads[q]) < len) {
        const int pos = atomicAdd(&S.heads[q], 1);
        if (pos < len) {
          const int v = S.queue[S.queue_off[q] + pos];
          item = (v >= 0 && v < S.n_items) ? v : -1;
        }
      }
      *s_item = item;
    }
    __syncthreads();
    int item = *s_item;
    while (item < 0) {
      __syncthreads();
      if (threadIdx.x == 0) *s_item = INT32_MAX;
      __syncthreads();
      // lowest offset (after the own queue) whose queue still has items
      for (int t = 1 + (int)threadIdx.x; t < S.n_queues; t += blockDim.x) {
        int q = (int)blockIdx.x + t;
        if (q >= S.n_queues) q -= S.n_queues;
        const int64_t len = S.queue_off[q + 1] - S.queue_off[q];
        if (*((volatile int32_t*)&S.heads[q]) < len) {
          atomicMin(s_item, t);
          break;
        }
      }
      __syncthreads();
      const int t = *s_item;
      __syncthreads();
      if (t == INT32_MAX) {
        item = -1;
        break;
      }
      if (threadIdx.x == 0) {
        int q = (int)blockIdx.x + t;
        if (q >= S.n_queues) q -= S.n_queues;
        const int64_t len = S.queue_off[q + 1] - S.queue_off[q];
        const int pos = atomicAdd(&S.heads[q], 1);
        int v = -2;  // lost the race for this queue: scan again
        if (pos < len) {
          v = S.queue[S.queue_off[q] + pos];
          v = (v >= 0 && v < S.n_items) ? v : -2;
        }
        *s_item = v;
      }
      __syncthreads();
      item = *s_item;
      if (item == -2) {  // another CTA took that item first: scan again
        item = -1;
        continue;
      }
      break;
    }
    __syncthreads();
    ++k;
    return item;
  }
  if (threadIdx.x == 0) {
    int item = -1;
    if (S.mode == FEA_SCHED_STEAL) {
      const int v = atomicAdd(S.counter, 1);
      if (v < S.n_items) item = S.queue ? S.queue[v] : v;
      if (item >= S.n_items) item = -1;
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
