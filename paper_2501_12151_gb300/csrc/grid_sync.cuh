// Grid barrier of the library's cooperative kernels (all CTAs resident).
//
// State: a monotonically increasing arrival counter (zeroed before the launch, never reset) and a
// generation word whose low 31 bits count completed barriers and whose top bit marks an error.
// Every CTA keeps its own count of barriers passed (`idx`, identical on all CTAs), so barrier
// idx + 1 is complete when the counter reaches (idx + 1) x (number of arrivals per barrier):
// thread 0 fences (release), adds its arrival, and either completes the generation (the last
// arrival) or polls it, then fences again (acquire).  A wait is bounded (kGridWaitNs): on expiry
// the CTA sets the error bit, which every other CTA sees in the word it polls, and all of them
// leave at their next barrier.  Compared with a counter that is reset by the last arrival, this
// takes no extra read of the generation before arriving, no reset, and no separate read of an
// error flag afterwards.
//
// Two-level arrival (grid_sync_groups): the CTAs of a group count on the group's own line and the
// last of each group counts on the top counter, so no address sees more than ~32 atomics per
// barrier.
#pragma once

#include "internal.h"

namespace tnfem {

constexpr unsigned long long kGridWaitNs = 2000000000ull;  // 2 s bound on one barrier wait
constexpr unsigned int kGridErrBit = 0x80000000u;

// Release / acquire fence at GPU scope: with the arrival atomic after it, the CTA's earlier writes
// (ordered before thread 0 by the CTA barrier) become visible to every CTA that observes the
// completed generation and fences again before reading.  Weaker and cheaper than the sequentially
// consistent __threadfence(), and all this pattern needs.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

struct GridSync {
  unsigned int arrive;  // arrivals since the launch (top level)
  unsigned int gen;     // completed barriers | error bit
};

// Waits until barrier `target` is complete or an error is flagged; thread 0 only.  Returns false
// on error (its own timeout or another CTA's).
__device__ __forceinline__ bool grid_wait_gen(GridSync* gs, unsigned int target,
                                              unsigned long long limit_ns = kGridWaitNs) {
  volatile unsigned int* vgen = &gs->gen;
  const unsigned long long t0 = global_ns();
  unsigned int spins = 0;
  for (;;) {
    const unsigned int v = *vgen;
    if (v & kGridErrBit) return false;
    if (v >= target) return true;
    if ((++spins & 63u) == 0 && global_ns() - t0 > limit_ns) {
      atomicOr(&gs->gen, kGridErrBit);
      return false;
    }
  }
}

// Flat barrier: every CTA arrives on gs->arrive.  idx: barriers this CTA has passed (all threads
// keep it; it is incremented here).  True when all CTAs arrived and no error is flagged.
__device__ __forceinline__ bool grid_sync(GridSync* gs, unsigned int& idx, unsigned long long limit_ns = kGridWaitNs) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int target = idx + 1;
    fence_acq_rel_gpu();
    const unsigned int old = atomicAdd(&gs->arrive, 1u);
    bool ok;
    if (old == target * gridDim.x - 1) {
      ok = (atomicAdd(&gs->gen, 1u) & kGridErrBit) == 0;
    } else {
      ok = grid_wait_gen(gs, target, limit_ns);
    }
    fence_acq_rel_gpu();
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  ++idx;
  return s_ok != 0;
}

// Two-level barrier: group counters at gcount[32 * g] (separate 128-byte lines), groups of
// ceil(gridDim.x / kGridGroupsMax) CTAs.
constexpr int kGridGroupsMax = 32;
__host__ __device__ inline int grid_group_size(int ncta) { return (ncta + kGridGroupsMax - 1) / kGridGroupsMax; }

__device__ __forceinline__ bool grid_sync_groups(GridSync* gs, unsigned int* gcount, unsigned int& idx) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int target = idx + 1;
    const int gsz = grid_group_size(gridDim.x);
    const int grp = blockIdx.x / gsz;
    const unsigned int ngrp = (gridDim.x + gsz - 1) / gsz;
    const unsigned int in_grp = (unsigned int)min(gsz, (int)gridDim.x - grp * gsz);
    fence_acq_rel_gpu();
    bool ok;
    bool last = false;
    if (atomicAdd(gcount + 32 * grp, 1u) == target * in_grp - 1) {
      if (atomicAdd(&gs->arrive, 1u) == target * ngrp - 1) {
        ok = (atomicAdd(&gs->gen, 1u) & kGridErrBit) == 0;
        last = true;
      }
    }
    if (!last) ok = grid_wait_gen(gs, target);
    fence_acq_rel_gpu();
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  ++idx;
  return s_ok != 0;
}

}  // namespace tnfem
