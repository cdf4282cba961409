// The persistent form of a batch step's sweeps (csrc/ebit_server.cu): both
// split sweeps of many square grids in one launch of resident blocks.
#pragma once
#include "ebit_tile.cuh"

namespace ebit {

// Both sweeps of many square grids in one persistent launch.  Work item w in
// [0, 2 n_items) is tile items[w mod n_items] of the grids' first sweep
// (w < n_items) or of their second, and blocks take items in increasing w
// from one counter.  A second-sweep tile of grid g starts once every tile of
// g's first sweep has been counted; each of those items was taken before it,
// by a block that waits for nothing, so the wait ends.  It is bounded all the
// same (budget_ns of the global timer, and a poll count the budget fixes even
// if the timer stood still): a tile whose wait runs out is skipped and its
// grid's status word gets ST_TIMEOUT.  The second sweep reads what the first
// wrote in this launch, so the state is loaded through L2 (LD = 1).
struct PersistCtl {
  unsigned* ctl;         // [0]: next work item; [1 + g]: first-sweep tiles of grid g done
  const unsigned* need;  // per grid: the count its second-sweep tiles wait for
  int n_items, n_grids;
  unsigned long long budget_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 1 once *count >= need (then fenced: what the counted blocks wrote before
// their count is visible), 0 when the budget runs out first.
__device__ __forceinline__ int wait_count(const unsigned* count, unsigned need,
                                          unsigned long long budget_ns) {
  const unsigned long long t0 = global_ns();
  const unsigned long long max_polls = budget_ns / 32 + 64;
  unsigned sleep_ns = 32;
  for (unsigned long long k = 0; k < max_polls; ++k) {
    if (*(volatile const unsigned*)count >= need) {
      __threadfence();
      return 1;
    }
    if (global_ns() - t0 > budget_ns) break;
    __nanosleep(sleep_ns);
    if (sleep_ns < 1024) sleep_ns <<= 1;
  }
  return 0;
}

// One work item: the tile in the direction its grid's split order gives.
// Not inlined, so that the tile is register-allocated as in the one-item
// kernels rather than together with the loop around it.
template <typename R>
__device__ __noinline__ void persistent_tile(const SweepDesc<R, 0>& X, const SweepDesc<R, 1>& Y,
                                             int tx, int ty) {
  if (X.active) {
    const GView<R, 0, 1> G{X.G.K, X.G.Z, X.G.sH, X.G.sV, X.G.w, X.G.d, X.G.lam};
    sweep_tile<R, 0, 1, batch_cand_cap<R>()>(G, X.out, X.line_only, X.ctr, X.cfl_bits, X.status,
                                             tx * kTI, ty * kTJ);
  } else {
    const GView<R, 1, 1> G{Y.G.K, Y.G.Z, Y.G.sH, Y.G.sV, Y.G.w, Y.G.d, Y.G.lam};
    sweep_tile<R, 1, 1, batch_cand_cap<R>()>(G, Y.out, Y.line_only, Y.ctr, Y.cfl_bits, Y.status,
                                             tx * kTI, ty * kTJ);
  }
}

template <typename R>
__global__ void __launch_bounds__(tile_threads<R>(), tile_min_blocks<R>())
k_sweep_persistent(const SweepDesc<R, 0>* __restrict__ dx, const SweepDesc<R, 1>* __restrict__ dy,
                   const WorkItem* __restrict__ items, PersistCtl P) {
  __shared__ int s_w, s_go;
  if (threadIdx.x == 0) s_w = (int)atomicAdd(P.ctl, 1u);
  __syncthreads();
  for (;;) {
    const int w = s_w;
    if (w >= 2 * P.n_items) return;  // the same in every thread
    const int second = w >= P.n_items ? 1 : 0;
    const WorkItem it = items[w - second * P.n_items];
    const SweepDesc<R, 0>& X = dx[second * P.n_grids + it.grid];
    const SweepDesc<R, 1>& Y = dy[second * P.n_grids + it.grid];
    if (second) {
      if (threadIdx.x == 0) s_go = wait_count(P.ctl + 1 + it.grid, P.need[it.grid], P.budget_ns);
      __syncthreads();
    }
    if (!second || s_go) {
      persistent_tile<R>(X, Y, it.tx, it.ty);
    } else if (threadIdx.x == 0) {
      atomicOr(X.status, ST_TIMEOUT);
    }
    // the block's next item (every thread read s_w before a barrier since:
    // the tile's, or the wait's); a first-sweep tile's writes are fenced
    // before its count
    if (second) {
      if (threadIdx.x == 0) s_w = (int)atomicAdd(P.ctl, 1u);
    } else {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        atomicAdd(P.ctl + 1 + it.grid, 1u);
        s_w = (int)atomicAdd(P.ctl, 1u);
      }
    }
    __syncthreads();
  }
}

}  // namespace ebit
