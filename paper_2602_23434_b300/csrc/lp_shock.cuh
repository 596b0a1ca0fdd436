// lp_shock.cuh -- shock bookkeeping shared by the FP64 and the paired-f32
// LP kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

// Shock bookkeeping of one LP at its new cell: an LP entering a shock cell
// (flag 0 -> 1) is appended to the list with the cell's compression ratio
// and slope index; the flag follows the cell.  Appends are warp-aggregated (one atomic per
// warp); list order is irrelevant, each entry is processed on its own.
static __device__ __forceinline__ void shock_mark(int64_t p, int64_t cell,
                                           const double* __restrict__ shock_r,
                                           const double* __restrict__ shock_q,
                                           uint8_t* __restrict__ shk,
                                           uint32_t* __restrict__ list,
                                           double* __restrict__ rs,
                                           double* __restrict__ qs) {
  const double rr = shock_r[cell];
  const uint8_t st = shk[p];
  const bool take = rr > 0.0 && st == 0;
  if (rr > 0.0) {
    if (st == 0) shk[p] = 1;
  } else if (st != 0) {
    shk[p] = 0;
  }
  const unsigned act = __activemask();
  const unsigned m = __ballot_sync(act, take);
  if (take) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(list, (uint32_t)__popc(m));
    base = __shfl_sync(m, base, leader);
    const uint32_t slot = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
    list[1 + slot] = (uint32_t)p;
    rs[slot] = rr;
    qs[slot] = shock_q[cell];
  }
}

