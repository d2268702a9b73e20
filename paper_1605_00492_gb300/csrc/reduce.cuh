// Deterministic two-value grid reduction with a device-side epilogue.
//
// Every block reduces its threads' values with warp shuffles (fixed order),
// writes one partial pair, and the last block to finish (ticket counter)
// sums the partials in block order and applies the Krylov epilogue: the
// scalars alpha and beta are formed on the device once, so no kernel divides
// per element and the host never has to read a scalar to continue.
#pragma once

#include "hmg_internal.h"

namespace hmg {

__device__ __forceinline__ void warp_sum2(double& a, double& b) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
}

// Block-wide sum; the result is valid in thread 0.  blockDim.x <= 1024.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  warp_sum2(a, b);
  __syncthreads();  // protect sa/sb from a previous use in the same kernel
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    warp_sum2(a, b);
  }
}

__device__ __forceinline__ void reduce_epilogue(const Reduce& red, double s0, double s1) {
  double* sc = red.sc;
  switch (red.epilogue) {
    case EPI_STORE0:
      sc[red.slot] = s0;
      sc[red.slot + 1] = s1;
      if (!isfinite(s0) || !isfinite(s1)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_NONFINITE);
      break;
    case EPI_ALPHA:
      sc[S_PQ] = s0;
      if (!isfinite(s0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_NONFINITE);
      else if (!(s0 > 0.0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_BREAKDOWN);
      sc[S_ALPHA] = sc[S_RZ] / s0;
      break;
    case EPI_RR:
      sc[S_RR] = s0;
      if (!isfinite(s0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_NONFINITE);
      break;
    case EPI_BETA_CG:
      if (!isfinite(s0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_NONFINITE);
      else if (!(s0 > 0.0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_BREAKDOWN);
      sc[S_BETA] = s0 / sc[S_RZ];
      sc[S_RZNEW] = s0;
      sc[S_RZ] = s0;
      break;
    case EPI_BETA_FCG:
      if (!isfinite(s0) || !isfinite(s1)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_NONFINITE);
      else if (!(s0 > 0.0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_BREAKDOWN);
      sc[S_BETA] = -sc[S_ALPHA] * s1 / sc[S_RZ];
      sc[S_ZQ] = s1;
      sc[S_RZNEW] = s0;
      sc[S_RZ] = s0;
      break;
    case EPI_INIT_RZ:
      if (!isfinite(s0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_NONFINITE);
      else if (!(s0 > 0.0)) sc[S_FLAG] = (double)((int)sc[S_FLAG] | F_BREAKDOWN);
      sc[S_RZ] = s0;
      break;
    default:
      break;
  }
}

// Called by every thread of every block of the grid exactly once, after the
// thread has accumulated its (a, b).  gridDim.x <= RED_MAX_BLOCKS.
__device__ __forceinline__ void grid_reduce2(double a, double b, const Reduce& red) {
  __shared__ bool is_last;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    red.partials[2 * blockIdx.x] = a;
    red.partials[2 * blockIdx.x + 1] = b;
    __threadfence();
    unsigned ticket = atomicAdd(red.counter, 1u);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    x += __ldcg(red.partials + 2 * i);
    y += __ldcg(red.partials + 2 * i + 1);
  }
  block_sum2(x, y);
  if (threadIdx.x == 0) {
    reduce_epilogue(red, x, y);
    *red.counter = 0u;
    __threadfence();
  }
}

}  // namespace hmg
