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

// Block-wide sum of NV (1 or 2) values per thread with few FP64
// instructions (FP64 adds are expensive on GB300): every thread writes its
// values to shared memory, then warp 0 adds blockDim / 32 values per lane and
// finishes with five shuffle steps.  The order is fixed, so the result is
// deterministic.  Valid in thread 0; blockDim.x a multiple of 32.  `sm` is
// shared scratch of NV * blockDim.x doubles (free for the block's use).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[2], double* sm) {
  __syncthreads();  // protect sm from a previous use in the same kernel
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k * blockDim.x + threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int per = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = sm[k * blockDim.x + threadIdx.x];
      for (int j = 1; j < per; ++j) a += sm[k * blockDim.x + threadIdx.x + 32 * j];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
      v[k] = a;
    }
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
// thread has accumulated its values (v[1] is ignored when NV = 1).
// gridDim.x <= RED_MAX_BLOCKS; sm: shared scratch of NV * blockDim.x doubles.
template <int NV>
__device__ __forceinline__ void grid_reduce(double v0, double v1, const Reduce& red, double* sm) {
  __shared__ bool is_last;
  double v[2] = {v0, NV == 2 ? v1 : 0.0};
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) {
    red.partials[2 * blockIdx.x] = v[0];
    red.partials[2 * blockIdx.x + 1] = NV == 2 ? v[1] : 0.0;
    __threadfence();
    unsigned ticket = atomicAdd(red.counter, 1u);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double w[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    w[0] += __ldcg(red.partials + 2 * i);
    if (NV == 2) w[1] += __ldcg(red.partials + 2 * i + 1);
  }
  block_sum<NV>(w, sm);
  if (threadIdx.x == 0) {
    reduce_epilogue(red, w[0], NV == 2 ? w[1] : 0.0);
    *red.counter = 0u;
    __threadfence();
  }
}

// Static shared scratch for kernels of at most 256 threads without dynamic
// shared memory.
#define HMG_RED_SCRATCH(name) __shared__ double name[2 * 256]

}  // namespace hmg
