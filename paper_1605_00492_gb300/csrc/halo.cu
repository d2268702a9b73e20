// Data movement of the horizontal domain decomposition (partition.cpp): the
// halo exchange of a partitioned level in three steps, as between processes
// (pack each part's send list into its send buffer; move each (sender,
// receiver) segment; unpack each part's receive buffer into its ghost
// columns), and the column copies that gather the parts' restricted
// residuals onto the coarsest level and scatter its correction back.
// Vectors are in the tiled layout of their part (owned tiles, then ghost
// tiles); a buffer entry is one column of nz layers.
#include "hmg_internal.h"

namespace hmg {

namespace {

__device__ __forceinline__ int64_t col_base(int c, int nz) {
  return (int64_t)(c >> 5) * (TW * nz) + (c & 31);
}

// one thread per (entry, layer): buf[e * nz + l] = part[e]'s vector at (col[e], l)
template <typename T>
__global__ void k_halo_pack(int n, int nz, const int32_t* __restrict__ part, const int32_t* __restrict__ col,
                            PartPtrs v, T* __restrict__ buf) {
  const int64_t total = (int64_t)n * nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(i / nz), l = (int)(i - (int64_t)e * nz);
    buf[i] = static_cast<const T*>(v.p[part[e]])[col_base(col[e], nz) + (int64_t)l * TW];
  }
}

template <typename T>
__global__ void k_halo_unpack(int n, int nz, const int32_t* __restrict__ part, const int32_t* __restrict__ col,
                              PartPtrs v, const T* __restrict__ buf) {
  const int64_t total = (int64_t)n * nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(i / nz), l = (int)(i - (int64_t)e * nz);
    static_cast<T*>(v.p[part[e]])[col_base(col[e], nz) + (int64_t)l * TW] = buf[i];
  }
}

// dst column dst0 + c <- src column src0 + c, c < ncols, all layers
template <typename T>
__global__ void k_copy_cols(int ncols, int nz, const T* __restrict__ src, int src0, T* __restrict__ dst, int dst0) {
  const int64_t total = (int64_t)ncols * nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / ncols), c = (int)(i - (int64_t)l * ncols);
    dst[col_base(dst0 + c, nz) + (int64_t)l * TW] = src[col_base(src0 + c, nz) + (int64_t)l * TW];
  }
}

int grid_for(int64_t work) {
  const int64_t b = (work + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

}  // namespace

void launch_halo_pack(int n, int nz, const int32_t* part, const int32_t* col, const PartPtrs& v, void* buf, int dt,
                      cudaStream_t s) {
  if (n <= 0) return;
  if (dt == HMG_FP64) k_halo_pack<double><<<grid_for((int64_t)n * nz), 256, 0, s>>>(n, nz, part, col, v, (double*)buf);
  else k_halo_pack<float><<<grid_for((int64_t)n * nz), 256, 0, s>>>(n, nz, part, col, v, (float*)buf);
}

void launch_halo_unpack(int n, int nz, const int32_t* part, const int32_t* col, const PartPtrs& v,
                        const void* buf, int dt, cudaStream_t s) {
  if (n <= 0) return;
  if (dt == HMG_FP64)
    k_halo_unpack<double><<<grid_for((int64_t)n * nz), 256, 0, s>>>(n, nz, part, col, v, (const double*)buf);
  else k_halo_unpack<float><<<grid_for((int64_t)n * nz), 256, 0, s>>>(n, nz, part, col, v, (const float*)buf);
}

void launch_copy_cols(int ncols, int nz, const void* src, int src0, void* dst, int dst0, int dt, cudaStream_t s) {
  if (ncols <= 0) return;
  if (dt == HMG_FP64)
    k_copy_cols<double><<<grid_for((int64_t)ncols * nz), 256, 0, s>>>(ncols, nz, (const double*)src, src0,
                                                                      (double*)dst, dst0);
  else
    k_copy_cols<float><<<grid_for((int64_t)ncols * nz), 256, 0, s>>>(ncols, nz, (const float*)src, src0,
                                                                     (float*)dst, dst0);
}

}  // namespace hmg
