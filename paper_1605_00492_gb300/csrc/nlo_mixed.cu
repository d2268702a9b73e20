// Kernels of the next-to-lowest-order velocity-pressure system (Eq.
// PressureVelocitySystem at NLO): the assembled operator and the two outer
// factors of the Schur-complement preconditioner (Eq. SchurComplement with
// the lumped inverse of Eq. LumpedMass) are CSR products, the form in which
// the paper's implementation holds them.  Rows have 10 to 50 entries; a few
// lanes share a row, each accumulating a strided part of it, and the partial
// sums are combined by shuffles in a fixed order, so the result does not
// depend on scheduling.
#include "hmg_internal.h"

namespace hmg {

namespace {

// Lanes per row.  On GB300 every FP64 warp instruction costs the same
// whatever its active lanes, and the FP64 pipe bounds this product: per row
// it issues the FMAs, the shuffle sum (log2 LPR adds per warp) and the
// epilogue (per warp).  Eight lanes per row made the sums and epilogues
// dominate (1.29 ms per product of the r4x64 system against 0.81 ms with
// four lanes); two lanes issue fewer sums still.
constexpr int LPR = 2;
constexpr unsigned FULL = 0xffffffffu;

// y[i] = (y0[i] + alpha * sum_j A_ij x_j) * s[i]   (y0, s optional).  TV, TX:
// types of the matrix values and of x; TA: the accumulation (the mixed form's
// preconditioner factors run in FP32 on the FP32 pipe); y, y0, s are FP64.
template <typename TV, typename TX, typename TA>
__global__ void k_csr_spmv(int64_t nrows, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const TV* __restrict__ val, const TX* __restrict__ x, double alpha,
                           const double* __restrict__ y0, const double* __restrict__ s, double* __restrict__ y) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = gid / LPR;
  const int sub = (int)(gid % LPR);
  TA acc = TA(0);
  if (row < nrows) {
    // (four entries per lane loaded ahead of their use measured slower: 1.48
    // against 1.29 ms for the r4x64 system with eight lanes per row)
    const int64_t p1 = ptr[row + 1];
    for (int64_t p = ptr[row] + sub; p < p1; p += LPR) acc = fma(TA(val[p]), TA(x[col[p]]), acc);
  }
#pragma unroll
  for (int off = LPR / 2; off > 0; off >>= 1) acc += __shfl_down_sync(FULL, acc, off, LPR);
  if (row < nrows && sub == 0) {
    double v = double(acc);
    if (y0) v = fma(alpha, v, y0[row]);
    else if (alpha != 1.0) v = alpha * v;
    if (s) v *= s[row];
    y[row] = v;
  }
}

template <typename TY>
__global__ void k_mul(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                      TY* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = TY(a[i] * b[i]);
}

int grid_of(int64_t threads) { return (int)((threads + 255) / 256); }

}  // namespace

void launch_csr_spmv(const DevCsr& A, const double* x, double alpha, const double* y0, const double* s, double* y,
                     cudaStream_t st) {
  k_csr_spmv<double, double, double><<<grid_of(A.nrows * LPR), 256, 0, st>>>(A.nrows, A.ptr, A.col, A.val, x, alpha,
                                                                           y0, s, y);
}

void launch_csr_spmv32(const DevCsr& A, const float* val32, const float* x, double alpha, const double* y0,
                       const double* s, double* y, cudaStream_t st) {
  k_csr_spmv<float, float, float><<<grid_of(A.nrows * LPR), 256, 0, st>>>(A.nrows, A.ptr, A.col, val32, x, alpha,
                                                                        y0, s, y);
}

void launch_mul(int64_t n, const double* a, const double* b, double* y, cudaStream_t st) {
  k_mul<double><<<grid_of(n), 256, 0, st>>>(n, a, b, y);
}

void launch_mul32(int64_t n, const double* a, const double* b, float* y, cudaStream_t st) {
  k_mul<float><<<grid_of(n), 256, 0, st>>>(n, a, b, y);
}

}  // namespace hmg
