// hmg_apply_noalloc: the COLUMN-layout FP64 operator application of
// hmg_apply, with its two tiled staging vectors held in a fixed device array
// of this file instead of memory allocated for the context.  It calls no
// allocating function (no cudaMalloc / cudaFree, no library allocator).
#include <exception>
#include <mutex>
#include <new>
#include <string>

#include "hmg_internal.h"

using namespace hmg;

namespace {

// Two staging vectors of at most HMG_NOALLOC_MAX_CELLS doubles each (8 MiB in
// total), resident on every device that loads the library until the process
// exits.
__device__ __align__(256) double g_noalloc_scratch[2 * HMG_NOALLOC_MAX_CELLS];

constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the array on the current device, looked up once per
// device (host code cannot use the array's name as a device pointer).
cudaError_t scratch_on_current_device(double** out, std::string& why) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return e;
  }
  if (dev < 0 || dev >= MAX_DEVICES) {
    why = "device ordinal out of range";
    return cudaErrorInvalidDevice;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return e;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

namespace {

hmg_status apply_noalloc(hmg_ctx* ctx, int level, const double* x, double* y, void* stream) {
  if (level < 0 || level >= (int)ctx->lv.size()) {
    ctx->err = "bad level";
    return HMG_ERR_INVALID_ARG;
  }
  if (!x || !y || x == y) {
    ctx->err = "x and y must be distinct non-NULL device pointers";
    return HMG_ERR_INVALID_ARG;
  }
  if (!ctx->assembled) {
    ctx->err = "operator not assembled (call hmg_assemble_helmholtz)";
    return HMG_ERR_STATE;
  }
  const Level& L = ctx->lv[level];
  if (L.Np > (int64_t)HMG_NOALLOC_MAX_CELLS) {
    ctx->err = "hmg_apply_noalloc: level has " + std::to_string(L.Np) + " padded cells, more than the " +
               std::to_string((long long)HMG_NOALLOC_MAX_CELLS) + " its fixed scratch holds";
    return HMG_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  std::string why;
  if (scratch_on_current_device(&scratch, why) != cudaSuccess) {
    ctx->err = why;
    return HMG_ERR_CUDA;
  }
  // Every entry of both staging vectors is written before it is read
  // (padding included), so nothing left by an earlier call is used.
  double* xt = scratch;
  double* yt = scratch + HMG_NOALLOC_MAX_CELLS;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The three launches are traced like hmg_apply's (hmg_profile_start).
  int rec = trace_begin(ctx, HMG_K_LAYOUT, level, s);
  launch_to_tiled(L, HMG_FP64, x, xt, s);
  trace_end(ctx, rec, s);
  rec = trace_begin(ctx, HMG_K_APPLY, level, s);
  launch_apply(L, HMG_FP64, xt, yt, nullptr, s);
  trace_end(ctx, rec, s);
  rec = trace_begin(ctx, HMG_K_LAYOUT, level, s);
  launch_to_column(L, HMG_FP64, yt, y, s);
  trace_end(ctx, rec, s);
  ctx->launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string("hmg_apply_noalloc: ") + cudaGetErrorString(e);
    return HMG_ERR_CUDA;
  }
  ctx->err.clear();
  return HMG_OK;
}

}  // namespace

// No exception leaves the C ABI: host allocation failures (the error strings)
// map to HMG_ERR_OOM, a CUDA error raised while tracing to HMG_ERR_CUDA.
extern "C" hmg_status hmg_apply_noalloc(hmg_ctx* ctx, int level, const double* x, double* y, void* stream) {
  if (!ctx) return HMG_ERR_INVALID_ARG;
  try {
    return apply_noalloc(ctx, level, x, y, stream);
  } catch (const std::bad_alloc&) {
    return HMG_ERR_OOM;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return HMG_ERR_CUDA;
  } catch (...) {
    ctx->err = "hmg_apply_noalloc: CUDA error while tracing";
    return HMG_ERR_CUDA;
  }
}
