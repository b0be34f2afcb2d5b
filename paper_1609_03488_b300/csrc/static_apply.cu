// Allocation-free operator apply for callers that cannot allocate device
// memory.  The scratch the operator kernels need (the dense adjoint's
// per-row-block partial sums, product and Kronecker intermediates) comes from
// one file-scope device array instead of a caller workspace or cudaMalloc.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)CF_STATIC_SCRATCH_BYTES;

// Held by every GPU that loads the library, for the life of the process.
static __device__ __align__(256) float g_static_scratch[kStaticScratchBytes / sizeof(float)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on `device` (which must be current).
// In host code the symbol's name is only a host-side stand-in, so the address
// is looked up once per device and cached.  The cache lives as long as the
// process: after cudaDeviceReset (or a release and re-creation of the
// device's primary context) the module is loaded again and the cached address
// is stale, so this entry point must not be used across such a reset.
cf_err scratch_for(int device, float** out) {
  if (device < 0 || device >= kMaxDevices) return cf::fail(CF_E_INVALID, "cf_op_apply_static: device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cf::cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)", __FILE__, __LINE__);
    g_scratch_ptr[device] = (float*)p;
  }
  *out = g_scratch_ptr[device];
  return CF_OK;
}

}  // namespace

extern "C" cf_err cf_op_apply_static(cf_op* op, int32_t adjoint, float alpha, const float* x,
                                     float* y, int32_t accumulate, void* stream) {
  if (!op || !x || !y) return cf::fail(CF_E_INVALID, "cf_op_apply_static: bad arguments");
  const bool tr = adjoint != 0;
  const size_t need = cf::op_ws_floats(op, tr) * sizeof(float);
  if (need > kStaticScratchBytes)
    return cf::fail(CF_E_INVALID, "cf_op_apply_static: operator needs " + std::to_string(need) +
                                      " bytes of scratch, more than the " +
                                      std::to_string(kStaticScratchBytes) + "-byte static array");
  if (!cf::is_device_ptr(x) || !cf::is_device_ptr(y))
    return cf::fail(CF_E_INVALID, "cf_op_apply_static: x and y must be device memory");
  // an error left pending by earlier work on this thread is reported, not
  // cleared: it belongs to the caller
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return cf::cuda_fail(pending, "cf_op_apply_static: pending CUDA error from earlier work", __FILE__, __LINE__);
  int prev = -1;
  cudaGetDevice(&prev);
  const int dev = op->device;
  if (prev != dev) cudaSetDevice(dev);
  float* scratch = nullptr;
  cf_err r = scratch_for(dev, &scratch);
  if (r == CF_OK) {
    // Every scratch element the kernels read is written earlier in the same
    // call, so nothing needs clearing between calls.
    cudaStream_t s = stream ? (cudaStream_t)stream : op->ctx->stream;
    cf::op_apply(op, tr, alpha, x, y, accumulate != 0, scratch, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) r = cf::cuda_fail(e, "cf_op_apply_static launch", __FILE__, __LINE__);
  }
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return r;
}
