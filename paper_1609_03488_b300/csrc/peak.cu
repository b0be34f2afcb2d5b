// Measured fused multiply-add rate of the GPU (float32 or float64): the
// denominator of the ALU-bound rooflines (the convolution leaves).  Every
// thread of a full-occupancy grid runs 8 independent FMA chains
// v <- v * a + b with |a| < 1, so no chain overflows and none can be folded
// away (a, b arrive as kernel arguments, the sums are conditionally stored).
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(T a, T b, int iters, T* __restrict__ sink) {
  T v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = (T)(threadIdx.x + j) * (T)1e-3;
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = fma(v[j], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  if (s == (T)-1) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

template <typename T>
cf_err run(cf_ctx* ctx, int iters, double* flops_per_s) {
  int per_sm = 0;
  CF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T>, kThreads, 0));
  per_sm = std::max(per_sm, 1);
  const int grid = ctx->sm_count * per_sm;
  T* sink = nullptr;
  CF_CUDA(cudaMallocAsync((void**)&sink, sizeof(T) * grid, ctx->stream));
  cudaEvent_t e0, e1;
  CF_CUDA(cudaEventCreate(&e0));
  CF_CUDA(cudaEventCreate(&e1));
  const T a = (T)0.999999, b = (T)1e-6;
  float best = 1e30f;
  cf_err r = CF_OK;
  for (int rep = 0; rep < 4 && r == CF_OK; ++rep) {   // rep 0 warms up
    cudaEventRecord(e0, ctx->stream);
    k_fma_rate<T><<<grid, kThreads, 0, ctx->stream>>>(a, b, iters, sink);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      r = cf::cuda_fail(e, "k_fma_rate", __FILE__, __LINE__);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaFreeAsync(sink, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != CF_OK) return r;
  const double flops = 2.0 * kChains * (double)iters * (double)grid * kThreads;
  *flops_per_s = flops / (best * 1e-3);
  return CF_OK;
}

}  // namespace

extern "C" cf_err cf_measure_fma_rate(cf_ctx* ctx, int32_t fp64, double* flops_per_s) {
  if (!ctx || !flops_per_s) return cf::fail(CF_E_INVALID, "cf_measure_fma_rate: NULL argument");
  CF_CUDA(cudaSetDevice(ctx->device));
  // ~10 ms a launch at the nominal rates (float64 runs far fewer FMA units)
  return fp64 ? run<double>(ctx, 1 << 11, flops_per_s) : run<float>(ctx, 1 << 17, flops_per_s);
}
