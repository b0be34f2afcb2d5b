// Long 1-D convolutions by overlap-save FFTs.  Section 2 names FFT-based
// convolution as the kind of fast procedural evaluation of A and A^T that
// makes matrix-free solvers pay; for a length-1000 kernel the direct sum costs
// 2000 flops per output, the FFT route under 100.
//
// The operation is the direct kernel's: out[i] = sum_{u < Lp} wrev[u] in[i + u - D]
// with D = Lp - 1 - shift (in = 0 outside [0, n_in)), i.e. a linear
// convolution of z[m] = in[m - D] with h[v] = wrev[Lp - 1 - v]:
// out[i] = (h * z)[i + Lp - 1].  Overlap-save: for a segment
// seg[t] = z[i0 + t], t < N (N = 4096 or 2048), the circular convolution with h
// (zero-padded to N) equals the linear one for t >= Lp - 1, giving outputs
// i0 .. i0 + V - 1 (V = N - Lp + 1).  Two consecutive segments travel as the
// real and imaginary parts of one complex FFT: h is real, so the inverse
// transform returns the two real convolutions in the two parts.
//
// One CTA of N/16 threads transforms one pair in shared memory:
//   forward: decimation in frequency, radix-16, radix-16 and radix-16 (N =
//            4096) or radix-8 (N = 2048) stages (natural order in,
//            digit-reversed order out);
//   product: with H (the DFT of h, precomputed in FP64 on the host, scaled
//            by 1/N, permuted to the digit-reversed order);
//   inverse: decimation in time, the three stages transposed (digit-reversed
//            in, natural order out).
// No reordering pass is needed.  The first forward stage reads the input from
// global memory and the last inverse stage writes the outputs; the innermost
// stage, the product and its inverse run in registers; four shared-memory
// round trips remain.  Twiddles come from tables rounded from FP64 and laid
// out so that a warp's loads are contiguous (fftconv.cuh).  The 2048-point
// transform (128 threads a pair) is taken when the 4096-point one would give
// fewer pairs than twice the SMs: 2.95x the CTAs for 1.37x the flops at 1000
// taps, so that several CTAs share each SM and hide each other's latency.
#include <mutex>

#include "fftconv.cuh"

namespace cf {
namespace {

template <int N, bool SC>
__global__ void __launch_bounds__(N / 16, N == 4096 ? 2 : 4)
k_conv1d_fft(int64_t n_out, int64_t n_in, int Lp, int64_t D, const float2* __restrict__ H,
             const float2* __restrict__ tw, float alpha, const float* __restrict__ x, float* __restrict__ y,
             bool acc, const float* __restrict__ sin, const float* __restrict__ sout) {
  constexpr int T = N / 16;
  __shared__ __align__(16) float2 buf[fftc::buf_f2<N>()];
  extern __shared__ float tail[];  // acc: y, SC: sout, over this pair's outputs
  const int t = threadIdx.x;
  const int V = N - Lp + 1;
  const int64_t i0 = (int64_t)blockIdx.x * 2 * V;  // first output of the pair
  // what the epilogue reads besides the transform is copied in now, while the
  // transform runs
  const int nout = (int)(n_out - i0 < 2 * (int64_t)V ? n_out - i0 : 2 * (int64_t)V);
  float* ys = tail;
  float* ss = tail + (acc ? 2 * V : 0);
  if (acc || SC) {
    for (int j = t; j < nout; j += T) {
      if (acc) fftc::cp_async4(ys + j, y + i0 + j);
      if (SC) fftc::cp_async4(ss + j, sout + i0 + j);
    }
    fftc::cp_async_commit();
  }
  fftc::pair<N, SC, true, true>(t, blockIdx.x, n_out, n_in, Lp, D, H, tw, alpha, x, y, acc, sin, sout, buf, ys,
                                ss, [] { __syncthreads(); }, acc || SC);
}

template <int N>
cudaError_t raise_limit() {
  const int lim = 2 * 2 * (N - 16 + 1) * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_conv1d_fft<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv1d_fft<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

template <int N>
void launch_n(cudaStream_t s, int64_t n_out, int64_t n_in, int64_t Lp, int64_t shift, const float2* H,
              const float2* tw, float alpha, const float* x, float* y, bool acc, const float* sin,
              const float* sout) {
  const int64_t V = N - Lp + 1;
  const int64_t pairs = (n_out + 2 * V - 1) / (2 * V);
  const int64_t D = Lp - 1 - shift;
  const bool sc = sin || sout;
  const size_t dyn = (size_t)((acc ? 2 * V : 0) + (sc ? 2 * V : 0)) * sizeof(float);
  if (sc)
    k_conv1d_fft<N, true><<<(unsigned)pairs, N / 16, dyn, s>>>(n_out, n_in, (int)Lp, D, H, tw, alpha, x, y, acc,
                                                                 sin, sout);
  else
    k_conv1d_fft<N, false><<<(unsigned)pairs, N / 16, dyn, s>>>(n_out, n_in, (int)Lp, D, H, tw, alpha, x, y,
                                                                  acc, nullptr, nullptr);
}

}  // namespace

// The dynamic tail needs more than the default 48 KB of shared memory next
// to the static transform buffer: the limit is raised once per device, at
// operator creation (outside any stream capture).
cf_err conv1d_fft_prepare(int device) {
  constexpr int kMaxDevices = 64;
  static std::once_flag once[kMaxDevices];
  static cudaError_t err[kMaxDevices];
  if (device < 0 || device >= kMaxDevices) return fail(CF_E_INVALID, "conv1d FFT: device index out of range");
  std::call_once(once[device], [device] {
    err[device] = raise_limit<4096>();
    if (err[device] == cudaSuccess) err[device] = raise_limit<2048>();
  });
  if (err[device] != cudaSuccess)
    return fail(CF_E_CUDA, std::string("conv1d FFT: shared memory limit: ") + cudaGetErrorString(err[device]));
  return CF_OK;
}

void launch_conv1d_fft(cudaStream_t s, int fft_n, int64_t n_out, int64_t n_in, int64_t Lp, int64_t shift,
                       const float2* H, const float2* tw, float alpha, const float* x, float* y, bool acc,
                       const float* sin, const float* sout) {
  if (n_out <= 0) return;
  if (fft_n == 2048)
    launch_n<2048>(s, n_out, n_in, Lp, shift, H, tw, alpha, x, y, acc, sin, sout);
  else
    launch_n<4096>(s, n_out, n_in, Lp, shift, H, tw, alpha, x, y, acc, sin, sout);
}

}  // namespace cf
