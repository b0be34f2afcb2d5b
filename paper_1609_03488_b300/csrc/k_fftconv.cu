// Long 1-D convolutions by overlap-save FFTs.  Section 2 names FFT-based
// convolution as the kind of fast procedural evaluation of A and A^T that
// makes matrix-free solvers pay; for a length-1000 kernel the direct sum costs
// 2000 flops per output, the FFT route under 100.
//
// The operation is the direct kernel's: out[i] = sum_{u < Lp} wrev[u] in[i + u - D]
// with D = Lp - 1 - shift (in = 0 outside [0, n_in)), i.e. a linear
// convolution of z[m] = in[m - D] with h[v] = wrev[Lp - 1 - v]:
// out[i] = (h * z)[i + Lp - 1].  Overlap-save: for a segment
// seg[t] = z[i0 + t], t < N (N = 4096), the circular convolution with h
// (zero-padded to N) equals the linear one for t >= Lp - 1, giving outputs
// i0 .. i0 + V - 1 (V = N - Lp + 1).  Two consecutive segments travel as the
// real and imaginary parts of one complex FFT: h is real, so the inverse
// transform returns the two real convolutions in the two parts.
//
// One CTA of 256 threads transforms one pair in shared memory:
//   forward: decimation in frequency, three radix-16 stages (natural order in,
//            base-16 digit-reversed order out);
//   product: with H (the DFT of h, precomputed in FP64 on the host, scaled
//            by 1/N, permuted to the digit-reversed order);
//   inverse: decimation in time, the three stages transposed (digit-reversed
//            in, natural order out).
// No reordering pass is needed.  The first forward stage reads the input from
// global memory and the last inverse stage writes the outputs; the innermost
// stage, the product and its inverse run in registers; four shared-memory
// round trips remain.  Twiddles come from tables rounded from FP64 and laid
// out so that a warp's loads are contiguous: stage 0's W4096^(t q) at
// tw[q 256 + t], stage 1's W256^(j q) at tw[4096 + q 16 + j]; the spectrum is
// stored the same way, H[q 256 + t] for the value thread t multiplies into its
// q-th output.
#include <mutex>

#include "devutil.cuh"

namespace cf {
namespace {

constexpr int kN = kFftConvN;    // 4096 = 16^3
constexpr int kT = kN / 16;      // threads: one radix-16 butterfly each per stage

// One padding slot per 16 complex values: the stride-16 accesses of the
// innermost stage then fall on distinct banks.
__device__ __forceinline__ int fpad(int e) { return e + (e >> 4); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// In-place 4-point DFT (forward: W4 = -i; inverse: +i).
template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y), d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
  const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y), d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
  // forward: -i * d13; inverse: +i * d13
  const float2 r = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
  a0 = make_float2(s02.x + s13.x, s02.y + s13.y);
  a2 = make_float2(s02.x - s13.x, s02.y - s13.y);
  a1 = make_float2(d02.x + r.x, d02.y + r.y);
  a3 = make_float2(d02.x - r.x, d02.y - r.y);
}

// exp(-2 pi i m / 16) (forward), its conjugate for the inverse.
template <bool INV>
__device__ __forceinline__ float2 w16(int m) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, r2 = 0.70710678118654752f;
  const float cs[16] = {1.f, c1, r2, s1, 0.f, -s1, -r2, -c1, -1.f, -c1, -r2, -s1, 0.f, s1, r2, c1};
  const float sn[16] = {0.f, s1, r2, c1, 1.f, c1, r2, s1, 0.f, -s1, -r2, -c1, -1.f, -c1, -r2, -s1};
  return make_float2(cs[m], INV ? sn[m] : -sn[m]);
}

// 16-point DFT of a[n] (n = 4 n1 + n2) as 4 x 4: DFT4 over n1, twiddles
// W16^(n2 k1), DFT4 over n2.  X[k1 + 4 k2] is left in a[4 k1 + k2]; XQ maps
// an output index to its register.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&a)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
#pragma unroll
  for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2) a[4 * k1 + n2] = cmul(a[4 * k1 + n2], w16<INV>(n2 * k1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
}
#define XQ(a, q) a[4 * ((q) & 3) + ((q) >> 2)]

// 4-byte asynchronous global -> shared copies (no registers held while in flight)
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Forward stage on positions base + r * stride (r < 16): DFT16, output q
// times twq[16 q] (this thread's twiddle for q), stored back at base + q * stride.
__device__ __forceinline__ void dif_stage(float2* buf, int base, int stride, const float2* __restrict__ twq) {
  float2 a[16], w[16];
#pragma unroll
  for (int q = 1; q < 16; ++q) w[q] = __ldg(twq + 16 * q);
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r] = buf[fpad(base + r * stride)];
  dft16<false>(a);
  buf[fpad(base)] = XQ(a, 0);
#pragma unroll
  for (int q = 1; q < 16; ++q) buf[fpad(base + q * stride)] = cmul(XQ(a, q), w[q]);
}

// Inverse of dif_stage: untwiddle, inverse DFT16, store in natural order.
__device__ __forceinline__ void dit_stage(float2* buf, int base, int stride, const float2* __restrict__ twq) {
  float2 a[16], w[16];
#pragma unroll
  for (int q = 1; q < 16; ++q) w[q] = __ldg(twq + 16 * q);
  a[0] = buf[fpad(base)];
#pragma unroll
  for (int q = 1; q < 16; ++q) a[q] = cmulc(buf[fpad(base + q * stride)], w[q]);
  dft16<true>(a);
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[fpad(base + r * stride)] = XQ(a, r);
}

template <bool SC>
__global__ void __launch_bounds__(kT, 2)
k_conv1d_fft(int64_t n_out, int64_t n_in, int Lp, int64_t D, const float2* __restrict__ H,
             const float2* __restrict__ tw, float alpha, const float* __restrict__ x, float* __restrict__ y,
             bool acc, const float* __restrict__ sin, const float* __restrict__ sout) {
  __shared__ __align__(16) float2 buf[kN + kN / 16];
  extern __shared__ float tail[];  // acc: y, SC: sout, over this pair's outputs
  const int t = threadIdx.x;
  const int V = kN - Lp + 1;
  const int64_t i0 = (int64_t)blockIdx.x * 2 * V;  // first output of the pair
  // what the epilogue reads besides the transform is copied in now, while the
  // transform runs
  const int nout = (int)(n_out - i0 < 2 * (int64_t)V ? n_out - i0 : 2 * (int64_t)V);
  float* ys = tail;
  float* ss = tail + (acc ? 2 * V : 0);
  if (acc || SC) {
    for (int j = t; j < nout; j += kT) {
      if (acc) cp_async4(ys + j, y + i0 + j);
      if (SC) cp_async4(ss + j, sout + i0 + j);
    }
    cp_async_commit();
  }
  // forward stage 0, straight from global: segment A in the real parts,
  // segment B (V outputs later) in the imaginary parts
  {
    float2 a[16], w[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int64_t ga = i0 - D + t + 256 * r, gb = ga + V;
      float va = 0.f, vb = 0.f;
      if (ga >= 0 && ga < n_in) va = SC ? __ldg(sin + ga) * __ldg(x + ga) : __ldg(x + ga);
      if (gb >= 0 && gb < n_in) vb = SC ? __ldg(sin + gb) * __ldg(x + gb) : __ldg(x + gb);
      a[r] = make_float2(va, vb);
    }
#pragma unroll
    for (int q = 1; q < 16; ++q) w[q] = __ldg(tw + 256 * q + t);
    dft16<false>(a);
    buf[fpad(t)] = XQ(a, 0);
#pragma unroll
    for (int q = 1; q < 16; ++q) buf[fpad(t + 256 * q)] = cmul(XQ(a, q), w[q]);
  }
  __syncthreads();
  // forward stage 1: groups of 256, stride 16, twiddles W256^(j q)
  dif_stage(buf, 256 * (t >> 4) + (t & 15), 16, tw + 4096 + (t & 15));
  __syncthreads();
  // forward stage 2 (no twiddles), product with H, inverse stage 2: in registers
  {
    float2 a[16], b[16], h[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) h[q] = __ldg(H + 256 * q + t);
#pragma unroll
    for (int r = 0; r < 16; ++r) a[r] = buf[fpad(16 * t + r)];
    dft16<false>(a);
#pragma unroll
    for (int q = 0; q < 16; ++q) b[q] = cmul(XQ(a, q), h[q]);
    dft16<true>(b);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[fpad(16 * t + r)] = XQ(b, r);
  }
  __syncthreads();
  // inverse stage 1
  dit_stage(buf, 256 * (t >> 4) + (t & 15), 16, tw + 4096 + (t & 15));
  if (acc || SC) cp_async_wait_all();
  __syncthreads();
  // inverse stage 0, straight to global: natural position p = t + 256 r
  {
    float2 a[16], w[16];
#pragma unroll
    for (int q = 1; q < 16; ++q) w[q] = __ldg(tw + 256 * q + t);
    a[0] = buf[fpad(t)];
#pragma unroll
    for (int q = 1; q < 16; ++q) a[q] = cmulc(buf[fpad(t + 256 * q)], w[q]);
    dft16<true>(a);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + 256 * r;
      if (p < Lp - 1) continue;  // wrapped part of the circular convolution
      const float2 c = XQ(a, r);
      const int ja = p - (Lp - 1), jb = ja + V;
      if (ja < nout) {
        const float v = (SC ? alpha * ss[ja] : alpha) * c.x;
        y[i0 + ja] = acc ? ys[ja] + v : v;
      }
      if (jb < nout) {
        const float v = (SC ? alpha * ss[jb] : alpha) * c.y;
        y[i0 + jb] = acc ? ys[jb] + v : v;
      }
    }
  }
}
#undef XQ

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
    const int lim = 2 * 2 * (kN - 16 + 1) * (int)sizeof(float);
    err[device] = cudaFuncSetAttribute(k_conv1d_fft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (err[device] == cudaSuccess)
      err[device] = cudaFuncSetAttribute(k_conv1d_fft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  });
  if (err[device] != cudaSuccess)
    return fail(CF_E_CUDA, std::string("conv1d FFT: shared memory limit: ") + cudaGetErrorString(err[device]));
  return CF_OK;
}

void launch_conv1d_fft(cudaStream_t s, int64_t n_out, int64_t n_in, int64_t Lp, int64_t shift, const float2* H,
                       const float2* tw, float alpha, const float* x, float* y, bool acc, const float* sin,
                       const float* sout) {
  if (n_out <= 0) return;
  const int64_t V = kN - Lp + 1;
  const int64_t pairs = (n_out + 2 * V - 1) / (2 * V);
  const int64_t D = Lp - 1 - shift;
  const bool sc = sin || sout;
  const size_t dyn = (size_t)((acc ? 2 * V : 0) + (sc ? 2 * V : 0)) * sizeof(float);
  if (sc)
    k_conv1d_fft<true><<<(unsigned)pairs, kT, dyn, s>>>(n_out, n_in, (int)Lp, D, H, tw, alpha, x, y, acc, sin,
                                                        sout);
  else
    k_conv1d_fft<false><<<(unsigned)pairs, kT, dyn, s>>>(n_out, n_in, (int)Lp, D, H, tw, alpha, x, y, acc,
                                                         nullptr, nullptr);
}

}  // namespace cf
