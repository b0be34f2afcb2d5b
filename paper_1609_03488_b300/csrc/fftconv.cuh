// Device code of the overlap-save FFT convolution (see k_fftconv.cu for the
// method): the radix-16 stages and the transform of one pair of segments by
// 256 threads, shared by the stand-alone kernel and the team engine's
// convolution term.
#pragma once

#include "devutil.cuh"

namespace cf {
namespace fftc {


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


constexpr int kBufF2 = kN + kN / 16;  // float2 slots of one pair's transform buffer

// The transform's input: through the read-only path when nothing in the
// running kernel writes it (stand-alone kernel), with ordinary loads when
// other CTAs of the same kernel wrote it before a barrier (team engine).
template <bool RO>
__device__ __forceinline__ float ld_in(const float* p) {
  if constexpr (RO)
    return __ldg(p);
  else
    return __ldcg(p);
}

// Outputs y[i0 .. i0 + 2V) of pair `pair` (i0 = 2 V pair, V = N - Lp + 1) by
// the 256 threads t = 0 .. 255 that share `buf` (kBufF2 float2 of shared
// memory) and synchronise with `sync()`:
//   y = alpha sout (K (sin x)) (+ y when acc),
// sin / sout the optional scalings (SC).  With TAIL the epilogue's y and sout
// values were copied into shared memory (ys, ss) by the caller; otherwise
// they are read from global memory in the epilogue.
template <bool SC, bool RO, bool TAIL, class Sync>
__device__ __forceinline__ void pair(int t, int64_t pr, int64_t n_out, int64_t n_in, int Lp, int64_t D,
                                     const float2* __restrict__ H, const float2* __restrict__ tw, float alpha,
                                     const float* x, float* y, bool acc, const float* sin, const float* sout,
                                     float2* buf, const float* ys, const float* ss, Sync&& sync,
                                     bool wait_tail = false) {
  const int V = kN - Lp + 1;
  const int64_t i0 = pr * 2 * V;  // first output of the pair
  const int nout = (int)(n_out - i0 < 2 * (int64_t)V ? n_out - i0 : 2 * (int64_t)V);
  // forward stage 0, straight from global: segment A in the real parts,
  // segment B (V outputs later) in the imaginary parts
  {
    float2 a[16], w[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int64_t ga = i0 - D + t + 256 * r, gb = ga + V;
      float va = 0.f, vb = 0.f;
      if (ga >= 0 && ga < n_in) va = SC ? __ldg(sin + ga) * ld_in<RO>(x + ga) : ld_in<RO>(x + ga);
      if (gb >= 0 && gb < n_in) vb = SC ? __ldg(sin + gb) * ld_in<RO>(x + gb) : ld_in<RO>(x + gb);
      a[r] = make_float2(va, vb);
    }
#pragma unroll
    for (int q = 1; q < 16; ++q) w[q] = __ldg(tw + 256 * q + t);
    dft16<false>(a);
    buf[fpad(t)] = XQ(a, 0);
#pragma unroll
    for (int q = 1; q < 16; ++q) buf[fpad(t + 256 * q)] = cmul(XQ(a, q), w[q]);
  }
  sync();
  // forward stage 1: groups of 256, stride 16, twiddles W256^(j q)
  dif_stage(buf, 256 * (t >> 4) + (t & 15), 16, tw + 4096 + (t & 15));
  sync();
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
  sync();
  // inverse stage 1
  dit_stage(buf, 256 * (t >> 4) + (t & 15), 16, tw + 4096 + (t & 15));
  if (TAIL && wait_tail) cp_async_wait_all();
  sync();
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
        const float s = SC ? (TAIL ? ss[ja] : __ldg(sout + i0 + ja)) : 1.f;
        const float v = (SC ? alpha * s : alpha) * c.x;
        y[i0 + ja] = acc ? (TAIL ? ys[ja] : ld_in<RO>(y + i0 + ja)) + v : v;
      }
      if (jb < nout) {
        const float s = SC ? (TAIL ? ss[jb] : __ldg(sout + i0 + jb)) : 1.f;
        const float v = (SC ? alpha * s : alpha) * c.y;
        y[i0 + jb] = acc ? (TAIL ? ys[jb] : ld_in<RO>(y + i0 + jb)) + v : v;
      }
    }
  }
}

}  // namespace fftc
}  // namespace cf
