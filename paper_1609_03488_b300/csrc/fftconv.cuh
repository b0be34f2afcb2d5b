// Device code of the overlap-save FFT convolution (see k_fftconv.cu for the
// method): the radix-16 stages and the transform of one pair of segments by
// N/16 threads (N = 4096 or 2048), shared by the stand-alone kernel and the
// team engine's convolution term.
#pragma once

#include "devutil.cuh"

namespace cf {
namespace fftc {


// Transform sizes: N = 16 x 16 x R with R = 16 (N = 4096) or 8 (N = 2048).
// T = N/16 threads per pair, one radix-16 butterfly each in the first two
// stages; G = N/16 is the length the second stage splits into 16 groups of,
// S = G/16 = R its stride; the last stage (length R, in registers) gives each
// thread 16 contiguous values: one 16-point or two 8-point butterflies.
template <int N>
struct Cfg {
  static_assert(N == 4096 || N == 2048, "transform size");
  static constexpr int T = N / 16;
  static constexpr int G = N / 16;
  static constexpr int S = G / 16;
  static constexpr int LG = N == 4096 ? 8 : 7;   // log2 G
  static constexpr int LS = N == 4096 ? 4 : 3;   // log2 S
  static constexpr int TW = N + G;               // twiddle table entries
};

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

// exp(-2 pi i m / 8) (forward), its conjugate for the inverse.
template <bool INV>
__device__ __forceinline__ float2 w8(int m) {
  constexpr float r2 = 0.70710678118654752f;
  const float cs[8] = {1.f, r2, 0.f, -r2, -1.f, -r2, 0.f, r2};
  const float sn[8] = {0.f, r2, 1.f, r2, 0.f, -r2, -1.f, -r2};
  return make_float2(cs[m], INV ? sn[m] : -sn[m]);
}

// 8-point DFT of a[o + n] (n = 4 n1 + n2) as 2 x 4: DFT2 over n1, twiddles
// W8^(n2 k1), DFT4 over n2.  X[k1 + 2 k2] is left in a[o + 4 k1 + k2]; XQ8
// maps an output index to its register.
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&a)[16], int o) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    const float2 u = a[o + n2], v = a[o + 4 + n2];
    a[o + n2] = make_float2(u.x + v.x, u.y + v.y);
    const float2 d = make_float2(u.x - v.x, u.y - v.y);
    a[o + 4 + n2] = n2 == 0 ? d : cmul(d, w8<INV>(n2));
  }
#pragma unroll
  for (int k1 = 0; k1 < 2; ++k1) dft4<INV>(a[o + 4 * k1], a[o + 4 * k1 + 1], a[o + 4 * k1 + 2], a[o + 4 * k1 + 3]);
}
#define XQ8(a, o, q) a[(o) + 4 * ((q) & 1) + ((q) >> 1)]

// 4-byte asynchronous global -> shared copies (no registers held while in flight)
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Forward stage on positions base + r * stride (r < 16): DFT16, output q
// times twq[TWS q] (this thread's twiddle for q), stored back at base + q * stride.
template <int TWS>
__device__ __forceinline__ void dif_stage(float2* buf, int base, int stride, const float2* __restrict__ twq) {
  float2 a[16], w[16];
#pragma unroll
  for (int q = 1; q < 16; ++q) w[q] = __ldg(twq + TWS * q);
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r] = buf[fpad(base + r * stride)];
  dft16<false>(a);
  buf[fpad(base)] = XQ(a, 0);
#pragma unroll
  for (int q = 1; q < 16; ++q) buf[fpad(base + q * stride)] = cmul(XQ(a, q), w[q]);
}

// Inverse of dif_stage: untwiddle, inverse DFT16, store in natural order.
template <int TWS>
__device__ __forceinline__ void dit_stage(float2* buf, int base, int stride, const float2* __restrict__ twq) {
  float2 a[16], w[16];
#pragma unroll
  for (int q = 1; q < 16; ++q) w[q] = __ldg(twq + TWS * q);
  a[0] = buf[fpad(base)];
#pragma unroll
  for (int q = 1; q < 16; ++q) a[q] = cmulc(buf[fpad(base + q * stride)], w[q]);
  dft16<true>(a);
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[fpad(base + r * stride)] = XQ(a, r);
}


// float2 slots of one pair's transform buffer
template <int N>
constexpr int buf_f2() { return N + N / 16; }

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

// Outputs y[i0 .. i0 + 2V) of pair `pr` (i0 = 2 V pr, V = N - Lp + 1) by
// the T = N/16 threads t = 0 .. T-1 that share `buf` (buf_f2<N>() float2 of
// shared memory) and synchronise with `sync()`:
//   y = alpha sout (K (sin x)) (+ y when acc),
// sin / sout the optional scalings (SC).  With TAIL the epilogue's y and sout
// values were copied into shared memory (ys, ss) by the caller; otherwise
// they are read from global memory in the epilogue.
//
// Stages (C = Cfg<N>): forward stage 0 on positions t + T r with twiddles
// W_N^(t q) at tw[q T + t]; stage 1 on positions G (t >> LS) + (t & (S-1))
// + S r with twiddles W_G^(j q) at tw[N + q S + j]; the last stage, the
// product with H and its inverse in registers on positions 16 t .. 16 t + 15
// (the spectrum's factor for the thread's q-th value at H[q T + t]); then the
// two inverse stages.
template <int N, bool SC, bool RO, bool TAIL, class Sync>
__device__ __forceinline__ void pair(int t, int64_t pr, int64_t n_out, int64_t n_in, int Lp, int64_t D,
                                     const float2* __restrict__ H, const float2* __restrict__ tw, float alpha,
                                     const float* x, float* y, bool acc, const float* sin, const float* sout,
                                     float2* buf, const float* ys, const float* ss, Sync&& sync,
                                     bool wait_tail = false) {
  using C = Cfg<N>;
  constexpr int T = C::T;
  const int V = N - Lp + 1;
  const int64_t i0 = pr * 2 * V;  // first output of the pair
  const int nout = (int)(n_out - i0 < 2 * (int64_t)V ? n_out - i0 : 2 * (int64_t)V);
  const int base1 = C::G * (t >> C::LS) + (t & (C::S - 1));
  const float2* tw1 = tw + N + (t & (C::S - 1));
  // forward stage 0, straight from global: segment A in the real parts,
  // segment B (V outputs later) in the imaginary parts
  {
    float2 a[16], w[16];
    const int64_t g0 = i0 - D;  // first input position of segment A
    bool inside = false;
    if constexpr (RO) inside = g0 >= 0 && g0 + V + N <= n_in;
    if (inside) {
      // stand-alone kernel, both segments inside the input (every pair but
      // the first and the last): one base pointer and constant offsets, no
      // bounds tests.  (Only here: the same code in the team kernel's term
      // changed that large kernel's register allocation and slowed it.)
      const float* xa = x + g0 + t;
      const float* sa = SC ? sin + g0 + t : nullptr;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        float va = ld_in<RO>(xa + T * r), vb = ld_in<RO>(xa + V + T * r);
        if (SC) {
          va = __ldg(sa + T * r) * va;
          vb = __ldg(sa + V + T * r) * vb;
        }
        a[r] = make_float2(va, vb);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int64_t ga = i0 - D + t + T * r, gb = ga + V;
        float va = 0.f, vb = 0.f;
        if (ga >= 0 && ga < n_in) va = SC ? __ldg(sin + ga) * ld_in<RO>(x + ga) : ld_in<RO>(x + ga);
        if (gb >= 0 && gb < n_in) vb = SC ? __ldg(sin + gb) * ld_in<RO>(x + gb) : ld_in<RO>(x + gb);
        a[r] = make_float2(va, vb);
      }
    }
#pragma unroll
    for (int q = 1; q < 16; ++q) w[q] = __ldg(tw + T * q + t);
    dft16<false>(a);
    buf[fpad(t)] = XQ(a, 0);
#pragma unroll
    for (int q = 1; q < 16; ++q) buf[fpad(t + T * q)] = cmul(XQ(a, q), w[q]);
  }
  sync();
  // forward stage 1: 16 groups of G, stride S, twiddles W_G^(j q)
  dif_stage<C::S>(buf, base1, C::S, tw1);
  sync();
  // last forward stage (no twiddles), product with H, its inverse: in registers
  {
    float2 a[16], h[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) h[q] = __ldg(H + T * q + t);
#pragma unroll
    for (int r = 0; r < 16; ++r) a[r] = buf[fpad(16 * t + r)];
    if constexpr (N == 4096) {
      float2 b[16];
      dft16<false>(a);
#pragma unroll
      for (int q = 0; q < 16; ++q) b[q] = cmul(XQ(a, q), h[q]);
      dft16<true>(b);
#pragma unroll
      for (int r = 0; r < 16; ++r) buf[fpad(16 * t + r)] = XQ(b, r);
    } else {
      float2 b[16];
      dft8<false>(a, 0);
      dft8<false>(a, 8);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        b[q] = cmul(XQ8(a, 0, q), h[q]);
        b[8 + q] = cmul(XQ8(a, 8, q), h[8 + q]);
      }
      dft8<true>(b, 0);
      dft8<true>(b, 8);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        buf[fpad(16 * t + r)] = XQ8(b, 0, r);
        buf[fpad(16 * t + 8 + r)] = XQ8(b, 8, r);
      }
    }
  }
  sync();
  // inverse stage 1
  dit_stage<C::S>(buf, base1, C::S, tw1);
  if (TAIL && wait_tail) cp_async_wait_all();
  sync();
  // inverse stage 0, straight to global: natural position p = t + T r
  {
    float2 a[16], w[16];
#pragma unroll
    for (int q = 1; q < 16; ++q) w[q] = __ldg(tw + T * q + t);
    a[0] = buf[fpad(t)];
#pragma unroll
    for (int q = 1; q < 16; ++q) a[q] = cmulc(buf[fpad(t + T * q)], w[q]);
    dft16<true>(a);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + T * r;
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
