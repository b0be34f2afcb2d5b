// Device helpers shared by the solver's vector kernels, the operator leaves
// and the persistent team solver.
#pragma once

#include "internal.cuh"

namespace cf {

__device__ __forceinline__ float4 ld4(const float* p, int64_t v) {
  return reinterpret_cast<const float4*>(p)[v];
}
__device__ __forceinline__ void st4(float* p, int64_t v, float4 a) { reinterpret_cast<float4*>(p)[v] = a; }
__device__ __forceinline__ float& el(float4& a, int k) { return (&a.x)[k]; }
__device__ __forceinline__ float elc(const float4& a, int k) { return (&a.x)[k]; }

// Per-thread sum in compensated float32 ("double-float": hi + lo), with each
// product taken exactly (p + e, e = fma(a, b, -p)) and each addition by
// TwoSum.  Its accuracy is close to float64 accumulation without a float64
// operation per element (the float64 rate of this GPU is a small fraction of
// its float32 rate); the per-thread value feeds the float64 block and grid
// sums.  Explicit-rounding intrinsics keep the compiler from contracting
// the error terms away.
struct Acc2 {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// The point projected onto K* for row i of y:
//   p_i = (alpha (z_y - u~_tau g_y) + (1 - alpha) u_y) - v_s
// evaluated with explicit roundings so both kernels that need it agree bit
// for bit.
__device__ __forceinline__ float y_pre(float a, float a1, float ut, float zy, float gy, float uy,
                                       float vs) {
  float uhat = __fadd_rn(__fmul_rn(a, __fsub_rn(zy, __fmul_rn(ut, gy))), __fmul_rn(a1, uy));
  return __fsub_rn(uhat, vs);
}

// 16-byte loads of the stored operand, unpacked to float32.
template <typename T> struct Vec;
template <> struct Vec<float> {
  static constexpr int N = 4;
  __device__ static void unpack(const uint4& u, float* f) {
    f[0] = __uint_as_float(u.x); f[1] = __uint_as_float(u.y);
    f[2] = __uint_as_float(u.z); f[3] = __uint_as_float(u.w);
  }
};
template <> struct Vec<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ static void unpack(const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      f[2 * k] = __uint_as_float(w[k] << 16);
      f[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
};
template <> struct Vec<__nv_fp8_e4m3> {
  static constexpr int N = 16;
  __device__ static void unpack(const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int b = 0; b < 4; b += 2) {
        __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[k] >> (8 * b)) & 0xffff);
        __half2_raw h2 = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
        __half2 hh = *reinterpret_cast<__half2*>(&h2);
        float2 ff = __half22float2(hh);
        f[4 * k + b] = ff.x;
        f[4 * k + b + 1] = ff.y;
      }
    }
  }
};

// Streaming loads of operator data that skip L1 (so that they do not evict
// the gathered vector) and stay cacheable in L2.
__device__ __forceinline__ int4 ld_stream_i4(const int32_t* p) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_stream_u4(const void* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

}  // namespace cf
