// Leaf kernels of the structured operators (Section 3.1): every kernel
// computes y = alpha * op(x) + (acc ? y : 0).
#include "devutil.cuh"

namespace cf {

// ------------------------------------------------------------ elementwise
__global__ void k_fill(int64_t n, float v, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = v;
}

__global__ void k_diag(int64_t n, const float* __restrict__ d, float alpha,
                       const float* __restrict__ x, float* __restrict__ y, bool acc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = alpha * (d ? d[i] * x[i] : x[i]);
    y[i] = acc ? y[i] + v : v;
  }
}

// blockIdx.y selects the segment; segments are independent (the host only
// batches operations without data hazards between them).
// Whether every array of a segment starts on a 16-byte boundary.
__device__ __forceinline__ bool ew_aligned16(const EwSeg& g) {
  uintptr_t a = reinterpret_cast<uintptr_t>(g.y) | reinterpret_cast<uintptr_t>(g.sout);
  for (int k = 0; k < g.nterm; ++k)
    a |= reinterpret_cast<uintptr_t>(g.x[k]) | reinterpret_cast<uintptr_t>(g.d[k]) |
         reinterpret_cast<uintptr_t>(g.sin[k]);
  return (a & 15) == 0;
}

// Rows 4v .. 4v + 3 of a segment with 16-byte loads; per row the arithmetic
// of ew_value, operation for operation.
__device__ __forceinline__ float4 ew_value4(const EwSeg& g, int64_t v) {
  float4 out = g.acc ? ld4(g.y, v) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 so = g.sout ? ld4(g.sout, v) : make_float4(1.f, 1.f, 1.f, 1.f);
  for (int k = 0; k < g.nterm; ++k) {
    float4 xv = ld4(g.x[k], v);
    if (g.sin[k]) {
      const float4 sv = ld4(g.sin[k], v);
#pragma unroll
      for (int e = 0; e < 4; ++e) el(xv, e) = elc(sv, e) * elc(xv, e);
    }
    if (g.d[k]) {
      const float4 dv = ld4(g.d[k], v);
#pragma unroll
      for (int e = 0; e < 4; ++e) el(xv, e) = elc(dv, e) * elc(xv, e);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) el(out, e) = fmaf(g.sout ? g.alpha[k] * elc(so, e) : g.alpha[k], elc(xv, e), el(out, e));
  }
  return out;
}

__global__ void k_ew(EwBatch b) {
  const EwSeg& g = b.seg[blockIdx.y];
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  int64_t head = 0;
  if (ew_aligned16(g)) {
    const int64_t n4 = g.n >> 2;
    for (int64_t v = t0; v < n4; v += stride) st4(g.y, v, ew_value4(g, v));
    head = n4 << 2;
  }
  for (int64_t i = head + t0; i < g.n; i += stride) g.y[i] = ew_value(g, i);
}

void launch_ew(cudaStream_t s, const EwBatch& b) {
  if (b.nseg <= 0) return;
  int64_t mx = 1;
  for (int k = 0; k < b.nseg; ++k) mx = std::max(mx, b.seg[k].n);
  dim3 grid((unsigned)grid_for(mx), (unsigned)b.nseg);
  k_ew<<<grid, kThreads, 0, s>>>(b);
}

void launch_fill(cudaStream_t s, int64_t n, float v, float* y) {
  if (n <= 0) return;
  k_fill<<<grid_for(n), kThreads, 0, s>>>(n, v, y);
}

void launch_diag(cudaStream_t s, int64_t n, const float* d, float alpha, const float* x, float* y,
                 bool acc) {
  if (n <= 0) return;
  k_diag<<<grid_for(n), kThreads, 0, s>>>(n, d, alpha, x, y, acc);
}

// ------------------------------------------------------------ 1-D convolution
// out[i] = sum_{l < Lp} w[l] in[i + shift - l]  (in = 0 outside [0, n_in)),
// given wrev[j] = w[Lp - 1 - j].  Forward full convolution: w = k, shift = 0;
// adjoint (correlation): w = k reversed, shift = Lp - 1.
//
// FP32 CUDA-core kernel (the operator is a matrix-vector product, not a
// dense contraction).  A CTA owns kConvTile consecutive outputs; each thread
// keeps kConvR consecutive outputs in registers.  For each block of kConvR
// taps it loads kConvR new inputs (four 16-byte shared loads) into one of two
// register windows that alternate roles, and the kConvR weights (four 16-byte
// broadcast loads), then issues kConvR x kConvR fused multiply-adds: about 95%
// of the issued instructions are FMAs.  Shared input element j lives at
// j + 4 floor(j / kConvR): the 16-byte loads of 8 neighbouring lanes (stride
// kConvR floats) then fall on distinct bank groups for every window offset.
// Taps are processed in chunks of at most kConvChunk.
constexpr int kConvOutThreads = 64;                    // threads sharing the output tile
constexpr int kConvGroups = 2;                         // tap groups per CTA
constexpr int kConvThreads = kConvOutThreads * kConvGroups;
constexpr int kConvR = 16;
constexpr int kConvTile = kConvOutThreads * kConvR;
constexpr int kConvChunk = 2048;
constexpr int kConvPadStride = kConvR + 4;             // padded floats per kConvR inputs

__host__ __device__ __forceinline__ int conv_pad(int j) { return j + ((j / kConvR) << 2); }

// One block of kConvR taps: acc[r] += w[dd] * window[r + dd], where window is
// lo[0..R) followed by hi[0..R).
__device__ __forceinline__ void conv_block(float (&acc)[kConvR], const float (&lo)[kConvR],
                                           const float (&hi)[kConvR], const float* __restrict__ wsm) {
  float wv[kConvR];
#pragma unroll
  for (int q = 0; q < kConvR; q += 4) {
    float4 t4 = *reinterpret_cast<const float4*>(wsm + q);
    wv[q] = t4.x; wv[q + 1] = t4.y; wv[q + 2] = t4.z; wv[q + 3] = t4.w;
  }
#pragma unroll
  for (int dd = 0; dd < kConvR; ++dd)
#pragma unroll
    for (int r = 0; r < kConvR; ++r)
      acc[r] = fmaf(wv[dd], (r + dd < kConvR) ? lo[r + dd] : hi[r + dd - kConvR], acc[r]);
}

// kConvR consecutive inputs starting at a multiple of kConvR (4 contiguous
// float4 in the padded layout).
__device__ __forceinline__ void conv_load(float (&dst)[kConvR], const float* __restrict__ p) {
#pragma unroll
  for (int q = 0; q < kConvR; q += 4) {
    float4 t4 = *reinterpret_cast<const float4*>(p + q);
    dst[q] = t4.x; dst[q + 1] = t4.y; dst[q + 2] = t4.z; dst[q + 3] = t4.w;
  }
}

// SC: the input is read as sin * x and the outputs are multiplied by sout.
template <bool SC>
__global__ void __launch_bounds__(kConvThreads)
k_conv1d(int64_t n_out, int64_t n_in, int64_t Lp, int64_t shift, const float* __restrict__ wrev,
         float alpha, const float* __restrict__ x, float* __restrict__ y, bool acc,
         const float* __restrict__ sin, const float* __restrict__ sout) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  const int grp = tid / kConvOutThreads;       // which part of the taps
  const int t = tid % kConvOutThreads;         // which outputs
  const int64_t i0 = (int64_t)blockIdx.x * kConvTile;
  float accum[kConvR];
#pragma unroll
  for (int r = 0; r < kConvR; ++r) accum[r] = 0.f;

  const int lc_max = (int)(Lp < kConvChunk ? Lp : (int64_t)kConvChunk);
  float* in_s = sm;
  float* w_s = sm + conv_pad(kConvTile + lc_max + kConvR) + 4;

  for (int64_t l0 = 0; l0 < Lp; l0 += kConvChunk) {
    const int lc = (int)((Lp - l0) < kConvChunk ? (Lp - l0) : (int64_t)kConvChunk);
    const int64_t base = i0 + shift - l0 - (lc - 1);
    __syncthreads();
    for (int j = tid; j < kConvTile + lc + kConvR; j += kConvThreads) {
      int64_t g = base + j;
      in_s[conv_pad(j)] = (g >= 0 && g < n_in) ? (SC ? __ldg(sin + g) * __ldg(x + g) : __ldg(x + g)) : 0.f;
    }
    const float* wsrc = wrev + (Lp - l0 - lc);
    for (int j = tid; j < lc; j += kConvThreads) w_s[j] = __ldg(wsrc + j);
    __syncthreads();

    // this group's tap blocks [b0, b1) of kConvR taps each
    const int nblk = lc / kConvR;
    const int b0 = (grp * nblk) / kConvGroups, b1 = ((grp + 1) * nblk) / kConvGroups;
    // window start of output block t at tap block b: conv_pad(t R + b R) = (t + b) * (R + 4)
    const float* ip = in_s + (t + b0) * kConvPadStride;
    const float* wp = w_s + b0 * kConvR;
    float wa[kConvR], wb[kConvR];
    conv_load(wa, ip);
    int b = b0;
    for (; b + 2 <= b1; b += 2) {
      conv_load(wb, ip + kConvPadStride);
      conv_block(accum, wa, wb, wp);
      conv_load(wa, ip + 2 * kConvPadStride);
      conv_block(accum, wb, wa, wp + kConvR);
      ip += 2 * kConvPadStride;
      wp += 2 * kConvR;
    }
    if (b < b1) {
      conv_load(wb, ip + kConvPadStride);
      conv_block(accum, wa, wb, wp);
    }
  }
  // fold the tap groups in a fixed order (group 0 adds group 1, 2, ...)
#pragma unroll
  for (int g = 1; g < kConvGroups; ++g) {
    __syncthreads();
    if (grp == g) {
#pragma unroll
      for (int r = 0; r < kConvR; ++r) in_s[t * (kConvR + 1) + r] = accum[r];
    }
    __syncthreads();
    if (grp == 0) {
#pragma unroll
      for (int r = 0; r < kConvR; ++r) accum[r] += in_s[t * (kConvR + 1) + r];
    }
  }
  if (grp != 0) return;
#pragma unroll
  for (int r = 0; r < kConvR; ++r) {
    int64_t i = i0 + t * kConvR + r;
    if (i < n_out) {
      float v = (SC ? alpha * __ldg(sout + i) : alpha) * accum[r];
      y[i] = acc ? y[i] + v : v;
    }
  }
}

void launch_conv1d(cudaStream_t s, int64_t n_out, int64_t n_in, int64_t Lp, int64_t shift,
                   const float* wrev, float alpha, const float* x, float* y, bool acc,
                   const float* sin, const float* sout) {
  if (n_out <= 0) return;
  const int lc_max = (int)std::min<int64_t>(Lp, kConvChunk);
  const size_t smem = (size_t)(conv_pad(kConvTile + lc_max + kConvR) + 4 + lc_max) * sizeof(float);
  const int64_t grid = (n_out + kConvTile - 1) / kConvTile;
  if (sin || sout)
    k_conv1d<true><<<(unsigned)grid, kConvThreads, smem, s>>>(n_out, n_in, Lp, shift, wrev, alpha, x, y, acc, sin,
                                                              sout);
  else
    k_conv1d<false><<<(unsigned)grid, kConvThreads, smem, s>>>(n_out, n_in, Lp, shift, wrev, alpha, x, y, acc,
                                                               nullptr, nullptr);
}

// ------------------------------------------------------------ 2-D convolution
// out[a, b] = sum_{p<kh, q<kw} w[p, q] in[a + sh - p, b + sw - q]; a 16 x 16
// output tile per CTA with its input halo and the taps staged in shared memory.
constexpr int kC2T = 16;

__global__ void __launch_bounds__(kC2T* kC2T)
k_conv2d(int64_t Ho, int64_t Wo, int64_t Hi, int64_t Wi, int kh, int kw, int64_t sh, int64_t sw,
         const float* __restrict__ kern, float alpha, const float* __restrict__ x,
         float* __restrict__ y, bool acc) {
  extern __shared__ float sm[];
  const int TH = kC2T + kh - 1, TW = kC2T + kw - 1;
  float* in_s = sm;
  float* k_s = sm + TH * TW;
  const int64_t a0 = (int64_t)blockIdx.y * kC2T, b0 = (int64_t)blockIdx.x * kC2T;
  const int tid = threadIdx.y * kC2T + threadIdx.x;
  for (int j = tid; j < kh * kw; j += kC2T * kC2T) k_s[j] = kern[j];
  // input rows a0 + sh - (kh-1) .. a0 + sh + kC2T - 1
  for (int j = tid; j < TH * TW; j += kC2T * kC2T) {
    int r = j / TW, c = j % TW;
    int64_t gi = a0 + sh - (kh - 1) + r, gj = b0 + sw - (kw - 1) + c;
    in_s[j] = (gi >= 0 && gi < Hi && gj >= 0 && gj < Wi) ? x[gi * Wi + gj] : 0.f;
  }
  __syncthreads();
  const int ty = threadIdx.y, tx = threadIdx.x;
  float accv = 0.f;
  for (int p = 0; p < kh; ++p)
    for (int q = 0; q < kw; ++q)
      accv = fmaf(k_s[p * kw + q], in_s[(ty + kh - 1 - p) * TW + (tx + kw - 1 - q)], accv);
  int64_t a = a0 + ty, b = b0 + tx;
  if (a < Ho && b < Wo) {
    float v = alpha * accv;
    y[a * Wo + b] = acc ? y[a * Wo + b] + v : v;
  }
}

void launch_conv2d(cudaStream_t s, int64_t Ho, int64_t Wo, int64_t Hi, int64_t Wi, int64_t kh,
                   int64_t kw, int64_t sh, int64_t sw, const float* kern, float alpha,
                   const float* x, float* y, bool acc) {
  if (Ho <= 0 || Wo <= 0) return;
  dim3 grid((unsigned)((Wo + kC2T - 1) / kC2T), (unsigned)((Ho + kC2T - 1) / kC2T));
  size_t smem = ((kC2T + kh - 1) * (kC2T + kw - 1) + kh * kw) * sizeof(float);
  k_conv2d<<<grid, dim3(kC2T, kC2T), smem, s>>>(Ho, Wo, Hi, Wi, (int)kh, (int)kw, sh, sw, kern,
                                                alpha, x, y, acc);
}

// ------------------------------------------------------------ dense GEMV

// y[i] = alpha * s_i * sum_j A[i, j] x[j]: a CTA handles RW consecutive
// rows and all its threads sweep the columns together, each thread taking
// the V columns of one 16-byte load, so that the CTA reads THREADS x 16
// contiguous bytes of each of its rows at once (long DRAM bursts) and each
// slice of x a thread loads serves RW rows.  PF: the next sweep's operand
// loads are issued before the current sweep's arithmetic (FP8, whose
// unpacking makes a sweep long enough to hide them behind).  The per-thread
// sums of a row are added by a warp tree and then across warps in warp
// order.
// SC: x is read as sin * x and the rows are multiplied by sout.
constexpr int kGemvNRows = 8;

template <typename T, int THREADS, bool PF, bool SC>
__global__ void __launch_bounds__(THREADS)
k_gemv_n(int64_t m, int64_t n, int64_t lda, const T* __restrict__ A, const float* __restrict__ rs,
         float alpha, const float* __restrict__ x, float* __restrict__ y, bool acc,
         const float* __restrict__ sin, const float* __restrict__ sout) {
  constexpr int V = Vec<T>::N;
  constexpr int RW = kGemvNRows;
  constexpr int NW = THREADS / 32;
  __shared__ float red[NW][RW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * RW;
  const bool xal = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) &&
                   (!SC || ((reinterpret_cast<uintptr_t>(sin) & 15) == 0));
  const T* arow[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) arow[r] = A + (row0 + r < m ? row0 + r : m - 1) * lda;  // rows past m: not stored
  float accv[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) accv[r] = 0.f;
  int64_t c = (int64_t)threadIdx.x * V;
  uint4 u[RW];
  if (PF && c < n) {
#pragma unroll
    for (int r = 0; r < RW; ++r) u[r] = __ldg(reinterpret_cast<const uint4*>(arow[r] + c));
  }
  for (; c < n; c += (int64_t)THREADS * V) {
    if (!PF) {
#pragma unroll
      for (int r = 0; r < RW; ++r) u[r] = __ldg(reinterpret_cast<const uint4*>(arow[r] + c));
    }
    float xv[V];
    if (xal && c + V <= n) {
#pragma unroll
      for (int q = 0; q < V; q += 4) {
        float4 t = __ldg(reinterpret_cast<const float4*>(x + c + q));
        if (SC) {
          const float4 w = __ldg(reinterpret_cast<const float4*>(sin + c + q));
          t.x *= w.x; t.y *= w.y; t.z *= w.z; t.w *= w.w;
        }
        xv[q] = t.x; xv[q + 1] = t.y; xv[q + 2] = t.z; xv[q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q)
        xv[q] = (c + q < n) ? (SC ? __ldg(sin + c + q) * __ldg(x + c + q) : __ldg(x + c + q)) : 0.f;
    }
    uint4 un[RW];
    if (PF) {
      const int64_t cn = c + (int64_t)THREADS * V;
#pragma unroll
      for (int r = 0; r < RW; ++r)
        un[r] = cn < n ? __ldg(reinterpret_cast<const uint4*>(arow[r] + cn)) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      float av[V];
      Vec<T>::unpack(u[r], av);
#pragma unroll
      for (int q = 0; q < V; ++q) accv[r] = fmaf(av[q], xv[q], accv[r]);
    }
    if (PF) {
#pragma unroll
      for (int r = 0; r < RW; ++r) u[r] = un[r];
    }
  }
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    float v = accv[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][r] = v;
  }
  __syncthreads();
  if (threadIdx.x < RW) {
    const int r = threadIdx.x;
    const int64_t row = row0 + r;
    if (row < m) {
      float v = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) v += red[w][r];
      float out = (SC ? alpha * sout[row] : alpha) * (rs ? rs[row] * v : v);
      y[row] = acc ? y[row] + out : out;
    }
  }
}

template <typename T>
static void gemv_n_typed(cudaStream_t s, int64_t m, int64_t n, int64_t lda, const void* A, const float* rs,
                         float alpha, const float* x, float* y, bool acc, const float* sin, const float* sout) {
  // 2048 columns a sweep for the 1- and 2-byte types, 1024 for float32
  constexpr int TH = sizeof(T) == 1 ? 128 : 256;
  constexpr bool PF = sizeof(T) == 1;
  const unsigned grid = (unsigned)((m + kGemvNRows - 1) / kGemvNRows);
  if (sin || sout)
    k_gemv_n<T, TH, PF, true><<<grid, TH, 0, s>>>(m, n, lda, (const T*)A, rs, alpha, x, y, acc, sin, sout);
  else
    k_gemv_n<T, TH, PF, false><<<grid, TH, 0, s>>>(m, n, lda, (const T*)A, rs, alpha, x, y, acc, nullptr,
                                                   nullptr);
}

void launch_gemv_n(cudaStream_t s, cf_prec p, int64_t m, int64_t n, int64_t lda, const void* A,
                   const float* rs, float alpha, const float* x, float* y, bool acc, const float* sin,
                   const float* sout) {
  if (m <= 0) return;
  if (p == CF_FP32)
    gemv_n_typed<float>(s, m, n, lda, A, rs, alpha, x, y, acc, sin, sout);
  else if (p == CF_BF16)
    gemv_n_typed<__nv_bfloat16>(s, m, n, lda, A, rs, alpha, x, y, acc, sin, sout);
  else
    gemv_n_typed<__nv_fp8_e4m3>(s, m, n, lda, A, rs, alpha, x, y, acc, sin, sout);
}

// x^T-side: part[rb, j] = sum_{i in row block rb} A[i, j] (s_i y_i); each
// thread owns the V columns of one 16-byte load, so every row is read once
// with coalesced loads.  A CTA covers kGemvTCols columns whatever the storage
// type: 256 / 128 / 64 threads span them for FP32 / BF16 / FP8, and FP8 runs
// RG = 4 such row groups per CTA (rows r0 + g, r0 + g + 4, ...; 256 threads)
// whose sums are added in group order through shared memory.  A thread has
// kGemvTUnroll rows' loads in flight.  The row blocks are sized for one wave
// of 8 CTAs per SM (4 for FP8), the shapes measured fastest at 20000 x
// 10000.  A second kernel sums the row blocks in a fixed order.
constexpr int kGemvTCols = 1024;
constexpr int kGemvTMaxRows = 512;
constexpr int kGemvTUnroll = 8;
constexpr int kGemvTThreads = 256;  // the largest CTA

template <typename T>
constexpr int gemv_t_groups() { return sizeof(T) == 1 ? 4 : 1; }

template <typename T>
__global__ void __launch_bounds__(kGemvTThreads)
k_gemv_t_part(int64_t m, int64_t n, int64_t lda, int64_t rows_per_block, const T* __restrict__ A,
              const float* __restrict__ rs, const float* __restrict__ yv, float* __restrict__ part,
              const float* __restrict__ sin) {
  constexpr int V = Vec<T>::N;
  constexpr int CT = kGemvTCols / V;  // threads across the columns
  constexpr int RG = gemv_t_groups<T>();
  __shared__ float sy[kGemvTMaxRows];
  __shared__ float red[RG > 1 ? RG - 1 : 1][RG > 1 ? kGemvTCols : 1];
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = (r0 + rows_per_block < m) ? r0 + rows_per_block : m;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
    sy[i - r0] = (rs ? rs[i] * yv[i] : yv[i]) * (sin ? sin[i] : 1.f);
  __syncthreads();
  const int ct = threadIdx.x % CT, g = threadIdx.x / CT;
  const int64_t c0 = ((int64_t)blockIdx.x * CT + ct) * V;
  const bool live = c0 < n;
  float accv[V];
#pragma unroll
  for (int q = 0; q < V; ++q) accv[q] = 0.f;
  if (live) {
    int64_t i = r0 + g;
    for (; i + (int64_t)(kGemvTUnroll - 1) * RG < r1; i += (int64_t)kGemvTUnroll * RG) {
      uint4 u[kGemvTUnroll];
#pragma unroll
      for (int k = 0; k < kGemvTUnroll; ++k)
        u[k] = __ldg(reinterpret_cast<const uint4*>(A + (i + (int64_t)k * RG) * lda + c0));
#pragma unroll
      for (int k = 0; k < kGemvTUnroll; ++k) {
        float av[V];
        Vec<T>::unpack(u[k], av);
        const float sv = sy[i + (int64_t)k * RG - r0];
#pragma unroll
        for (int q = 0; q < V; ++q) accv[q] = fmaf(av[q], sv, accv[q]);
      }
    }
    for (; i < r1; i += RG) {
      uint4 u = __ldg(reinterpret_cast<const uint4*>(A + i * lda + c0));
      float av[V];
      Vec<T>::unpack(u, av);
      const float sv = sy[i - r0];
#pragma unroll
      for (int q = 0; q < V; ++q) accv[q] = fmaf(av[q], sv, accv[q]);
    }
  }
  if (RG > 1) {
    if (g > 0) {
#pragma unroll
      for (int q = 0; q < V; ++q) red[g - 1][ct * V + q] = accv[q];
    }
    __syncthreads();
    if (g > 0) return;
#pragma unroll
    for (int h = 0; h < RG - 1; ++h)
#pragma unroll
      for (int q = 0; q < V; ++q) accv[q] += red[h][ct * V + q];
  }
  if (!live) return;
  float* dst = part + (int64_t)blockIdx.y * lda + c0;
#pragma unroll
  for (int q = 0; q < V; q += 4)
    *reinterpret_cast<float4*>(dst + q) = make_float4(accv[q], accv[q + 1], accv[q + 2], accv[q + 3]);
}

// x[j] = alpha sout_j sum_rb part[rb, j]: a CTA takes 32 columns; its 8 warps
// sum interleaved row blocks (coalesced over the columns) and warp 0 adds
// the 8 results in warp order, so the sum's order is fixed.
constexpr int kGemvTRedRows = 8;

__global__ void __launch_bounds__(32 * kGemvTRedRows)
k_gemv_t_reduce(int64_t n, int64_t lda, int nrb, const float* __restrict__ part, float alpha,
                float* __restrict__ x, bool acc, const float* __restrict__ sout) {
  constexpr int R = kGemvTRedRows;
  __shared__ float sh[R][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + tx;
  float s4[4] = {0.f, 0.f, 0.f, 0.f};
  if (j < n) {
    int b = ty;
    for (; b + 3 * R < nrb; b += 4 * R) {
#pragma unroll
      for (int k = 0; k < 4; ++k) s4[k] += __ldcg(part + (int64_t)(b + k * R) * lda + j);
    }
    for (; b < nrb; b += R) s4[0] += __ldcg(part + (int64_t)b * lda + j);
  }
  sh[ty][tx] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
  __syncthreads();
  if (ty == 0 && j < n) {
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) sum += sh[k][tx];
    const float v = (sout ? alpha * sout[j] : alpha) * sum;
    x[j] = acc ? x[j] + v : v;
  }
}

// Row blocks for `per_sm` CTAs per SM, rounded down so the grid is one wave.
static int gemv_t_row_blocks(int64_t m, int64_t n, int per_sm = 8) {
  const int64_t col_tiles = (n + kGemvTCols - 1) / kGemvTCols;
  const int64_t want = std::max<int64_t>(1, (int64_t)per_sm * 148 / col_tiles);
  const int64_t min_rb = (m + kGemvTMaxRows - 1) / kGemvTMaxRows;  // shared-memory cap
  const int64_t max_rb = std::max<int64_t>(1, m / 32);
  const int64_t rb = std::min(want, max_rb);
  return (int)std::max<int64_t>(std::max<int64_t>(rb, min_rb), 1);
}

size_t gemv_t_ws_floats(int64_t m, int64_t n, int64_t lda) {
  return (size_t)gemv_t_row_blocks(m, n) * (size_t)lda;
}

void launch_gemv_t(cudaStream_t s, cf_prec p, int64_t m, int64_t n, int64_t lda, const void* A,
                   const float* rs, float alpha, const float* x, float* y, bool acc, float* ws,
                   const float* sin, const float* sout) {
  if (n <= 0) return;
  if (m <= 0) {
    if (!acc) launch_fill(s, n, 0.f, y);
    return;
  }
  const int rb = gemv_t_row_blocks(m, n, p == CF_FP8_E4M3 ? 4 : 8);  // <= the workspace's (8)
  const int64_t rows_per_block = (m + rb - 1) / rb;
  const int threads = p == CF_FP32 ? 256 : (p == CF_BF16 ? 128 : 64 * gemv_t_groups<__nv_fp8_e4m3>());
  dim3 grid((unsigned)((n + kGemvTCols - 1) / kGemvTCols), (unsigned)rb);
  if (p == CF_FP32)
    k_gemv_t_part<float><<<grid, threads, 0, s>>>(m, n, lda, rows_per_block, (const float*)A, rs, x, ws, sin);
  else if (p == CF_BF16)
    k_gemv_t_part<__nv_bfloat16><<<grid, threads, 0, s>>>(m, n, lda, rows_per_block, (const __nv_bfloat16*)A, rs, x,
                                                          ws, sin);
  else
    k_gemv_t_part<__nv_fp8_e4m3><<<grid, threads, 0, s>>>(m, n, lda, rows_per_block, (const __nv_fp8_e4m3*)A, rs, x,
                                                          ws, sin);
  k_gemv_t_reduce<<<(unsigned)((n + 31) / 32), 32 * kGemvTRedRows, 0, s>>>(n, lda, rb, ws, alpha, y, acc, sout);
}

// ------------------------------------------------------------ quantisation
// One CTA per row: row max, then codes (the stored operand defines the
// problem instance).  Columns n..lda-1 are zero padding.
__global__ void k_quantize(cf_prec p, int64_t n, int64_t lda, const float* __restrict__ src,
                           void* __restrict__ dst, float* __restrict__ rs) {
  const int64_t row = blockIdx.x;
  const float* a = src + row * n;
  __shared__ float smax[32];
  __shared__ float s_scale;
  float scale = 1.f;
  if (p == CF_FP8_E4M3) {
    float mx = 0.f;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(a[j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, smax[w]);
      s_scale = t > 0.f ? t / 448.0f : 1.0f;
      rs[row] = s_scale;
    }
    __syncthreads();
    scale = s_scale;
  }
  for (int64_t j = threadIdx.x; j < lda; j += blockDim.x) {
    float v = j < n ? a[j] : 0.f;
    if (p == CF_FP32) {
      ((float*)dst)[row * lda + j] = v;
    } else if (p == CF_BF16) {
      ((__nv_bfloat16*)dst)[row * lda + j] = __float2bfloat16_rn(v);
    } else {
      float q = v / scale;
      ((__nv_fp8_storage_t*)dst)[row * lda + j] = __nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    }
  }
}

void launch_quantize(cudaStream_t s, cf_prec p, int64_t m, int64_t n, int64_t lda,
                     const float* src, void* dst, float* rs) {
  if (m <= 0) return;
  k_quantize<<<(unsigned)m, 256, 0, s>>>(p, n, lda, src, dst, rs);
}

// ------------------------------------------------------------ CSR SpMV
// Warps are persistent (the grid is what fits on the GPU at once) and walk
// rows row, row + W, ... (W warps in the grid).  A row's first 32 U entries
// are held as U (index, value) pairs a lane; while the warp gathers x for
// the current row and sums it, the index and value loads of its next row and
// the row-pointer loads of the row after are already in flight, so a row
// costs about one memory latency instead of three (row pointers -> entries
// -> x).  Entries past 32 U in a row (rows far above the average) are taken
// by a plain strided loop.  U = 16 for matrices that average more than 256
// entries a row, else 8.
template <bool BF16>
__device__ __forceinline__ float csr_val(const void* __restrict__ val, int32_t k) {
  return BF16 ? __bfloat162float(__ldg(((const __nv_bfloat16*)val) + k)) : __ldg(((const float*)val) + k);
}

template <bool BF16, int U>
__device__ __forceinline__ void csr_fetch(const int32_t* __restrict__ col, const void* __restrict__ val, int32_t b,
                                          int32_t e, int lane, int32_t (&c)[U], float (&v)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int32_t k = b + lane + 32 * u;
    c[u] = k < e ? __ldg(col + k) : -1;
    v[u] = k < e ? csr_val<BF16>(val, k) : 0.f;
  }
}

// SC: input / output scalings (sin, sout) are applied.
template <bool BF16, bool SC, int U>
__global__ void __launch_bounds__(256)
k_csr(int64_t m, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
      const void* __restrict__ val, float alpha, const float* __restrict__ x,
      float* __restrict__ y, bool acc, const float* __restrict__ sin, const float* __restrict__ sout) {
  const int lane = threadIdx.x & 31;
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= m) return;
  auto xin = [&](int32_t j) { return SC ? __ldg(sin + j) * __ldg(x + j) : __ldg(x + j); };
  int32_t b = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
  int32_t c[U];
  float v[U];
  csr_fetch<BF16, U>(col, val, b, e, lane, c, v);
  int32_t b1 = 0, e1 = 0;
  if (row + W < m) { b1 = __ldg(rowptr + row + W); e1 = __ldg(rowptr + row + W + 1); }
  while (true) {
    float xg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xg[u] = c[u] >= 0 ? xin(c[u]) : 0.f;
    const int64_t next = row + W;
    int32_t cn[U];
    float vn[U];
    int32_t b2 = 0, e2 = 0;
    if (next < m) {
      csr_fetch<BF16, U>(col, val, b1, e1, lane, cn, vn);
      if (next + W < m) { b2 = __ldg(rowptr + next + W); e2 = __ldg(rowptr + next + W + 1); }
    }
    float s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) s[u] = v[u] * xg[u];
    for (int32_t k = b + lane + 32 * U; k < e; k += 32) {
      const int32_t j = __ldg(col + k);
      s[0] = fmaf(csr_val<BF16>(val, k), xin(j), s[0]);
    }
#pragma unroll
    for (int w = U / 2; w > 0; w >>= 1)
#pragma unroll
      for (int u = 0; u < w; ++u) s[u] += s[u + w];
    float sum = s[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0) {
      float out = (SC ? alpha * __ldg(sout + row) : alpha) * sum;
      y[row] = acc ? y[row] + out : out;
    }
    if (next >= m) break;
    row = next;
    b = b1;
    e = e1;
    b1 = b2;
    e1 = e2;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = cn[u];
      v[u] = vn[u];
    }
  }
}

// The persistent grid: CTAs that fit at once (occupancy x SMs), no more
// than the rows need.  Cached per kernel instance.
template <bool BF16, bool SC, int U>
static unsigned csr_grid(int64_t m) {
  static const int resident = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_csr<BF16, SC, U>, 256, 0);
    return std::max(1, sms * std::max(per_sm, 1));
  }();
  return (unsigned)std::min<int64_t>((m + 7) / 8, resident);
}

template <bool BF16, bool SC, int U>
static void csr_launch_one(cudaStream_t s, int64_t m, const int32_t* rowptr, const int32_t* col, const void* val,
                           float alpha, const float* x, float* y, bool acc, const float* sin, const float* sout) {
  k_csr<BF16, SC, U><<<csr_grid<BF16, SC, U>(m), 256, 0, s>>>(m, rowptr, col, val, alpha, x, y, acc, sin, sout);
}

template <int U>
static void csr_launch_u(cudaStream_t s, cf_prec p, int64_t m, const int32_t* rowptr, const int32_t* col,
                         const void* val, float alpha, const float* x, float* y, bool acc, const float* sin,
                         const float* sout) {
  // both scalings or none (op_apply folds a product only when both diagonals are stored)
  if (sin || sout) {
    if (p == CF_BF16)
      csr_launch_one<true, true, U>(s, m, rowptr, col, val, alpha, x, y, acc, sin, sout);
    else
      csr_launch_one<false, true, U>(s, m, rowptr, col, val, alpha, x, y, acc, sin, sout);
  } else if (p == CF_BF16) {
    csr_launch_one<true, false, U>(s, m, rowptr, col, val, alpha, x, y, acc, nullptr, nullptr);
  } else {
    csr_launch_one<false, false, U>(s, m, rowptr, col, val, alpha, x, y, acc, nullptr, nullptr);
  }
}

void csr_prepare() {
  const int64_t big = INT32_MAX;
  (void)csr_grid<false, false, 8>(big); (void)csr_grid<true, false, 8>(big);
  (void)csr_grid<false, true, 8>(big); (void)csr_grid<true, true, 8>(big);
  (void)csr_grid<false, false, 16>(big); (void)csr_grid<true, false, 16>(big);
  (void)csr_grid<false, true, 16>(big); (void)csr_grid<true, true, 16>(big);
}

void launch_csr(cudaStream_t s, cf_prec p, int64_t m, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                const void* val, float alpha, const float* x, float* y, bool acc, const float* sin,
                const float* sout) {
  if (m <= 0) return;
  if (nnz > 256 * m)
    csr_launch_u<16>(s, p, m, rowptr, col, val, alpha, x, y, acc, sin, sout);
  else
    csr_launch_u<8>(s, p, m, rowptr, col, val, alpha, x, y, acc, sin, sout);
}

// ------------------------------------------------------------ small GEMM
// C (M x N, row-major, ldc = N) = alpha op(A) op(B) + (acc ? C : 0) for the
// Kronecker operator's two factor products; 16 x 16 shared-memory tiles.
constexpr int kGT = 16;

__global__ void k_gemm(int64_t M, int64_t N, int64_t K, const float* __restrict__ A, int64_t lda,
                       bool ta, const float* __restrict__ B, int64_t ldb, bool tb, float alpha,
                       float* __restrict__ C, bool acc) {
  __shared__ float As[kGT][kGT + 1], Bs[kGT][kGT + 1];
  const int64_t row = (int64_t)blockIdx.y * kGT + threadIdx.y;
  const int64_t colj = (int64_t)blockIdx.x * kGT + threadIdx.x;
  float sum = 0.f;
  for (int64_t k0 = 0; k0 < K; k0 += kGT) {
    int64_t ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] =
        (row < M && ka < K) ? (ta ? A[ka * lda + row] : A[row * lda + ka]) : 0.f;
    Bs[threadIdx.y][threadIdx.x] =
        (kb < K && colj < N) ? (tb ? B[colj * ldb + kb] : B[kb * ldb + colj]) : 0.f;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGT; ++k) sum = fmaf(As[threadIdx.y][k], Bs[k][threadIdx.x], sum);
    __syncthreads();
  }
  if (row < M && colj < N) {
    float v = alpha * sum;
    C[row * N + colj] = acc ? C[row * N + colj] + v : v;
  }
}

void launch_gemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                 bool ta, const float* B, int64_t ldb, bool tb, float alpha, float* C, bool acc) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)((N + kGT - 1) / kGT), (unsigned)((M + kGT - 1) / kGT));
  k_gemm<<<grid, dim3(kGT, kGT), 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, alpha, C, acc);
}

}  // namespace cf
