// Internal declarations shared by the translation units of libcvxb300.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <atomic>
#include <mutex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cvxb300.h"

namespace cf {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
cf_err fail(cf_err code, const std::string& msg);
cf_err cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CF_CUDA(expr)                                                       \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess) return ::cf::cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

#define CF_TRY(expr)                 \
  do {                               \
    cf_err _r = (expr);              \
    if (_r != CF_OK) return _r;      \
  } while (0)

// Copy between any two addresses (host or device) through unified addressing.
cf_err copy_any(void* dst, const void* src, size_t bytes, cudaStream_t s);
bool is_device_ptr(const void* p);

constexpr int kThreads = 256;       // block size of the vector kernels
constexpr int kMaxRedBlocks = 1184; // 148 SMs x 8: cap on reduction grids
constexpr int kRedSlots = 8;        // doubles per block in a partial-sum buffer

inline int grid_for(int64_t n, int per_thread = 4) {
  int64_t g = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  if (g < 1) g = 1;
  if (g > kMaxRedBlocks) g = kMaxRedBlocks;
  return (int)g;
}

// Grids of kernels that end in a grid-wide sum: 2 CTAs per SM.  Every CTA
// pays a fence and an atomic ticket on one counter, which on this two-die
// GPU costs more than the extra elements per thread do.
constexpr int kRedGrid = 296;
inline int red_grid(int64_t n) {
  int g = grid_for(n);
  return g < kRedGrid ? g : kRedGrid;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Team-engine schedule held by a new context.
cf_schedule default_schedule();
bool schedule_valid(const cf_schedule& s, std::string* why);

}  // namespace cf

// ----------------------------------------------------------------- context
struct cf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 148;
  std::mutex sched_mu;   // guards sched
  cf_schedule sched{};   // team-engine launch schedule
};

// ---------------------------------------------------------------- operators
enum OpKind {
  OP_DENSE, OP_CSR, OP_CONV1D, OP_CONV2D, OP_DIAG, OP_ZERO,
  OP_VSTACK, OP_HSTACK, OP_BLOCKDIAG, OP_PRODUCT, OP_SUM, OP_SCALE, OP_ADJOINT, OP_KRON
};

struct cf_op {
  std::atomic<int> refs{1};
  cf_ctx* ctx = nullptr;
  int device = 0;  // the context's device, kept so that freeing never reads the context
  OpKind kind = OP_ZERO;
  int64_t m = 0, n = 0;
  std::vector<cf_op*> parts;
  double alpha = 1.0;
  // dense: row-major, leading dimension lda >= n (multiple of 16 elements)
  cf_prec prec = CF_FP32;
  void* a = nullptr;
  float* row_scale = nullptr;
  int64_t lda = 0;
  // csr (and its transpose, built at creation for a deterministic adjoint);
  // col / val arrays padded with zeros to whole 8-entry chunks plus one chunk
  int64_t nnz = 0;
  int32_t *rowptr = nullptr, *col = nullptr, *t_rowptr = nullptr, *t_col = nullptr;
  void *val = nullptr, *t_val = nullptr;
  // conv1d: taps reversed and zero-padded to Lp (multiple of 16), for the
  // forward map and for the adjoint (whose taps are k reversed)
  int64_t L = 0, Lp = 0;
  float *w_fwd = nullptr, *w_adj = nullptr;
  // conv1d by overlap-save FFTs (when chosen): the twiddle table and the
  // spectra of the forward and adjoint taps (see k_fftconv.cu)
  float2 *fft_tw = nullptr, *fft_hf = nullptr, *fft_ha = nullptr;
  int fft_n = 0;  // transform size of the FFT method (4096 or 2048)
  // conv2d
  int64_t h = 0, w = 0, kh = 0, kw = 0;
  float *k2_fwd = nullptr, *k2_adj = nullptr;
  // diag (nullptr: identity)
  float* d = nullptr;
  size_t device_bytes = 0;  // bytes this node itself owns on the device
};

namespace cf {

// Makes `dev` current for the scope and clears any error an unrelated earlier
// runtime call left behind, so that the error checks after this library's
// launches report only its own failures.
struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetLastError();
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Workspace (float count) op_apply needs for this node and below.
size_t op_ws_floats(const cf_op* op, bool trans);
// Device bytes of the whole tree (shared parts counted once per reference).
size_t op_tree_bytes(const cf_op* op);
// y = alpha * op(x) + (acc ? y : 0), op(x) = A x or A^T x; ws: op_ws_floats floats.
// direct_conv: 1-D convolution leaves use the direct sum even where the leaf
// is evaluated by FFTs (entrywise float32 accuracy instead of a per-segment
// 2-norm bound).
// skip_parts: when the operator is a vstack (possibly inside the
// equilibration product), parts k with skip_parts[k] != 0 are left out: no
// outputs written forward, no contribution adjoint.
void op_apply(const cf_op* op, bool trans, float alpha, const float* x, float* y, bool acc,
              float* ws, cudaStream_t s, bool direct_conv = false, const uint8_t* skip_parts = nullptr);

// Row blocks of a vstack operator that are one diagonal leaf on a column
// slice (the other leaves of the block zero): rows [r0, r0 + len) of A hold
// alpha d_j at column c0 + j (d == nullptr: the identity).  Such a block adds
// the diagonal alpha^2 d^2 to A^T A, and its rows of A z are alpha d z[cols],
// so the solver folds it out of its CG passes.
constexpr int kMaxFold = 4;
struct DiagBlock {
  int64_t r0, c0, len;
  float alpha;
  const float* d;
};
// Fills `blocks` (at most kMaxFold) and `skip` (one flag per vstack part) for
// the solver's operator A (the core of an equilibration product, if any);
// false when nothing can be folded or nothing would remain.
bool fold_diag_blocks(const cf_op* A, std::vector<DiagBlock>* blocks, std::vector<uint8_t>* skip);
void op_retain(cf_op* op);

// ---- elementwise segments: y = sout * sum_k alpha_k d_k sin_k x_k (+ y if
// acc); no terms and acc == 0 is a zero fill.  Several independent segments
// go out in one launch.  (sin / sout: diagonal scalings around the operator,
// nullptr = 1.)
constexpr int kEwMaxTerms = 4;
constexpr int kEwMaxSegs = 8;
struct EwSeg {
  float* y;
  int64_t n;
  int acc, nterm;
  const float* x[kEwMaxTerms];
  const float* d[kEwMaxTerms];  // nullptr: identity
  const float* sin[kEwMaxTerms];
  const float* sout;
  float alpha[kEwMaxTerms];
};
struct EwBatch {
  int nseg;
  EwSeg seg[kEwMaxSegs];
};
void launch_ew(cudaStream_t s, const EwBatch& b);

#ifdef __CUDACC__
// Row i of an elementwise segment.
__device__ __forceinline__ float ew_value(const EwSeg& g, int64_t i) {
  float v = g.acc ? g.y[i] : 0.f;
  const float so = g.sout ? g.sout[i] : 1.f;
  for (int k = 0; k < g.nterm; ++k) {
    const float xv = g.sin[k] ? g.sin[k][i] * g.x[k][i] : g.x[k][i];
    v = fmaf(g.sout ? g.alpha[k] * so : g.alpha[k], g.d[k] ? g.d[k][i] * xv : xv, v);
  }
  return v;
}
#endif

// ---- leaf launchers (kernels in k_*.cu)
void launch_fill(cudaStream_t s, int64_t n, float v, float* y);
void launch_diag(cudaStream_t s, int64_t n, const float* d, float alpha, const float* x, float* y,
                 bool acc);
// Leaves taking sin / sout compute y (+)= sout * alpha * leaf(sin * x)
// (elementwise scalings of the input and output, nullptr = 1).
void launch_conv1d(cudaStream_t s, int64_t n_out, int64_t n_in, int64_t Lp, int64_t shift,
                   const float* wrev, float alpha, const float* x, float* y, bool acc,
                   const float* sin = nullptr, const float* sout = nullptr);
// The same operation as launch_conv1d by overlap-save FFTs of fft_n points
// (4096, or 2048 when Lp <= kFftConv2048MaxLp and the larger transform would
// leave SMs idle; Lp <= kFftConvMaxLp); H = the spectrum of the taps in the
// kernel's order, scaled by 1 / fft_n (fft_n values); tw = the kernel's
// twiddle tables (fft_n + fft_n / 16 values; fftconv.cuh gives both layouts).
constexpr int kFftConvN = 4096;            // largest transform
constexpr int kFftConvMaxLp = 2048;
constexpr int kFftConv2048MaxLp = 1024;    // the 2048-point transform keeps >= half its outputs
constexpr int kFftConvAutoMinLp = 256;     // CF_CONV_AUTO uses the FFT from here on
constexpr int kFftConvTw = kFftConvN + 256;
cf_err conv1d_fft_prepare(int device);  // once per device before the first launch (not during capture)
void launch_conv1d_fft(cudaStream_t s, int fft_n, int64_t n_out, int64_t n_in, int64_t Lp, int64_t shift,
                       const float2* H, const float2* tw, float alpha, const float* x, float* y, bool acc,
                       const float* sin = nullptr, const float* sout = nullptr);
void launch_conv2d(cudaStream_t s, int64_t Ho, int64_t Wo, int64_t Hi, int64_t Wi, int64_t kh,
                   int64_t kw, int64_t sh, int64_t sw, const float* kern, float alpha,
                   const float* x, float* y, bool acc);
void launch_gemv_n(cudaStream_t s, cf_prec p, int64_t m, int64_t n, int64_t lda, const void* A,
                   const float* rs, float alpha, const float* x, float* y, bool acc,
                   const float* sin = nullptr, const float* sout = nullptr);
size_t gemv_t_ws_floats(int64_t m, int64_t n, int64_t lda);
void launch_gemv_t(cudaStream_t s, cf_prec p, int64_t m, int64_t n, int64_t lda, const void* A,
                   const float* rs, float alpha, const float* x, float* y, bool acc, float* ws,
                   const float* sin = nullptr, const float* sout = nullptr);
// Resident-grid sizes of the CSR kernels, queried once per process before the
// first launch (at operator creation, not during stream capture).
void csr_prepare();
void launch_csr(cudaStream_t s, cf_prec p, int64_t m, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                const void* val, float alpha, const float* x, float* y, bool acc,
                const float* sin = nullptr, const float* sout = nullptr);
void launch_gemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                 bool ta, const float* B, int64_t ldb, bool tb, float alpha, float* C, bool acc);
void launch_quantize(cudaStream_t s, cf_prec p, int64_t m, int64_t n, int64_t lda,
                     const float* src, void* dst, float* rs);

}  // namespace cf
