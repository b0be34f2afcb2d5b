// The team engine's data: an operator tree flattened into a list of leaf
// terms, and the per-problem table entry its persistent kernel reads.
#pragma once

#include <string>
#include <vector>

#include "internal.cuh"

namespace cf {

struct Ctl;

namespace team {

constexpr int kMaxSeg = 4;          // second-order cones per problem
constexpr int kConvMaxLp = 2048;    // padded taps of a 1-D convolution leaf
constexpr int kConvTile = 4096;     // convolution outputs per shared-memory tile
constexpr int kDenseMaxCols = 16384;// forward dense input staged in shared memory
constexpr int kDenseTGroups = 16;   // row groups of the adjoint dense product
constexpr int kCsrStageFloats = 40960; // CSR input staged in shared memory up to this length

enum TermKind : int32_t { T_FILL = 0, T_DIAG = 1, T_CSR = 2, T_DENSE_N = 3, T_DENSE_T = 4, T_CONV = 5, T_FFT = 6 };

// One leaf application y[yo : yo + rows] (+)= sout * alpha * leaf(sin * x[xo : xo + cols]).
// `sync`: a team barrier runs first (an earlier term since the last barrier
// wrote overlapping outputs under another partition of the rows).
struct __align__(16) Term {
  int32_t kind, acc, sync, prec;
  int64_t xo, yo, rows, cols;
  float alpha;
  int32_t fftn;           // FFT convolution: transform size (4096 or 2048)
  const void* a;          // dense / CSR values, reversed conv taps, diagonal (may be null)
  const float* scale;     // per-row scales of an FP8 dense leaf
  const int32_t* rowptr;  // CSR (for the adjoint: the stored transpose)
  const int32_t* col;
  int64_t lda, Lp, shift; // dense leading dimension; conv padded taps and shift
  const float2* tw;       // FFT convolution: twiddle tables (a: the spectrum)
  // diagonal scalings around the leaf (equilibration), aligned with the
  // term's slices: x[xo + j] is read as sin[j] x[xo + j], and the term's
  // result for y[yo + i] is multiplied by sout[i]; null means 1
  const float* sin;
  const float* sout;
};

// A problem's flattened operator: forward (t = A p), adjoint (q = A^T t) and
// the right-hand-side form (rhs -= A^T w), with the sizes the launch needs.
struct Plan {
  bool ok = false;
  std::string why;          // reason when !ok
  std::vector<Term> fwd, adj, adj_m;
  double pass_bytes = 0;    // bytes (and flop-equivalents) of one forward pass
  double avg_row_nnz = 0;   // CSR leaves of the forward pass
  int64_t dense_t_cols = 0; // widest adjoint dense output (row-group partials)
  int64_t smem_floats = 0;  // dynamic shared memory the terms need (FFT terms aside)
  bool has_fft = false;     // FFT convolution terms: one transform buffer per 256 threads
};

}  // namespace team
}  // namespace cf
