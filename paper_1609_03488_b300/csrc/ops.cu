// Operator trees: leaves own device data, compositions reference their parts
// (Section 3.1's structured linear operators; Section 4.1's adjoint by graph
// transformation: the adjoint of a composition is formed node by node --
// vstack <-> hstack, products reversed -- and never materialised).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>

#include "internal.cuh"

namespace cf {

void op_retain(cf_op* op) { op->refs.fetch_add(1); }

static void op_free(cf_op* op) {
  for (cf_op* p : op->parts) cf_op_destroy(p);
  void* bufs[] = {op->a, op->row_scale, op->rowptr, op->col, op->t_rowptr, op->t_col,
                  op->val, op->t_val, op->w_fwd, op->w_adj, op->k2_fwd, op->k2_adj, op->d,
                  op->fft_tw, op->fft_hf, op->fft_ha};
  {
    DevGuard g(op->device);
    for (void* b : bufs)
      if (b) cudaFree(b);
  }
  delete op;
}

size_t op_tree_bytes(const cf_op* op) {
  size_t s = op->device_bytes;
  for (const cf_op* p : op->parts) s += op_tree_bytes(p);
  return s;
}

static size_t al16(size_t n) { return align_up(n, 16); }

size_t op_ws_floats(const cf_op* op, bool trans) {
  switch (op->kind) {
    case OP_DENSE:
      return trans ? al16(gemv_t_ws_floats(op->m, op->n, op->lda)) : 0;
    case OP_CSR: case OP_CONV1D: case OP_CONV2D: case OP_DIAG: case OP_ZERO:
      return 0;
    case OP_SCALE:
      return op_ws_floats(op->parts[0], trans);
    case OP_ADJOINT:
      return op_ws_floats(op->parts[0], !trans);
    case OP_VSTACK: case OP_HSTACK: case OP_BLOCKDIAG: case OP_SUM: {
      size_t mx = 0;
      for (const cf_op* p : op->parts) mx = std::max(mx, op_ws_floats(p, trans));
      return mx;
    }
    case OP_PRODUCT: {
      // two ping-pong intermediates of the largest inner dimension
      int64_t inner = 0;
      for (size_t i = 0; i + 1 < op->parts.size(); ++i) inner = std::max(inner, op->parts[i]->n);
      size_t mx = 0;
      for (const cf_op* p : op->parts) mx = std::max(mx, op_ws_floats(p, trans));
      return 2 * al16((size_t)inner) + mx;
    }
    case OP_KRON: {
      const cf_op *A = op->parts[0], *B = op->parts[1];
      return al16((size_t)std::max(A->n * B->m, A->m * B->n));
    }
  }
  return 0;
}

namespace {

bool overlap(const float* a, int64_t na, const float* b, int64_t nb) {
  return a < b + nb && b < a + na;
}

// Pending elementwise leaf operations of one tree walk, launched together.
struct EwQueue {
  EwBatch b{};
  cudaStream_t s;
  bool direct_conv = false;  // evaluate FFT-method convolution leaves by the direct sum
  explicit EwQueue(cudaStream_t st) : s(st) { b.nseg = 0; }
  void flush() {
    launch_ew(s, b);
    b.nseg = 0;
  }
  // y = sout alpha d (sin x) (+ y): nterm 0 is a zero fill.
  void add(float* y, int64_t n, bool acc, const float* x, const float* d, float alpha, bool fill,
           const float* sin = nullptr, const float* sout = nullptr) {
    // same output and output scaling (a pending zero fill has no terms to
    // scale and takes this one's), accumulating, no reads of pending outputs:
    // one more term
    for (int k = 0; k < b.nseg; ++k) {
      EwSeg& g = b.seg[k];
      const bool bare_fill = g.nterm == 0 && !g.acc;
      if (!fill && acc && g.y == y && g.n == n && g.nterm < kEwMaxTerms && (g.sout == sout || bare_fill)) {
        bool hazard = false;
        for (int j = 0; j < b.nseg; ++j) hazard |= overlap(x, n, b.seg[j].y, b.seg[j].n);
        if (!hazard) {
          if (bare_fill) g.sout = sout;
          g.x[g.nterm] = x;
          g.d[g.nterm] = d;
          g.sin[g.nterm] = sin;
          g.alpha[g.nterm] = alpha;
          ++g.nterm;
          return;
        }
      }
    }
    bool hazard = b.nseg == kEwMaxSegs;
    for (int j = 0; j < b.nseg && !hazard; ++j) {
      const EwSeg& g = b.seg[j];
      hazard |= overlap(y, n, g.y, g.n);                       // write after write
      if (!fill) hazard |= overlap(x, n, g.y, g.n);            // read after write
      for (int k = 0; k < g.nterm; ++k) hazard |= overlap(g.x[k], g.n, y, n);  // write after read
    }
    if (hazard) flush();
    EwSeg& g = b.seg[b.nseg++];
    g.y = y;
    g.n = n;
    g.acc = acc ? 1 : 0;
    g.nterm = fill ? 0 : 1;
    g.sout = fill ? nullptr : sout;
    if (!fill) {
      g.x[0] = x;
      g.d[0] = d;
      g.sin[0] = sin;
      g.alpha[0] = alpha;
    }
  }
};

// Scalings around a subtree, aligned with its x (in) and y (out); nullptr = 1.
struct Scales {
  const float* in = nullptr;
  const float* out = nullptr;
  Scales shift(int64_t dx, int64_t dy) const {
    return Scales{in ? in + dx : nullptr, out ? out + dy : nullptr};
  }
};

void op_apply_rec(const cf_op* op, bool trans, float alpha, const float* x, float* y, bool acc,
                  float* ws, cudaStream_t s, EwQueue& q, Scales sc, const uint8_t* skip = nullptr);

// Whether every leaf below takes input / output scalings.
bool scalable(const cf_op* op) {
  switch (op->kind) {
    case OP_DENSE: case OP_CSR: case OP_CONV1D: case OP_DIAG: case OP_ZERO:
      return true;
    case OP_VSTACK: case OP_HSTACK: case OP_BLOCKDIAG: case OP_SUM: case OP_SCALE: case OP_ADJOINT:
      for (const cf_op* p : op->parts)
        if (!scalable(p)) return false;
      return true;
    default:
      return false;
  }
}

}  // namespace

// y = alpha * op(x) + (acc ? y : 0).  An equilibrated operator
// diag(D) A diag(E) whose leaves all take scalings is applied as A with the
// two diagonals folded into A's leaf kernels (no separate passes).
void op_apply(const cf_op* op, bool trans, float alpha, const float* x, float* y, bool acc,
              float* ws, cudaStream_t s, bool direct_conv, const uint8_t* skip_parts) {
  EwQueue q(s);
  q.direct_conv = direct_conv;
  if (op->kind == OP_PRODUCT && op->parts.size() == 3 && op->parts[0]->kind == OP_DIAG &&
      op->parts[2]->kind == OP_DIAG && op->parts[0]->d && op->parts[2]->d && scalable(op->parts[1])) {
    const float* D = op->parts[0]->d;
    const float* E = op->parts[2]->d;
    op_apply_rec(op->parts[1], trans, alpha, x, y, acc, ws, s, q, trans ? Scales{D, E} : Scales{E, D}, skip_parts);
  } else {
    op_apply_rec(op, trans, alpha, x, y, acc, ws, s, q, Scales{}, skip_parts);
  }
  q.flush();
}

namespace {

// A diagonal leaf (possibly under scale nodes): its product of scales and d.
bool diag_leaf(const cf_op* op, float* alpha, const float** d) {
  float a = 1.f;
  while (op->kind == OP_SCALE) {
    a *= (float)op->alpha;
    op = op->parts[0];
  }
  if (op->kind != OP_DIAG) return false;
  *alpha = a;
  *d = op->d;
  return true;
}

}  // namespace

bool fold_diag_blocks(const cf_op* A, std::vector<DiagBlock>* blocks, std::vector<uint8_t>* skip) {
  blocks->clear();
  skip->clear();
  const cf_op* core = A;
  if (A->kind == OP_PRODUCT && A->parts.size() == 3 && A->parts[0]->kind == OP_DIAG &&
      A->parts[2]->kind == OP_DIAG && A->parts[0]->d && A->parts[2]->d) {
    if (!scalable(A->parts[1])) return false;  // op_apply would not fold the scalings
    core = A->parts[1];
  }
  if (core->kind != OP_VSTACK) return false;
  skip->assign(core->parts.size(), 0);
  int64_t r0 = 0;
  size_t kept = 0;
  for (size_t k = 0; k < core->parts.size(); ++k) {
    const cf_op* p = core->parts[k];
    float alpha = 1.f;
    const float* d = nullptr;
    int64_t c0 = -1;
    if (diag_leaf(p, &alpha, &d)) {
      c0 = 0;
    } else if (p->kind == OP_HSTACK) {
      int64_t off = 0;
      int ndiag = 0;
      bool other = false;
      for (const cf_op* c : p->parts) {
        float a2;
        const float* d2;
        if (c->kind == OP_ZERO) {
        } else if (diag_leaf(c, &a2, &d2)) {
          ++ndiag;
          alpha = a2;
          d = d2;
          c0 = off;
        } else {
          other = true;
        }
        off += c->n;
      }
      if (other || ndiag != 1) c0 = -1;
    }
    if (c0 >= 0 && blocks->size() < (size_t)kMaxFold) {
      blocks->push_back(DiagBlock{r0, c0, p->m, alpha, d});
      (*skip)[k] = 1;
    } else {
      ++kept;
    }
    r0 += p->m;
  }
  if (blocks->empty() || kept == 0) {
    blocks->clear();
    skip->clear();
    return false;
  }
  return true;
}

namespace {

void op_apply_rec(const cf_op* op, bool trans, float alpha, const float* x, float* y, bool acc,
                  float* ws, cudaStream_t s, EwQueue& q, Scales sc, const uint8_t* skip) {
  const int64_t out_dim = trans ? op->n : op->m;
  // Elementwise leaves are queued; any other leaf first launches the queue,
  // so operations keep their order wherever they could interact.
  if (op->kind != OP_ZERO && op->kind != OP_DIAG && op->kind != OP_SCALE && op->kind != OP_ADJOINT &&
      op->kind != OP_VSTACK && op->kind != OP_HSTACK && op->kind != OP_BLOCKDIAG && op->kind != OP_SUM &&
      op->kind != OP_PRODUCT)
    q.flush();
  switch (op->kind) {
    case OP_ZERO:
      if (!acc) q.add(y, out_dim, false, nullptr, nullptr, 0.f, true);
      return;
    case OP_DIAG:
      q.add(y, op->n, acc, x, op->d, alpha, false, sc.in, sc.out);
      return;
    case OP_DENSE:
      if (!trans)
        launch_gemv_n(s, op->prec, op->m, op->n, op->lda, op->a, op->row_scale, alpha, x, y, acc, sc.in, sc.out);
      else
        launch_gemv_t(s, op->prec, op->m, op->n, op->lda, op->a, op->row_scale, alpha, x, y, acc, ws, sc.in,
                      sc.out);
      return;
    case OP_CSR:
      if (!trans)
        launch_csr(s, op->prec, op->m, op->nnz, op->rowptr, op->col, op->val, alpha, x, y, acc, sc.in, sc.out);
      else
        launch_csr(s, op->prec, op->n, op->nnz, op->t_rowptr, op->t_col, op->t_val, alpha, x, y, acc, sc.in,
                   sc.out);
      return;
    case OP_CONV1D: {
      const int64_t nx = op->n, ny = op->m;
      if (op->fft_tw && !q.direct_conv) {
        if (!trans)
          launch_conv1d_fft(s, op->fft_n, ny, nx, op->Lp, 0, op->fft_hf, op->fft_tw, alpha, x, y, acc, sc.in, sc.out);
        else
          launch_conv1d_fft(s, op->fft_n, nx, ny, op->Lp, op->Lp - 1, op->fft_ha, op->fft_tw, alpha, x, y, acc,
                            sc.in, sc.out);
      } else if (!trans) {
        launch_conv1d(s, ny, nx, op->Lp, 0, op->w_fwd, alpha, x, y, acc, sc.in, sc.out);
      } else {
        launch_conv1d(s, nx, ny, op->Lp, op->Lp - 1, op->w_adj, alpha, x, y, acc, sc.in, sc.out);
      }
      return;
    }
    case OP_CONV2D: {
      const int64_t Ho = op->h + op->kh - 1, Wo = op->w + op->kw - 1;
      if (!trans)
        launch_conv2d(s, Ho, Wo, op->h, op->w, op->kh, op->kw, 0, 0, op->k2_fwd, alpha, x, y, acc);
      else
        launch_conv2d(s, op->h, op->w, Ho, Wo, op->kh, op->kw, op->kh - 1, op->kw - 1, op->k2_adj,
                      alpha, x, y, acc);
      return;
    }
    case OP_SCALE:
      op_apply_rec(op->parts[0], trans, (float)(alpha * op->alpha), x, y, acc, ws, s, q, sc);
      return;
    case OP_ADJOINT:
      op_apply_rec(op->parts[0], !trans, alpha, x, y, acc, ws, s, q, sc);
      return;
    case OP_VSTACK:
    case OP_HSTACK: {
      // "stacked" along the output dimension: vstack forward, hstack adjoint;
      // skipped parts (a vstack's folded diagonal blocks) are left out
      const bool split_out = (op->kind == OP_VSTACK) != trans;
      int64_t off = 0;
      bool first = true;
      for (size_t k = 0; k < op->parts.size(); ++k) {
        const cf_op* p = op->parts[k];
        const bool skipped = skip && op->kind == OP_VSTACK && skip[k];
        if (split_out) {
          if (!skipped) op_apply_rec(p, trans, alpha, x, y + off, acc, ws, s, q, sc.shift(0, off));
          off += trans ? p->n : p->m;
        } else {
          if (!skipped) {
            op_apply_rec(p, trans, alpha, x + off, y, first ? acc : true, ws, s, q, sc.shift(off, 0));
            first = false;
          }
          off += trans ? p->m : p->n;
        }
      }
      return;
    }
    case OP_BLOCKDIAG: {
      int64_t ro = 0, co = 0;
      for (const cf_op* p : op->parts) {
        const int64_t din = trans ? p->m : p->n, dout = trans ? p->n : p->m;
        op_apply_rec(p, trans, alpha, x + ro, y + co, acc, ws, s, q, sc.shift(ro, co));
        ro += din;
        co += dout;
      }
      return;
    }
    case OP_SUM: {
      bool first = true;
      for (const cf_op* p : op->parts) {
        op_apply_rec(p, trans, alpha, x, y, first ? acc : true, ws, s, q, sc);
        first = false;
      }
      return;
    }
    case OP_PRODUCT: {
      // forward: apply P_k ... P_1 right to left; adjoint: P_1^T first.
      // (Scalings never reach a product: op_apply folds them only into
      // trees without products.)
      int64_t inner = 0;
      for (size_t i = 0; i + 1 < op->parts.size(); ++i) inner = std::max(inner, op->parts[i]->n);
      float* buf[2] = {ws, ws + al16((size_t)inner)};
      float* rest = ws + 2 * al16((size_t)inner);
      const size_t k = op->parts.size();
      const float* cur = x;
      for (size_t step = 0; step < k; ++step) {
        const cf_op* p = trans ? op->parts[step] : op->parts[k - 1 - step];
        const bool last = step + 1 == k;
        float* dst = last ? y : buf[step & 1];
        op_apply_rec(p, trans, last ? alpha : 1.f, cur, dst, last ? acc : false, rest, s, q, Scales{});
        cur = dst;
      }
      return;
    }
    case OP_KRON: {
      // (A (x) B) vec(X) = vec(A X B^T); adjoint: vec(A^T Y B).
      const cf_op *A = op->parts[0], *B = op->parts[1];
      float* T = ws;
      if (!trans) {
        // T (nA x mB) = X (nA x nB) B^T;  Y (mA x mB) = A T
        launch_gemm(s, A->n, B->m, B->n, x, B->n, false, (const float*)B->a, B->lda, true, 1.f, T, false);
        launch_gemm(s, A->m, B->m, A->n, (const float*)A->a, A->lda, false, T, B->m, false, alpha, y, acc);
      } else {
        // T (mA x nB) = Y (mA x mB) B;  X (nA x nB) = A^T T
        launch_gemm(s, A->m, B->n, B->m, x, B->m, false, (const float*)B->a, B->lda, false, 1.f, T, false);
        launch_gemm(s, A->n, B->n, A->m, (const float*)A->a, A->lda, true, T, B->n, false, alpha, y, acc);
      }
      return;
    }
  }
}

}  // namespace

}  // namespace cf

using namespace cf;

// ------------------------------------------------------------------ C ABI
namespace {

template <typename T>
cf_err dev_alloc(T** p, size_t count, size_t* bytes) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(CF_E_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  *bytes += count * sizeof(T);
  return CF_OK;
}

cf_op* new_op(cf_ctx* ctx, OpKind k, int64_t m, int64_t n) {
  cf_op* op = new cf_op();
  op->ctx = ctx;
  op->device = ctx->device;
  op->kind = k;
  op->m = m;
  op->n = n;
  return op;
}

cf_err finish(cf_op* op, cf_err r, cf_op** out) {
  if (r != CF_OK) {
    cf_op_destroy(op);
    return r;
  }
  *out = op;
  return CF_OK;
}

}  // namespace

extern "C" {

cf_err cf_op_dense(cf_ctx* ctx, int64_t m, int64_t n, const float* A, cf_prec storage,
                   cf_op** out) {
  if (!ctx || !out || !A || m <= 0 || n <= 0)
    return fail(CF_E_INVALID, "cf_op_dense: bad arguments");
  if (storage != CF_FP32 && storage != CF_BF16 && storage != CF_FP8_E4M3)
    return fail(CF_E_INVALID, "cf_op_dense: unknown storage");
  DevGuard g(ctx->device);
  cf_op* op = new_op(ctx, OP_DENSE, m, n);
  op->prec = storage;
  op->lda = (int64_t)align_up((size_t)n, 16);
  auto run = [&]() -> cf_err {
    size_t esz = storage == CF_FP32 ? 4 : (storage == CF_BF16 ? 2 : 1);
    CF_TRY(dev_alloc((uint8_t**)&op->a, (size_t)m * op->lda * esz, &op->device_bytes));
    if (storage == CF_FP8_E4M3) CF_TRY(dev_alloc(&op->row_scale, (size_t)m, &op->device_bytes));
    float* tmp = nullptr;
    size_t dummy = 0;
    CF_TRY(dev_alloc(&tmp, (size_t)m * n, &dummy));
    cf_err r = copy_any(tmp, A, (size_t)m * n * sizeof(float), ctx->stream);
    if (r == CF_OK) {
      launch_quantize(ctx->stream, storage, m, n, op->lda, tmp, op->a, op->row_scale);
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) r = cuda_fail(e, "quantize", __FILE__, __LINE__);
    }
    cudaFree(tmp);
    return r;
  };
  return finish(op, run(), out);
}

cf_err cf_op_csr(cf_ctx* ctx, int64_t m, int64_t n, int64_t nnz, const int32_t* rowptr,
                 const int32_t* col, const float* val, cf_prec storage, cf_op** out) {
  if (!ctx || !out || !rowptr || m <= 0 || n <= 0 || nnz < 0 || (nnz > 0 && (!col || !val)))
    return fail(CF_E_INVALID, "cf_op_csr: bad arguments");
  if (storage != CF_FP32 && storage != CF_BF16)
    return fail(CF_E_INVALID, "cf_op_csr: storage must be CF_FP32 or CF_BF16");
  if (nnz > INT32_MAX) return fail(CF_E_INVALID, "cf_op_csr: nnz exceeds int32");
  DevGuard g(ctx->device);
  csr_prepare();
  // Host copies: validate, then build the transpose (CSR of A^T) by a
  // counting sort over columns, keeping row order inside each column.
  std::vector<int32_t> rp(m + 1), cl(nnz), trp(n + 1, 0), tcl(nnz);
  std::vector<float> vl(nnz), tvl(nnz);
  CF_TRY(copy_any(rp.data(), rowptr, (m + 1) * sizeof(int32_t), ctx->stream));
  if (nnz) {
    CF_TRY(copy_any(cl.data(), col, nnz * sizeof(int32_t), ctx->stream));
    CF_TRY(copy_any(vl.data(), val, nnz * sizeof(float), ctx->stream));
  }
  if (rp[0] != 0 || rp[m] != nnz) return fail(CF_E_INVALID, "cf_op_csr: rowptr[0] != 0 or rowptr[m] != nnz");
  for (int64_t i = 0; i < m; ++i)
    if (rp[i + 1] < rp[i]) return fail(CF_E_INVALID, "cf_op_csr: rowptr not monotone");
  for (int64_t k = 0; k < nnz; ++k) {
    if (cl[k] < 0 || cl[k] >= n) return fail(CF_E_INVALID, "cf_op_csr: column index out of range");
    trp[cl[k] + 1]++;
  }
  for (int64_t j = 0; j < n; ++j) trp[j + 1] += trp[j];
  {
    std::vector<int32_t> fill(trp.begin(), trp.end() - 1);
    for (int64_t i = 0; i < m; ++i)
      for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        int32_t pos = fill[cl[k]]++;
        tcl[pos] = (int32_t)i;
        tvl[pos] = vl[k];
      }
  }
  cf_op* op = new_op(ctx, OP_CSR, m, n);
  op->prec = storage;
  op->nnz = nnz;
  // Index and value arrays hold whole 8-entry chunks plus one spare chunk of
  // zeros, so that a kernel may load any aligned chunk that starts before
  // nnz with 16-byte vector loads.
  const int64_t npad = (int64_t)align_up((size_t)nnz, 8) + 8;
  const size_t vsz = storage == CF_FP32 ? 4 : 2;
  auto run = [&]() -> cf_err {
    CF_TRY(dev_alloc(&op->rowptr, m + 1, &op->device_bytes));
    CF_TRY(dev_alloc(&op->col, npad, &op->device_bytes));
    CF_TRY(dev_alloc(&op->t_rowptr, n + 1, &op->device_bytes));
    CF_TRY(dev_alloc(&op->t_col, npad, &op->device_bytes));
    CF_CUDA(cudaMemset(op->col, 0, npad * 4));
    CF_CUDA(cudaMemset(op->t_col, 0, npad * 4));
    CF_CUDA(cudaMemcpy(op->rowptr, rp.data(), (m + 1) * 4, cudaMemcpyHostToDevice));
    CF_CUDA(cudaMemcpy(op->t_rowptr, trp.data(), (n + 1) * 4, cudaMemcpyHostToDevice));
    if (nnz) {
      CF_CUDA(cudaMemcpy(op->col, cl.data(), nnz * 4, cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(op->t_col, tcl.data(), nnz * 4, cudaMemcpyHostToDevice));
    }
    if (storage == CF_FP32) {
      CF_TRY(dev_alloc((float**)&op->val, npad, &op->device_bytes));
      CF_TRY(dev_alloc((float**)&op->t_val, npad, &op->device_bytes));
    } else {
      CF_TRY(dev_alloc((__nv_bfloat16**)&op->val, npad, &op->device_bytes));
      CF_TRY(dev_alloc((__nv_bfloat16**)&op->t_val, npad, &op->device_bytes));
    }
    CF_CUDA(cudaMemset(op->val, 0, npad * vsz));
    CF_CUDA(cudaMemset(op->t_val, 0, npad * vsz));
    if (storage == CF_FP32) {
      if (nnz) {
        CF_CUDA(cudaMemcpy(op->val, vl.data(), nnz * 4, cudaMemcpyHostToDevice));
        CF_CUDA(cudaMemcpy(op->t_val, tvl.data(), nnz * 4, cudaMemcpyHostToDevice));
      }
    } else {
      std::vector<__nv_bfloat16> b1(nnz), b2(nnz);
      for (int64_t k = 0; k < nnz; ++k) {
        b1[k] = __float2bfloat16_rn(vl[k]);
        b2[k] = __float2bfloat16_rn(tvl[k]);
      }
      if (nnz) {
        CF_CUDA(cudaMemcpy(op->val, b1.data(), nnz * 2, cudaMemcpyHostToDevice));
        CF_CUDA(cudaMemcpy(op->t_val, b2.data(), nnz * 2, cudaMemcpyHostToDevice));
      }
    }
    return CF_OK;
  };
  return finish(op, run(), out);
}

namespace {

// In-place radix-2 FFT in double (natural order in and out), sign -1.
void fft_host(std::vector<std::complex<double>>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1)
    for (size_t i = 0; i < n; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<double> w = std::polar(1.0, -2.0 * M_PI * (double)k / (double)len);
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
}

// Spectrum of h[v] = wrev[Lp - 1 - v] (zero-padded to N) in the FFT kernel's
// order, scaled by 1 / N: after the forward stages the value at position
// p = 16 t + q holds frequency (p >> lg) + 16 ((p >> ls) & 15) + 256 (p & (S-1))
// (G = N/16 = 2^lg, S = G/16 = 2^ls), and thread t reads its q-th factor at
// q (N/16) + t.
std::vector<float2> fft_taps(const std::vector<float>& wrev, int N) {
  const int64_t Lp = (int64_t)wrev.size();
  const int T = N / 16, lg = N == 4096 ? 8 : 7, ls = lg - 4, S = 1 << ls;
  std::vector<std::complex<double>> h(N, 0.0);
  for (int64_t v = 0; v < Lp; ++v) h[v] = wrev[Lp - 1 - v];
  fft_host(h);
  std::vector<float2> out(N);
  for (int p = 0; p < N; ++p) {
    const int k = (p >> lg) + ((p >> ls) & 15) * 16 + (p & (S - 1)) * 256;
    const std::complex<double> v = h[k] / (double)N;
    out[(p & 15) * T + (p >> 4)] = make_float2((float)v.real(), (float)v.imag());
  }
  return out;
}

// The FFT kernel's twiddles: W_N^(t q) at q T + t (t < T = N/16, q < 16),
// then W_G^(j q) at N + q S + j (j < S, q < 16; G = N/16, S = G/16),
// W_M = exp(-2 pi i / M).
std::vector<float2> fft_twiddles(int N) {
  const int T = N / 16, G = N / 16, S = G / 16;
  std::vector<float2> tw(N + G);
  auto w = [](int64_t e, int64_t n) {
    const double th = -2.0 * M_PI * (double)(e % n) / (double)n;
    return make_float2((float)std::cos(th), (float)std::sin(th));
  };
  for (int q = 0; q < 16; ++q)
    for (int t = 0; t < T; ++t) tw[q * T + t] = w((int64_t)t * q, N);
  for (int q = 0; q < 16; ++q)
    for (int j = 0; j < S; ++j) tw[N + q * S + j] = w((int64_t)j * q, G);
  return tw;
}

}  // namespace

cf_err cf_op_conv1d(cf_ctx* ctx, int64_t n, const float* kernel, int64_t L, cf_op** out) {
  return cf_op_conv1d_method(ctx, n, kernel, L, CF_CONV_AUTO, out);
}

cf_err cf_op_conv1d_method(cf_ctx* ctx, int64_t n, const float* kernel, int64_t L, int32_t method, cf_op** out) {
  if (!ctx || !out || !kernel || n <= 0 || L <= 0 || method < CF_CONV_AUTO || method > CF_CONV_FFT)
    return fail(CF_E_INVALID, "cf_op_conv1d: bad arguments");
  const int64_t Lp_ = (int64_t)align_up((size_t)L, 16);
  if (method == CF_CONV_FFT && Lp_ > kFftConvMaxLp)
    return fail(CF_E_INVALID, "cf_op_conv1d: the FFT method takes kernels of at most " +
                                  std::to_string(kFftConvMaxLp) + " taps");
  const bool use_fft = method == CF_CONV_FFT ||
                       (method == CF_CONV_AUTO && Lp_ >= kFftConvAutoMinLp && Lp_ <= kFftConvMaxLp);
  DevGuard g(ctx->device);
  std::vector<float> k(L);
  CF_TRY(copy_any(k.data(), kernel, L * sizeof(float), ctx->stream));
  cf_op* op = new_op(ctx, OP_CONV1D, n + L - 1, n);
  op->L = L;
  op->Lp = Lp_;
  // forward taps w = k padded with zeros to Lp; stored reversed.
  // adjoint taps w' = k reversed (w'[l] = k[L-1-l]); padding zeros at the end
  // shift nothing because the adjoint kernel is called with shift Lp - 1.
  std::vector<float> wf(op->Lp, 0.f), wa(op->Lp, 0.f);
  for (int64_t l = 0; l < L; ++l) wf[op->Lp - 1 - l] = k[l];
  // adjoint: out[j] = sum_l k[l] y[j + l] = sum_{l'} w'[l'] y[j + (Lp-1) - l']
  // with w'[l'] = k[Lp-1-l'] (zero where Lp-1-l' >= L); reversed storage:
  // wrev'[i] = w'[Lp-1-i] = k[i].
  for (int64_t l = 0; l < L; ++l) wa[l] = k[l];
  auto run = [&]() -> cf_err {
    CF_TRY(dev_alloc(&op->w_fwd, op->Lp, &op->device_bytes));
    CF_TRY(dev_alloc(&op->w_adj, op->Lp, &op->device_bytes));
    CF_CUDA(cudaMemcpy(op->w_fwd, wf.data(), op->Lp * 4, cudaMemcpyHostToDevice));
    CF_CUDA(cudaMemcpy(op->w_adj, wa.data(), op->Lp * 4, cudaMemcpyHostToDevice));
    if (use_fft) {
      CF_TRY(conv1d_fft_prepare(ctx->device));
      // 2048-point transforms when the 4096-point ones would give fewer pairs
      // (CTAs) than twice the SMs and the kernel leaves them >= half their outputs
      const int64_t pairs4096 = (n + L - 1 + 2 * (4096 - Lp_ + 1) - 1) / (2 * (4096 - Lp_ + 1));
      const int N = (Lp_ <= kFftConv2048MaxLp && pairs4096 < 2 * (int64_t)ctx->sm_count) ? 2048 : 4096;
      op->fft_n = N;
      const std::vector<float2> tw = fft_twiddles(N), hf = fft_taps(wf, N), ha = fft_taps(wa, N);
      CF_TRY(dev_alloc(&op->fft_tw, tw.size(), &op->device_bytes));
      CF_TRY(dev_alloc(&op->fft_hf, N, &op->device_bytes));
      CF_TRY(dev_alloc(&op->fft_ha, N, &op->device_bytes));
      CF_CUDA(cudaMemcpy(op->fft_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(op->fft_hf, hf.data(), N * sizeof(float2), cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(op->fft_ha, ha.data(), N * sizeof(float2), cudaMemcpyHostToDevice));
    }
    return CF_OK;
  };
  return finish(op, run(), out);
}

cf_err cf_op_conv2d(cf_ctx* ctx, int64_t h, int64_t w, const float* kernel, int64_t kh,
                    int64_t kw, cf_op** out) {
  if (!ctx || !out || !kernel || h <= 0 || w <= 0 || kh <= 0 || kw <= 0)
    return fail(CF_E_INVALID, "cf_op_conv2d: bad arguments");
  if (kh > 64 || kw > 64) return fail(CF_E_INVALID, "cf_op_conv2d: kernel larger than 64 x 64");
  DevGuard g(ctx->device);
  std::vector<float> k(kh * kw), kr(kh * kw);
  CF_TRY(copy_any(k.data(), kernel, kh * kw * sizeof(float), ctx->stream));
  for (int64_t p = 0; p < kh; ++p)
    for (int64_t q = 0; q < kw; ++q) kr[p * kw + q] = k[(kh - 1 - p) * kw + (kw - 1 - q)];
  cf_op* op = new_op(ctx, OP_CONV2D, (h + kh - 1) * (w + kw - 1), h * w);
  op->h = h; op->w = w; op->kh = kh; op->kw = kw;
  auto run = [&]() -> cf_err {
    CF_TRY(dev_alloc(&op->k2_fwd, kh * kw, &op->device_bytes));
    CF_TRY(dev_alloc(&op->k2_adj, kh * kw, &op->device_bytes));
    CF_CUDA(cudaMemcpy(op->k2_fwd, k.data(), kh * kw * 4, cudaMemcpyHostToDevice));
    CF_CUDA(cudaMemcpy(op->k2_adj, kr.data(), kh * kw * 4, cudaMemcpyHostToDevice));
    return CF_OK;
  };
  return finish(op, run(), out);
}

cf_err cf_op_diag(cf_ctx* ctx, int64_t n, const float* d, cf_op** out) {
  if (!ctx || !out || n <= 0) return fail(CF_E_INVALID, "cf_op_diag: bad arguments");
  DevGuard g(ctx->device);
  cf_op* op = new_op(ctx, OP_DIAG, n, n);
  auto run = [&]() -> cf_err {
    if (d) {
      CF_TRY(dev_alloc(&op->d, n, &op->device_bytes));
      CF_TRY(copy_any(op->d, d, n * sizeof(float), ctx->stream));
    }
    return CF_OK;
  };
  return finish(op, run(), out);
}

cf_err cf_op_zero(cf_ctx* ctx, int64_t m, int64_t n, cf_op** out) {
  if (!ctx || !out || m <= 0 || n <= 0) return fail(CF_E_INVALID, "cf_op_zero: bad arguments");
  *out = new_op(ctx, OP_ZERO, m, n);
  return CF_OK;
}

cf_err operator_compose(cf_ctx* ctx, cf_compose_kind kind, cf_op* const* parts, int32_t k,
                        double alpha, cf_op** out) {
  if (!ctx || !out || !parts || k < 1) return fail(CF_E_INVALID, "operator_compose: bad arguments");
  for (int32_t i = 0; i < k; ++i)
    if (!parts[i]) return fail(CF_E_INVALID, "operator_compose: NULL part");
  int64_t m = 0, n = 0;
  OpKind ok;
  switch (kind) {
    case CF_VSTACK:
      ok = OP_VSTACK;
      n = parts[0]->n;
      for (int32_t i = 0; i < k; ++i) {
        if (parts[i]->n != n) return fail(CF_E_INVALID, "vstack: parts differ in column count");
        m += parts[i]->m;
      }
      break;
    case CF_HSTACK:
      ok = OP_HSTACK;
      m = parts[0]->m;
      for (int32_t i = 0; i < k; ++i) {
        if (parts[i]->m != m) return fail(CF_E_INVALID, "hstack: parts differ in row count");
        n += parts[i]->n;
      }
      break;
    case CF_BLOCKDIAG:
      ok = OP_BLOCKDIAG;
      for (int32_t i = 0; i < k; ++i) {
        m += parts[i]->m;
        n += parts[i]->n;
      }
      break;
    case CF_PRODUCT:
      ok = OP_PRODUCT;
      for (int32_t i = 0; i + 1 < k; ++i)
        if (parts[i]->n != parts[i + 1]->m) return fail(CF_E_INVALID, "product: inner dimensions differ");
      m = parts[0]->m;
      n = parts[k - 1]->n;
      break;
    case CF_SUM:
      ok = OP_SUM;
      m = parts[0]->m;
      n = parts[0]->n;
      for (int32_t i = 0; i < k; ++i)
        if (parts[i]->m != m || parts[i]->n != n) return fail(CF_E_INVALID, "sum: shapes differ");
      break;
    case CF_SCALE:
      if (k != 1) return fail(CF_E_INVALID, "scale takes one part");
      ok = OP_SCALE;
      m = parts[0]->m;
      n = parts[0]->n;
      break;
    case CF_ADJOINT:
      if (k != 1) return fail(CF_E_INVALID, "adjoint takes one part");
      ok = OP_ADJOINT;
      m = parts[0]->n;
      n = parts[0]->m;
      break;
    case CF_KRON:
      if (k != 2) return fail(CF_E_INVALID, "kron takes two parts");
      for (int32_t i = 0; i < 2; ++i)
        if (parts[i]->kind != OP_DENSE || parts[i]->prec != CF_FP32)
          return fail(CF_E_INVALID, "kron: both parts must be dense FP32 leaves");
      ok = OP_KRON;
      m = parts[0]->m * parts[1]->m;
      n = parts[0]->n * parts[1]->n;
      break;
    default:
      return fail(CF_E_INVALID, "operator_compose: unknown kind");
  }
  cf_op* op = new_op(ctx, ok, m, n);
  op->alpha = alpha;
  for (int32_t i = 0; i < k; ++i) {
    op_retain(parts[i]);
    op->parts.push_back(parts[i]);
  }
  *out = op;
  return CF_OK;
}

cf_err cf_op_kron(cf_ctx* ctx, cf_op* A, cf_op* B, cf_op** out) {
  if (!A || !B) return fail(CF_E_INVALID, "cf_op_kron: NULL part");
  cf_op* parts[2] = {A, B};
  return operator_compose(ctx, CF_KRON, parts, 2, 1.0, out);
}

void cf_op_destroy(cf_op* op) {
  if (!op) return;
  if (op->refs.fetch_sub(1) == 1) op_free(op);
}

cf_err cf_op_shape(const cf_op* op, int64_t* m, int64_t* n) {
  if (!op) return fail(CF_E_INVALID, "cf_op_shape: NULL operator");
  if (m) *m = op->m;
  if (n) *n = op->n;
  return CF_OK;
}

cf_err cf_op_apply(cf_op* op, int32_t adjoint, const float* x, float* y) {
  if (!op || !x || !y) return fail(CF_E_INVALID, "cf_op_apply: bad arguments");
  cf_ctx* ctx = op->ctx;
  DevGuard g(ctx->device);
  const bool tr = adjoint != 0;
  const int64_t din = tr ? op->m : op->n, dout = tr ? op->n : op->m;
  size_t wsf = op_ws_floats(op, tr);
  float *dx = nullptr, *dy = nullptr, *ws = nullptr;
  size_t dummy = 0;
  auto run = [&]() -> cf_err {
    CF_TRY(dev_alloc(&dx, (size_t)din, &dummy));
    CF_TRY(dev_alloc(&dy, (size_t)dout, &dummy));
    CF_TRY(dev_alloc(&ws, wsf, &dummy));
    CF_TRY(copy_any(dx, x, din * sizeof(float), ctx->stream));
    op_apply(op, tr, 1.f, dx, dy, false, ws, ctx->stream);
    CF_CUDA(cudaGetLastError());
    CF_TRY(copy_any(y, dy, dout * sizeof(float), ctx->stream));
    CF_CUDA(cudaStreamSynchronize(ctx->stream));
    return CF_OK;
  };
  cf_err r = run();
  cudaFree(dx);
  cudaFree(dy);
  cudaFree(ws);
  return r;
}

cf_err cf_op_workspace_bytes(const cf_op* op, int32_t adjoint, size_t* bytes) {
  if (!op || !bytes) return fail(CF_E_INVALID, "cf_op_workspace_bytes: bad arguments");
  *bytes = op_ws_floats(op, adjoint != 0) * sizeof(float);
  return CF_OK;
}

cf_err cf_op_apply_async(cf_op* op, int32_t adjoint, float alpha, const float* x, float* y,
                         int32_t accumulate, void* workspace, void* stream) {
  if (!op || !x || !y) return fail(CF_E_INVALID, "cf_op_apply_async: bad arguments");
  const bool tr = adjoint != 0;
  if (op_ws_floats(op, tr) > 0 && !workspace)
    return fail(CF_E_INVALID, "cf_op_apply_async: workspace required");
  if (!is_device_ptr(x) || !is_device_ptr(y) || (workspace && !is_device_ptr(workspace)))
    return fail(CF_E_INVALID, "cf_op_apply_async: x, y and workspace must be device memory");
  DevGuard g(op->device);
  cudaStream_t s = stream ? (cudaStream_t)stream : op->ctx->stream;
  op_apply(op, tr, alpha, x, y, accumulate != 0, (float*)workspace, s);
  CF_CUDA(cudaGetLastError());
  return CF_OK;
}

cf_err cf_op_dense_stored(const cf_op* op, void* codes, float* row_scale) {
  if (!op || op->kind != OP_DENSE || !codes) return fail(CF_E_INVALID, "cf_op_dense_stored: not a dense leaf");
  DevGuard g(op->device);
  const size_t esz = op->prec == CF_FP32 ? 4 : (op->prec == CF_BF16 ? 2 : 1);
  // strip the row padding
  CF_CUDA(cudaMemcpy2D(codes, op->n * esz, op->a, op->lda * esz, op->n * esz, op->m, cudaMemcpyDefault));
  if (op->prec == CF_FP8_E4M3 && row_scale)
    CF_CUDA(cudaMemcpy(row_scale, op->row_scale, op->m * sizeof(float), cudaMemcpyDefault));
  return CF_OK;
}

}  // extern "C"
