// The SCS iteration (Section 5.2, following the published SCS method the
// paper cites) on one GPU.
//
// One ADMM iteration on the homogeneous self-dual embedding, u = (x, y, tau),
// v = (r, s, kappa), relaxation alpha:
//   w        = u + v
//   z_x      : CG on (I + A^T A) z_x = w_x - A^T w_y, warm-started (Section 4.2)
//   z_y      = w_y + A z_x
//   u~_tau   = (w_tau + c^T z_x + b^T z_y) / (1 + h^T g),  u~_xy = z - u~_tau g
//   u_hat    = alpha u~ + (1 - alpha) u
//   u+       = Pi_C(u_hat - v),   v+ = v - u_hat + u+      (C = R^n x K* x R_+)
// with g = M^{-1} h computed once by CG at setup.  The r block of v is zero
// at every iterate (x is free) and is not stored.
//
// The whole solve is one CUDA graph: a device-side WHILE node runs ADMM
// iterations, a nested WHILE node runs CG steps with the stopping test
// evaluated on the device, and an IF node runs the residual check every
// check_interval iterations; the host sees the GPU once per solve.  Every loop
// is bounded by a counter that a single thread advances (max_iters ADMM
// iterations, cg cap CG steps), independent of the reductions.
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <utility>

#include "devutil.cuh"
#include "solver.cuh"

namespace cf {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr int kSocChunk = 2048;        // rows of a second-order cone per CTA
constexpr int kRefreshInterval = 50;   // ADMM iterations between exact G z_x, A z_x

// ------------------------------------------------------------ reductions
// Sum NV doubles over the block; thread 0 receives the totals.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double t = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    v[j] = t;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[j][wid] = v[j];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = lane < nw ? sh[j][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      v[j] = t;
    }
  }
}

// Grid-wide deterministic sum: every block stores its partials; the last
// block to finish (atomic ticket) adds them in block order.  Returns true in
// the last block, where thread 0 holds the totals.  No block waits on another.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double* part, unsigned int* counter) {
  block_sum<NV>(v);
  __shared__ int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[blockIdx.x * NV + j] = v[j];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double t[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) t[j] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int j = 0; j < NV; ++j) t[j] += __ldcg(part + b * NV + j);
  block_sum<NV>(t);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = t[j];
    *counter = 0u;
  }
  return true;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Vector kernels walk float4 groups (the solver's vectors start on 256-byte
// boundaries of their arena) and then the scalar tail, so that a thread's
// loads for four elements go out as one 16-byte access.
#define VEC4_LOOP(v, n4) \
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < (n4); v += (int64_t)gridDim.x * blockDim.x)
#define TAIL_LOOP(i, n)                                                                  \
  for (int64_t i = ((n) & ~(int64_t)3) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; \
       i < (n); i += (int64_t)gridDim.x * blockDim.x)

// The same walk in batches of U consecutive strides: the loads of U groups
// (load(v) returns them) go out before the first is used (use(v, data)), so
// a thread has U groups in flight.  The groups are used in the order of the
// plain walk, so per-thread sums come out bit for bit the same.  The grids of
// the kernels that end in a grid-wide sum hold only 16 warps per SM (their
// per-CTA ticket costs more than extra elements per thread do); this is
// where their memory-level parallelism comes from.
constexpr int kVecBatch = 4;

template <int U, class Load, class Use>
__device__ __forceinline__ void vec4_batched(int64_t n4, Load&& load, Use&& use) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v0 < n4; v0 += U * stride) {
    decltype(load(v0)) d[U] = {};  // value-initialised: the unused slots are never read uninitialised
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v0 + u * stride < n4) d[u] = load(v0 + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v0 + u * stride < n4) use(v0 + u * stride, d[u]);
  }
}

__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
// 16-byte load through L2 only (no L1 allocation): for data a still-running
// predecessor wrote, read after pdl_wait.
__device__ __forceinline__ float4 ld4cg(const float* p, int64_t v) {
  return __ldcg(reinterpret_cast<const float4*>(p) + v);
}

// Programmatic dependent launch.  k_cg_update (after k_cg_dot) and k_cg_p
// (after k_cg_update) are launched with programmatic stream serialisation:
// such a dependent may start while its predecessor still runs, issues the
// loads of data the
// predecessor does not write, then waits (pdl_wait: until the predecessor
// has completed and its writes are visible) before it reads anything the
// predecessor writes or writes anything itself.  A predecessor lets its
// dependent launch (pdl_release) only once it is past its own wait, so every
// kernel before the predecessor is complete when the dependent starts.  The
// dependent's first loads then overlap the predecessor's tail (the last
// CTA's grid-wide sum), when most SMs are idle.  Launched plainly, the wait
// returns at once and the release does nothing.  A dependent reads no
// field of the control block before its wait (a line loaded early would
// hold the predecessor's scalars stale in L1: k_cg_p once read an old beta
// that way), and it reads what the predecessor wrote through L2 (__ldcg).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// vec4_batched with a hook run once per thread after its first batch of
// loads is issued (or at the end, for a thread without groups): the place
// for pdl_wait and the scalars the predecessor wrote.
template <int U, class Load, class Hook, class Use>
__device__ __forceinline__ void vec4_batched_first(int64_t n4, Load&& load, Hook&& hook, Use&& use) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool hooked = false;
  for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v0 < n4; v0 += U * stride) {
    decltype(load(v0)) d[U] = {};  // value-initialised: the unused slots are never read uninitialised
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v0 + u * stride < n4) d[u] = load(v0 + u * stride);
    if (!hooked) {
      hook();
      hooked = true;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (v0 + u * stride < n4) use(v0 + u * stride, d[u]);
  }
  if (!hooked) hook();
}

// ------------------------------------------------------------ problem data
// b, c (float64, already on the device) -> float32 copies, per-CTA float64
// sums of b_i^2 and c_i^2 (summed on the host in CTA order), and a flag set
// when an entry is not finite.
constexpr int kPrepGrid = 296;
__global__ void k_prep_data(int64_t m, int64_t n, const double* __restrict__ bd, const double* __restrict__ cd,
                            float* __restrict__ bf, float* __restrict__ cf, double* __restrict__ part,
                            int* __restrict__ bad) {
  double v[2] = {0.0, 0.0};
  int nf = 0;
  GRID_STRIDE(i, m) {
    const double x = bd[i];
    nf |= !isfinite(x);
    v[0] = fma(x, x, v[0]);
    bf[i] = (float)x;
  }
  GRID_STRIDE(i, n) {
    const double x = cd[i];
    nf |= !isfinite(x);
    v[1] = fma(x, x, v[1]);
    cf[i] = (float)x;
  }
  if (nf) atomicOr(bad, 1);
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = v[0];
    part[2 * blockIdx.x + 1] = v[1];
  }
}

// ------------------------------------------------------------ iteration start
__global__ void k_init(Ctl* c, int64_t n, int64_t m, float* ux, float* uy, float* vs, float* zx,
                       float* gz, float* az, const double* warm) {
  const bool w = c->st.warm != 0;
  const int64_t N = n + m + 1;
  GRID_STRIDE(i, n) {
    ux[i] = w ? (float)warm[i] : 0.f;
    zx[i] = 0.f;
    gz[i] = 0.f;
  }
  GRID_STRIDE(i, m) {
    uy[i] = w ? (float)warm[n + i] : 0.f;
    vs[i] = w ? (float)warm[N + n + i] : 0.f;
    az[i] = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->tau = w ? warm[n + m] : 1.0;
    c->kappa = w ? warm[N + n + m] : 1.0;
    c->k = 0;
    c->cg_total = 0;
    c->checks = 0;
    c->refreshes = 0;
    c->status = CF_MAX_ITERS;
    c->stop = 0;
    c->lam = 1.0;
    c->pri = c->dual = c->gap = INFINITY;
    c->cx = c->by = 0.0;
  }
}

// ---- folded diagonal row blocks
// Block of row r, or -1.
__device__ __forceinline__ int fold_row(const Fold& f, int64_t r) {
  for (int b = 0; b < f.nb; ++b)
    if (r >= f.r0[b] && r < f.r0[b] + f.len[b]) return b;
  return -1;
}
// The helpers below walk the blocks with static indices (unrolled over
// kMaxFold), so the Fold parameter is read in place, never copied to the
// stack.
// Column of the folded block entry in row r (c0 + r - r0), or -1.
__device__ __forceinline__ int64_t fold_row_col(const Fold& f, int64_t r) {
  int64_t c = -1;
#pragma unroll
  for (int b = 0; b < kMaxFold; ++b)
    if (b < f.nb && c < 0 && r >= f.r0[b] && r < f.r0[b] + f.len[b]) c = f.c0[b] + (r - f.r0[b]);
  return c;
}
// Whether any folded block touches columns (or rows) [lo, lo + 4).
__device__ __forceinline__ bool fold_cols_touch(const Fold& f, int64_t lo) {
  bool t = false;
#pragma unroll
  for (int b = 0; b < kMaxFold; ++b) t |= b < f.nb && lo < f.c0[b] + f.len[b] && f.c0[b] < lo + 4;
  return t;
}
__device__ __forceinline__ bool fold_rows_touch(const Fold& f, int64_t lo) {
  bool t = false;
#pragma unroll
  for (int b = 0; b < kMaxFold; ++b) t |= b < f.nb && lo < f.r0[b] + f.len[b] && f.r0[b] < lo + 4;
  return t;
}
__device__ __forceinline__ bool fold_rows_cover(const Fold& f, int64_t lo) {
  bool t = false;
#pragma unroll
  for (int b = 0; b < kMaxFold; ++b) t |= b < f.nb && lo >= f.r0[b] && lo + 4 <= f.r0[b] + f.len[b];
  return t;
}
// Whether one block's rows (COLS: its columns) hold all of [lo, lo + 4),
// with its column-minus-row offset a multiple of 4 (16-byte loads on both
// sides), and no other block touching them; the offset c0 - r0 in *delta.
template <bool COLS>
__device__ __forceinline__ bool fold_vec_delta(const Fold& f, int64_t lo, int64_t* delta) {
  int hits = 0;
  bool ok = true;
#pragma unroll
  for (int b = 0; b < kMaxFold; ++b) {
    if (b >= f.nb) break;
    const int64_t a = COLS ? f.c0[b] : f.r0[b];
    if (lo < a + f.len[b] && a < lo + 4) {
      ++hits;
      ok = ok && lo >= a && lo + 4 <= a + f.len[b] && ((f.c0[b] - f.r0[b]) & 3) == 0;
      *delta = f.c0[b] - f.r0[b];
    }
  }
  return hits == 1 && ok;
}

// Diagonal of each folded block's rows, s_r = D_r alpha d_j E_(c0 + j)
// (j = r - r0; D, E the equilibration, 1 without), and per column the sum of
// s^2 over the blocks covering it.
struct FoldSrc {
  float alpha[kMaxFold];
  const float* d[kMaxFold];
};
__global__ void k_fold_prep(Fold f, FoldSrc src, int64_t m, int64_t n, const float* __restrict__ D,
                            const float* __restrict__ E, float* __restrict__ s, float* __restrict__ gd) {
  auto val = [&](int b, int64_t j) {
    const int64_t r = f.r0[b] + j, c = f.c0[b] + j;
    float v = src.alpha[b] * (src.d[b] ? src.d[b][j] : 1.f);
    if (D) v *= D[r];
    if (E) v *= E[c];
    return v;
  };
  GRID_STRIDE(r, m) {
    const int b = fold_row(f, r);
    s[r] = b >= 0 ? val(b, r - f.r0[b]) : 0.f;
  }
  GRID_STRIDE(c, n) {
    float g = 0.f;
    for (int b = 0; b < f.nb; ++b)
      if (c >= f.c0[b] && c < f.c0[b] + f.len[b]) {
        const float v = val(b, c - f.c0[b]);
        g = fmaf(v, v, g);
      }
    gd[c] = g;
  }
}

// w_y = u_y + v_s, rhs = u_x (then rhs -= A^T w_y by the operator walk); the
// folded blocks' part of A^T w_y is subtracted here: rhs_c -= s_r w_y,r for
// the rows r of the blocks covering column c.
__global__ void k_rhs(Ctl* c, int64_t n, int64_t m, const float* __restrict__ ux,
                      const float* __restrict__ uy, const float* __restrict__ vs,
                      float* __restrict__ wy, float* __restrict__ rhs, Fold f) {
  VEC4_LOOP(v, m >> 2) {
    const float4 a = ld4(uy, v), b = ld4(vs, v);
    st4(wy, v, make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w));
  }
  TAIL_LOOP(i, m) wy[i] = uy[i] + vs[i];
  auto folded = [&](int64_t col, float x) {
#pragma unroll
    for (int b = 0; b < kMaxFold; ++b)
      if (b < f.nb && col >= f.c0[b] && col < f.c0[b] + f.len[b]) {
        const int64_t r = f.r0[b] + (col - f.c0[b]);
        x = fmaf(-f.s[r], uy[r] + vs[r], x);
      }
    return x;
  };
  VEC4_LOOP(v, n >> 2) {
    float4 x = ld4(ux, v);
    if (f.nb && fold_cols_touch(f, 4 * v)) {
      int64_t delta = 0;
      if (fold_vec_delta<true>(f, 4 * v, &delta)) {
        const int64_t rv = v - delta / 4;
        const float4 s4 = ld4(f.s, rv), a4 = ld4(uy, rv), b4 = ld4(vs, rv);
#pragma unroll
        for (int k = 0; k < 4; ++k) el(x, k) = fmaf(-elc(s4, k), elc(a4, k) + elc(b4, k), el(x, k));
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) el(x, k) = folded(4 * v + k, el(x, k));
      }
    }
    st4(rhs, v, x);
  }
  TAIL_LOOP(i, n) rhs[i] = f.nb ? folded(i, ux[i]) : ux[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) c->w_tau = c->tau + c->kappa;
}

// ------------------------------------------------------------ CG (Section 4.2)
// CG on G z = rhs with G = lam I + A^T A.  gz holds G z for the current z and
// az holds A z: both are carried along by the CG updates (gz += alpha G p,
// az += alpha A p), so starting CG at the warm-start z needs no operator pass,
// and neither does z_y = w_y + A z_x afterwards.  They are recomputed exactly
// every kRefreshInterval ADMM iterations.
//
// Every kernel that decides a loop stores the decision in the control block
// and, inside a graph, also sets the conditional node's value.

// r = rhs - G z; p = r; stopping threshold.  fresh != 0: gz holds A^T A z
// just computed, and G z = gz + lam z is formed (and kept) here.
//
// gd (folded diagonal blocks, may be null): the Gram's diagonal part beyond
// lam; then q is started at (lam + gd) p, onto which the next Gram pass adds
// the remaining blocks' A^T A p.
__global__ void k_cg_init(Ctl* c, int64_t n, const float* __restrict__ rhs,
                          const float* __restrict__ z, float* __restrict__ gz,
                          float* __restrict__ r, float* __restrict__ p, double* part, int mode,
                          int fresh, cudaGraphConditionalHandle h, int in_graph,
                          const float* __restrict__ gd, float* __restrict__ q) {
  const float lam = (float)c->lam;
  Acc2 a0, a1;
  struct In { float4 g, rh, dg, zz; };
  vec4_batched<kVecBatch>(
      n >> 2,
      [&](int64_t v) {
        In d;
        d.g = ld4(gz, v);
        d.rh = ld4(rhs, v);
        d.dg = gd ? ld4(gd, v) : zero4();
        d.zz = fresh ? ld4(z, v) : zero4();
        return d;
      },
      [&](int64_t v, In& d) {
        float4 g = d.g;
        const float4 rh = d.rh, dg = d.dg;
        if (fresh) {
#pragma unroll
          for (int k = 0; k < 4; ++k) el(g, k) = fmaf(lam + elc(dg, k), elc(d.zz, k), el(g, k));
          st4(gz, v, g);
        }
        float4 rr, qq;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          el(rr, k) = elc(rh, k) - elc(g, k);
          el(qq, k) = (lam + elc(dg, k)) * el(rr, k);
          a0.add_prod(elc(rr, k), elc(rr, k));
          a1.add_prod(elc(rh, k), elc(rh, k));
        }
        st4(r, v, rr);
        st4(p, v, rr);
        if (gd) st4(q, v, qq);
      });
  TAIL_LOOP(i, n) {
    float g = gz[i];
    const float dg = gd ? gd[i] : 0.f;
    if (fresh) {
      g = fmaf(lam + dg, z[i], g);
      gz[i] = g;
    }
    const float rh = rhs[i];
    float ri = rh - g;
    r[i] = ri;
    p[i] = ri;
    if (gd) q[i] = (lam + dg) * ri;
    a0.add_prod(ri, ri);
    a1.add_prod(rh, rh);
  }
  double v[2] = {a0.value(), a1.value()};
  if (blockIdx.x == 0 && threadIdx.x == 0) c->cg_guard = 0;
  if (grid_sum<2>(v, part, &c->red_count) && threadIdx.x == 0) {
    const double rr = v[0], nrhs = sqrt(v[1]);
    double tol;
    int cap, fixed;
    if (mode == CG_SETUP) {
      tol = c->st.setup_tol * nrhs;
      cap = c->st.setup_cg_max;
      fixed = 0;
    } else {
      tol = c->st.cg_tol_rel * nrhs * (double)powf((float)c->k + 1.0f, -(float)c->st.cg_tol_exp);
      tol = fmax(tol, c->st.cg_tol_min);
      cap = c->st.cg_max;
      fixed = c->st.cg_fixed;
    }
    c->rr = rr;
    c->tol2 = tol * tol;
    c->cg_it = 0;
    const int cont = fixed > 0 ? 1 : ((rr > c->tol2 && cap > 0) ? 1 : 0);
    c->cg_cont = cont;
    c->cg_go = cont;
    if (in_graph) cudaGraphSetConditional(h, (unsigned)cont);
  }
}

// q += lam p (q held A^T A p); alpha = rr / p^T q.  folded: q already holds
// (lam + gd) p + A^T A p over the remaining blocks, and is only read.
__global__ void k_cg_dot(Ctl* c, int64_t n, const float* __restrict__ p, float* __restrict__ q,
                         double* part, int folded) {
  pdl_release();  // k_cg_update loads nothing this kernel writes unless !folded (then it waits first)
  const float lam = (float)c->lam;
  Acc2 a0;
  struct In { float4 pp, qq; };
  vec4_batched<kVecBatch>(
      n >> 2, [&](int64_t w) { return In{ld4(p, w), ld4(q, w)}; },
      [&](int64_t w, In& d) {
        float4 qq = d.qq;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (!folded) el(qq, k) = el(qq, k) + lam * elc(d.pp, k);
          a0.add_prod(elc(d.pp, k), elc(qq, k));
        }
        if (!folded) st4(q, w, qq);
      });
  TAIL_LOOP(i, n) {
    const float pi = p[i];
    float qi = folded ? q[i] : q[i] + lam * pi;
    if (!folded) q[i] = qi;
    a0.add_prod(pi, qi);
  }
  double v[1] = {a0.value()};
  if (grid_sum<1>(v, part, &c->red_count) && threadIdx.x == 0) {
    const double pq = v[0];
    c->alpha_cg = pq > 0.0 ? c->rr / pq : 0.0;
  }
}

// z += alpha p; r -= alpha q; gz += alpha q; az += alpha t (t = A p; az may
// be null); beta = ||r_new||^2 / ||r||^2; continue test
__global__ void k_cg_update(Ctl* c, int64_t n, int64_t m, float* __restrict__ z, float* __restrict__ r,
                            const float* __restrict__ p, const float* __restrict__ q,
                            float* __restrict__ gz, float* __restrict__ az,
                            const float* __restrict__ t, double* part, int mode, Fold f, int prefetch) {
  // prefetch: the predecessor (k_cg_dot, folded form) writes none of q, p,
  // z, gz, r, so their first loads go out before the wait
  float a = 0.f;
  bool waited = false;
  auto wait = [&] {
    if (waited) return;
    pdl_wait();
    a = (float)__ldcg(&c->alpha_cg);
    waited = true;
    pdl_release();
  };
  if (!prefetch) wait();
  Acc2 a0;
  struct In { float4 qq, pp, zz, gg, rr; };
  vec4_batched_first<kVecBatch>(
      n >> 2, [&](int64_t v) { return In{ld4cg(q, v), ld4(p, v), ld4(z, v), ld4(gz, v), ld4(r, v)}; }, wait,
      [&](int64_t v, In& d) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          el(d.zz, k) = fmaf(a, elc(d.pp, k), el(d.zz, k));
          el(d.gg, k) = fmaf(a, elc(d.qq, k), el(d.gg, k));
          el(d.rr, k) = fmaf(-a, elc(d.qq, k), el(d.rr, k));
          a0.add_prod(elc(d.rr, k), elc(d.rr, k));
        }
        st4(z, v, d.zz);
        st4(gz, v, d.gg);
        st4(r, v, d.rr);
      });
  TAIL_LOOP(i, n) {
    const float qi = q[i];
    z[i] = fmaf(a, p[i], z[i]);
    gz[i] = fmaf(a, qi, gz[i]);
    float ri = fmaf(-a, qi, r[i]);
    r[i] = ri;
    a0.add_prod(ri, ri);
  }
  double v[1] = {a0.value()};
  if (az) {
    // rows of folded blocks: A z there is s z, formed where it is used
    struct InA { float4 tt, aa; bool skip; };
    vec4_batched<kVecBatch>(
        m >> 2,
        [&](int64_t w) {
          InA d;
          d.skip = f.nb && fold_rows_cover(f, 4 * w);
          if (!d.skip) {
            d.tt = ld4(t, w);
            d.aa = ld4(az, w);
          }
          return d;
        },
        [&](int64_t w, InA& d) {
          if (d.skip) return;
#pragma unroll
          for (int k = 0; k < 4; ++k) el(d.aa, k) = fmaf(a, elc(d.tt, k), el(d.aa, k));
          st4(az, w, d.aa);
        });
    TAIL_LOOP(i, m) az[i] = fmaf(a, t[i], az[i]);
  }
  if (grid_sum<1>(v, part, &c->red_count) && threadIdx.x == 0) {
    const double rr_new = v[0];
    c->beta_cg = c->rr > 0.0 ? rr_new / c->rr : 0.0;
    c->rr = rr_new;
    c->cg_it += 1;
    int cap, fixed;
    if (mode == CG_SETUP) {
      c->setup_iters += 1;
      cap = c->st.setup_cg_max;
      fixed = 0;
    } else {
      c->cg_total += 1;
      cap = c->st.cg_max;
      fixed = c->st.cg_fixed;
    }
    c->cg_cont = fixed > 0 ? (c->cg_it < fixed) : (rr_new > c->tol2 && c->cg_it < cap);
  }
}

// p = r + beta p; decide whether the CG loop runs again.  The guard counter
// is advanced here by one thread, so the loop ends after at most `cap` steps
// whatever the reductions produced.
// gd (folded blocks): also start the next Gram pass's q at (lam + gd) p.
__global__ void k_cg_p(Ctl* c, int64_t n, const float* __restrict__ r, float* __restrict__ p,
                       int mode, cudaGraphConditionalHandle h, int in_graph, const float* __restrict__ gd,
                       float* __restrict__ q) {
  // p and gd are not written by the predecessor (k_cg_update): their first
  // loads go out before the wait; r and beta come after it
  float lam = 0.f, b = 0.f;
  struct In { float4 pp, dg; };
  vec4_batched_first<1>(
      n >> 2, [&](int64_t v) { return In{ld4(p, v), gd ? ld4(gd, v) : zero4()}; },
      [&] {
        pdl_wait();
        lam = (float)c->lam;
        b = (float)__ldcg(&c->beta_cg);
      },
      [&](int64_t v, In& d) {
        const float4 rr = ld4cg(r, v);
        float4 pp = d.pp;
#pragma unroll
        for (int k = 0; k < 4; ++k) el(pp, k) = fmaf(b, el(pp, k), elc(rr, k));
        st4(p, v, pp);
        if (gd) {
          const float4 dg = d.dg;
          st4(q, v, make_float4((lam + dg.x) * pp.x, (lam + dg.y) * pp.y, (lam + dg.z) * pp.z, (lam + dg.w) * pp.w));
        }
      });
  TAIL_LOOP(i, n) {
    const float pi = fmaf(b, p[i], __ldcg(r + i));
    p[i] = pi;
    if (gd) q[i] = (lam + gd[i]) * pi;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int g = ++c->cg_guard;
    int cap = mode == CG_SETUP ? c->st.setup_cg_max : (c->st.cg_fixed > 0 ? c->st.cg_fixed : c->st.cg_max);
    const int cont = (__ldcg(&c->cg_cont) && g < cap) ? 1 : 0;
    c->cg_go = cont;
    if (in_graph) cudaGraphSetConditional(h, (unsigned)cont);
  }
}

// gz += lam z (after gz = A^T A z was recomputed exactly)
__global__ void k_gz_shift(const Ctl* c, int64_t n, const float* __restrict__ z, float* __restrict__ gz) {
  const float lam = (float)c->lam;
  GRID_STRIDE(i, n) gz[i] = fmaf(lam, z[i], gz[i]);
}

// ------------------------------------------------------------ subspace step
// z_y = w_y + A z_x (A z_x carried in az); u~_tau = (w_tau + c^T z_x + b^T z_y) / (1 + h^T g)
// (rows of folded blocks: A z_x there is s z_x[c0 + j])
__global__ void k_utau(Ctl* c, int64_t n, int64_t m, const float* __restrict__ zx,
                       const float* __restrict__ az, float* __restrict__ zy, const float* __restrict__ wy,
                       const float* __restrict__ bf, const float* __restrict__ cf, double* part, Fold f) {
  Acc2 a0;
  auto azr = [&](int64_t r, float carried) {
    const int64_t col = fold_row_col(f, r);
    return col < 0 ? carried : f.s[r] * zx[col];
  };
  struct In { float4 ww, bb, aa; };
  vec4_batched<kVecBatch>(
      m >> 2,
      [&](int64_t w) {
        In d;
        d.ww = ld4(wy, w);
        d.bb = ld4(bf, w);
        const bool touch = f.nb && fold_rows_touch(f, 4 * w);
        int64_t delta = 0;
        if (touch && fold_vec_delta<false>(f, 4 * w, &delta)) {  // four rows of one block: s z_x[c0 + j]
          const float4 s4 = ld4(f.s, w), z4 = ld4(zx, w + delta / 4);
          d.aa = make_float4(s4.x * z4.x, s4.y * z4.y, s4.z * z4.z, s4.w * z4.w);
        } else {
          d.aa = ld4(az, w);
          if (touch) {
#pragma unroll
            for (int k = 0; k < 4; ++k) el(d.aa, k) = azr(4 * w + k, el(d.aa, k));
          }
        }
        return d;
      },
      [&](int64_t w, In& d) {
        float4 zz;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          el(zz, k) = elc(d.aa, k) + elc(d.ww, k);
          a0.add_prod(elc(d.bb, k), elc(zz, k));
        }
        st4(zy, w, zz);
      });
  TAIL_LOOP(i, m) {
    float zi = (f.nb ? azr(i, az[i]) : az[i]) + wy[i];
    zy[i] = zi;
    a0.add_prod(bf[i], zi);
  }
  struct InX { float4 cc, xx; };
  vec4_batched<kVecBatch>(
      n >> 2, [&](int64_t w) { return InX{ld4(cf, w), ld4(zx, w)}; },
      [&](int64_t, InX& d) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a0.add_prod(elc(d.cc, k), elc(d.xx, k));
      });
  TAIL_LOOP(i, n) a0.add_prod(cf[i], zx[i]);
  double v[1] = {a0.value()};
  if (grid_sum<1>(v, part, &c->red_count) && threadIdx.x == 0)
    c->ut_tau = (c->w_tau + v[0]) / (1.0 + c->hg);
}

// Per-chunk squared norm of the tail of each second-order cone block of the
// pre-projection point; the chunk holding a block's head row stores p_head.
__global__ void k_soc_norm(const Ctl* c, const int32_t* __restrict__ chunk_seg,
                           const int64_t* __restrict__ chunk_r0, const int64_t* __restrict__ chunk_r1,
                           const int64_t* __restrict__ seg_head, const int32_t* __restrict__ seg_c0,
                           const int32_t* __restrict__ seg_nc, const float* __restrict__ zy,
                           const float* __restrict__ gy, const float* __restrict__ uy,
                           const float* __restrict__ vs, double* __restrict__ chunk_n2,
                           double* __restrict__ seg_p0, double* __restrict__ seg_nrm,
                           unsigned int* __restrict__ seg_cnt) {
  const int64_t ch = blockIdx.x;
  const int32_t sg = chunk_seg[ch];
  const int64_t head = seg_head[sg];
  const int64_t r0 = chunk_r0[ch], r1 = chunk_r1[ch];
  const float a = (float)c->st.alpha, a1 = (float)(1.0 - c->st.alpha), ut = (float)c->ut_tau;
  Acc2 a0;
  auto row = [&](int64_t i, float pi) {
    if (i == head)
      seg_p0[sg] = (double)pi;
    else
      a0.add_prod(pi, pi);
  };
  // 16-byte loads over the chunk's 4-aligned interior, single rows at its edges
  const int64_t q0 = (r0 + 3) & ~(int64_t)3, q1 = r1 & ~(int64_t)3;
  const int64_t e0 = q0 < q1 ? q0 : r1;
  for (int64_t i = r0 + threadIdx.x; i < e0; i += blockDim.x) row(i, y_pre(a, a1, ut, zy[i], gy[i], uy[i], vs[i]));
  if (q0 < q1) {
#pragma unroll 2
    for (int64_t v = (q0 >> 2) + threadIdx.x; v < (q1 >> 2); v += blockDim.x) {
      const float4 z4 = ld4(zy, v), g4 = ld4(gy, v), u4 = ld4(uy, v), s4 = ld4(vs, v);
#pragma unroll
      for (int k = 0; k < 4; ++k) row(4 * v + k, y_pre(a, a1, ut, elc(z4, k), elc(g4, k), elc(u4, k), elc(s4, k)));
    }
    for (int64_t i = q1 + threadIdx.x; i < r1; i += blockDim.x) row(i, y_pre(a, a1, ut, zy[i], gy[i], uy[i], vs[i]));
  }
  double v[1] = {a0.value()};
  block_sum<1>(v);
  // the last chunk of the segment to finish forms the segment's norm once,
  // adding the chunk partials in chunk order
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    chunk_n2[ch] = v[0];
    __threadfence();
    s_last = atomicAdd(&seg_cnt[sg], 1u) == (unsigned)seg_nc[sg] - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int32_t c0 = seg_c0[sg], nc = seg_nc[sg];
  double t[1] = {0.0};
  for (int32_t k = threadIdx.x; k < nc; k += blockDim.x) t[0] += __ldcg(chunk_n2 + c0 + k);
  block_sum<1>(t);
  if (threadIdx.x == 0) {
    seg_nrm[sg] = sqrt(t[0]);
    seg_cnt[sg] = 0u;
  }
}

// Projection and dual update.  Blocks [0, nlin) cover x (free) and the zero
// and nonnegative rows of y elementwise; blocks [nlin, nlin + nchunk) cover
// the second-order cone chunks.  Thread 0 of block 0 updates tau, kappa and
// the iteration counter and decides whether this iteration ends with a
// residual check.
__global__ void k_apply(Ctl* c, int64_t n, int64_t m, int64_t z, int64_t l, int nlin,
                        float* __restrict__ ux, float* __restrict__ uy, float* __restrict__ vs,
                        const float* __restrict__ zx, const float* __restrict__ zy,
                        const float* __restrict__ gx, const float* __restrict__ gy,
                        const int32_t* __restrict__ chunk_seg, const int64_t* __restrict__ chunk_r0,
                        const int64_t* __restrict__ chunk_r1, const int64_t* __restrict__ seg_head,
                        const double* __restrict__ seg_nrm, const double* __restrict__ seg_p0,
                        cudaGraphConditionalHandle h_check, cudaGraphConditionalHandle h_refresh,
                        cudaGraphConditionalHandle h_outer, int in_graph) {
  const double al = c->st.alpha;
  const float a = (float)al, a1 = (float)(1.0 - al), ut = (float)c->ut_tau;
  if ((int)blockIdx.x < nlin) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)nlin * blockDim.x;
    // x (free): u_x = alpha (z_x - u~_tau g_x) + (1 - alpha) u_x
    for (int64_t v = tid; v < (n >> 2); v += stride) {
      const float4 zz = ld4(zx, v), gg = ld4(gx, v);
      float4 uu = ld4(ux, v);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        el(uu, k) = __fadd_rn(__fmul_rn(a, __fsub_rn(elc(zz, k), __fmul_rn(ut, elc(gg, k)))),
                              __fmul_rn(a1, el(uu, k)));
      st4(ux, v, uu);
    }
    for (int64_t i = (n & ~(int64_t)3) + tid; i < n; i += stride)
      ux[i] = __fadd_rn(__fmul_rn(a, __fsub_rn(zx[i], __fmul_rn(ut, gx[i]))), __fmul_rn(a1, ux[i]));
    // zero rows (dual: free) and nonnegative rows of y
    const int64_t nl = z + l;
    for (int64_t v = tid; v < (nl >> 2); v += stride) {
      const float4 zz = ld4(zy, v), gg = ld4(gy, v);
      float4 uu = ld4(uy, v), ss = ld4(vs, v);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float pj = y_pre(a, a1, ut, elc(zz, k), elc(gg, k), el(uu, k), el(ss, k));
        const float uj = (4 * v + k) < z ? pj : fmaxf(pj, 0.f);
        el(uu, k) = uj;
        el(ss, k) = __fsub_rn(uj, pj);
      }
      st4(uy, v, uu);
      st4(vs, v, ss);
    }
    for (int64_t j = (nl & ~(int64_t)3) + tid; j < nl; j += stride) {
      float pj = y_pre(a, a1, ut, zy[j], gy[j], uy[j], vs[j]);
      float uj = j < z ? pj : fmaxf(pj, 0.f);
      uy[j] = uj;
      vs[j] = __fsub_rn(uj, pj);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const double uhat = al * c->ut_tau + (1.0 - al) * c->tau;
      const double pt = uhat - c->kappa;
      const double tn = pt > 0.0 ? pt : 0.0;
      c->tau = tn;
      c->kappa = tn - pt;
      const int k = c->k + 1;
      c->k = k;
      const int chk = (k % c->st.check_interval == 0) || (k >= c->st.max_iters);
      const int ref = (k % kRefreshInterval == 0) && (k < c->st.max_iters);
      c->do_check = chk;
      c->do_refresh = ref;
      c->refreshes += ref;
      // loop decision; a residual check run after this kernel may revise it
      if (!isfinite(tn) || !isfinite(c->kappa)) {
        c->status = CF_NUMERICAL;
        c->stop = 1;
      }
      const int go = (!c->stop && k < c->st.max_iters) ? 1 : 0;
      c->outer_go = go;
      if (in_graph) {
        cudaGraphSetConditional(h_check, (unsigned)chk);
        cudaGraphSetConditional(h_refresh, (unsigned)ref);
        cudaGraphSetConditional(h_outer, (unsigned)go);
      }
    }
    return;
  }
  // second-order cone chunk: its segment's norm and head value come from
  // k_soc_norm
  const int64_t ch = blockIdx.x - nlin;
  const int32_t sg = chunk_seg[ch];
  const int64_t head = seg_head[sg];
  const double nrm = seg_nrm[sg], p0 = seg_p0[sg];
  // 0: keep, 1: zero, 2: scale onto the boundary
  const int mode = nrm <= p0 ? 0 : (nrm <= -p0 ? 1 : 2);
  const double ah = 0.5 * (p0 + nrm);
  const float head_val = (float)ah;
  const float scl = mode == 2 ? (float)(ah / nrm) : 0.f;
  const int64_t r0 = chunk_r0[ch], r1 = chunk_r1[ch];
  auto proj = [&](int64_t i, float pi) {
    if (mode == 0) return pi;
    if (mode == 1) return 0.f;
    return (i == head) ? head_val : __fmul_rn(scl, pi);
  };
  auto row = [&](int64_t i) {
    const float pi = y_pre(a, a1, ut, zy[i], gy[i], uy[i], vs[i]);
    const float ui = proj(i, pi);
    uy[i] = ui;
    vs[i] = __fsub_rn(ui, pi);
  };
  // 16-byte accesses over the chunk's 4-aligned interior, single rows at its edges
  const int64_t q0 = (r0 + 3) & ~(int64_t)3, q1 = r1 & ~(int64_t)3;
  if (q0 >= q1) {
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) row(i);
    return;
  }
  for (int64_t i = r0 + threadIdx.x; i < q0; i += blockDim.x) row(i);
  for (int64_t i = q1 + threadIdx.x; i < r1; i += blockDim.x) row(i);
#pragma unroll 2
  for (int64_t v = (q0 >> 2) + threadIdx.x; v < (q1 >> 2); v += blockDim.x) {
    const float4 z4 = ld4(zy, v), g4 = ld4(gy, v);
    float4 u4 = ld4(uy, v), s4 = ld4(vs, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float pi = y_pre(a, a1, ut, elc(z4, k), elc(g4, k), elc(u4, k), elc(s4, k));
      const float ui = proj(4 * v + k, pi);
      el(u4, k) = ui;
      el(s4, k) = __fsub_rn(ui, pi);
    }
    st4(uy, v, u4);
    st4(vs, v, s4);
  }
}

// ------------------------------------------------------------ termination
// With cm = A u_x and cn = A^T u_y (A the solver's, possibly equilibrated,
// operator), weights w_i = 1/D_i on rows and 1/E_j on columns (1 without
// equilibration):
//   S0 = ||w (cm + v_s - b tau)||^2   S1 = ||w (cm + v_s)||^2   S2 = b^T u_y
//   S3 = ||w (cn + c tau)||^2         S4 = ||w cn||^2         S5 = c^T u_x
// The original problem's point is x = E u_x / (sigma tau), y = D u_y / (rho tau),
// s = v_s / (sigma D tau), so
//   pri = sqrt(S0)/(sigma tau)/(1+||b||), dual = sqrt(S3)/(rho tau)/(1+||c||),
//   c^T x = S5/(rho sigma tau), b^T y = S2/(rho sigma tau),
// and the certificates (invariant to the common factors) read
//   infeasible: -S2 > 0 and sigma sqrt(S4) <= eps_infeas (-S2),
//   unbounded:  -S5 > 0 and rho sqrt(S1) <= eps_infeas (-S5).
__global__ void k_resid(Ctl* c, int64_t n, int64_t m, const float* __restrict__ cm,
                        const float* __restrict__ cn, const float* __restrict__ ux,
                        const float* __restrict__ uy, const float* __restrict__ vs,
                        const float* __restrict__ bf, const float* __restrict__ cf,
                        const float* __restrict__ dinv, const float* __restrict__ einv, double* part,
                        cudaGraphConditionalHandle h_outer, int in_graph) {
  const double tau = c->tau;
  const float tf = (float)tau;
  Acc2 s0, s1, s2, s3, s4, s5;
  auto row_y = [&](float w, float cmi, float vsi, float bfi, float uyi) {
    const float e = cmi + vsi;
    const float d = w * fmaf(-bfi, tf, e);
    const float we = w * e;
    s0.add_prod(d, d);
    s1.add_prod(we, we);
    s2.add_prod(bfi, uyi);
  };
  auto row_x = [&](float w, float cni, float cfi, float uxi) {
    const float d = w * fmaf(cfi, tf, cni);
    const float wc = w * cni;
    s3.add_prod(d, d);
    s4.add_prod(wc, wc);
    s5.add_prod(cfi, uxi);
  };
  const float4 one4 = make_float4(1.f, 1.f, 1.f, 1.f);
  struct InY { float4 w, a, b, c4, u; };
  vec4_batched<kVecBatch>(
      m >> 2,
      [&](int64_t v) { return InY{dinv ? ld4(dinv, v) : one4, ld4(cm, v), ld4(vs, v), ld4(bf, v), ld4(uy, v)}; },
      [&](int64_t, InY& d) {
#pragma unroll
        for (int k = 0; k < 4; ++k) row_y(elc(d.w, k), elc(d.a, k), elc(d.b, k), elc(d.c4, k), elc(d.u, k));
      });
  TAIL_LOOP(i, m) row_y(dinv ? dinv[i] : 1.f, cm[i], vs[i], bf[i], uy[i]);
  struct InX { float4 w, a, c4, u; };
  vec4_batched<kVecBatch>(
      n >> 2, [&](int64_t v) { return InX{einv ? ld4(einv, v) : one4, ld4(cn, v), ld4(cf, v), ld4(ux, v)}; },
      [&](int64_t, InX& d) {
#pragma unroll
        for (int k = 0; k < 4; ++k) row_x(elc(d.w, k), elc(d.a, k), elc(d.c4, k), elc(d.u, k));
      });
  TAIL_LOOP(i, n) row_x(einv ? einv[i] : 1.f, cn[i], cf[i], ux[i]);
  double v[6] = {s0.value(), s1.value(), s2.value(), s3.value(), s4.value(), s5.value()};
  if (grid_sum<6>(v, part, &c->red_count) && threadIdx.x == 0) {
    const double sig = c->sigma, rho = c->rho;
    c->checks += 1;
    c->cx = v[5] / (rho * sig);
    c->by = v[2] / (rho * sig);
    bool bad = false;
    for (int j = 0; j < 6; ++j) bad |= !isfinite(v[j]);
    if (bad || !isfinite(tau) || !isfinite(c->kappa)) {
      c->status = CF_NUMERICAL;
      c->stop = 1;
    } else {
      if (tau > 0.0) {
        const double pri = sqrt(v[0]) / (sig * tau) / (1.0 + c->nb);
        const double dual = sqrt(v[3]) / (rho * tau) / (1.0 + c->nc);
        const double cx = c->cx / tau, by = c->by / tau;
        const double gap = fabs(cx + by) / (1.0 + fabs(cx) + fabs(by));
        c->pri = pri;
        c->dual = dual;
        c->gap = gap;
        if (pri <= c->st.eps && dual <= c->st.eps && gap <= c->st.eps) {
          c->status = CF_SOLVED;
          c->stop = 1;
        }
      }
      if (!c->stop) {
        if (-v[2] > 0.0 && sig * sqrt(v[4]) <= c->st.eps_inf * (-v[2])) {
          c->status = CF_INFEASIBLE;
          c->stop = 1;
        } else if (-v[5] > 0.0 && rho * sqrt(v[1]) <= c->st.eps_inf * (-v[5])) {
          c->status = CF_UNBOUNDED;
          c->stop = 1;
        }
      }
    }
    const int go = (!c->stop && c->k < c->st.max_iters) ? 1 : 0;
    c->outer_go = go;
    if (in_graph) cudaGraphSetConditional(h_outer, (unsigned)go);
  }
}

// ------------------------------------------------------------ setup kernels
__global__ void k_setup_init(Ctl* c, int64_t n, int64_t m, float* gx, float* gz, float* az, float* rhs,
                             const float* cf) {
  GRID_STRIDE(i, n) {
    gx[i] = 0.f;
    gz[i] = 0.f;
    rhs[i] = cf[i];
  }
  GRID_STRIDE(i, m) az[i] = 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->lam = 1.0;
    c->setup_iters = 0;
    c->k = 0;
  }
}

// g_y += b (g_y held A g_x); h^T g = c^T g_x + b^T g_y
__global__ void k_setup_fin(Ctl* c, int64_t n, int64_t m, const float* __restrict__ gx,
                            float* __restrict__ gy, const float* __restrict__ bf,
                            const float* __restrict__ cf, double* part) {
  Acc2 a0;
  GRID_STRIDE(i, m) {
    float gi = gy[i] + bf[i];
    gy[i] = gi;
    a0.add_prod(bf[i], gi);
  }
  GRID_STRIDE(i, n) a0.add_prod(cf[i], gx[i]);
  double v[1] = {a0.value()};
  if (grid_sum<1>(v, part, &c->red_count) && threadIdx.x == 0) c->hg = v[0];
}

// ------------------------------------------------------------ outputs
// The original problem's point (see k_resid): x = E u_x / sigma, y = D u_y / rho,
// s = v_s / (sigma D), divided by tau, or normalised as a certificate
// (b^T y = -1, or c^T x = -1 with s scaled alike).  c->cx, c->by hold
// c^T x, b^T y of the undivided point.
__global__ void k_output(const Ctl* c, int64_t n, int64_t m, const float* __restrict__ ux,
                         const float* __restrict__ uy, const float* __restrict__ vs,
                         const float* __restrict__ d, const float* __restrict__ e,
                         const float* __restrict__ dinv, double* __restrict__ out) {
  const int st = c->status;
  const double tau = c->tau;
  double sx, sy, ss;  // multipliers for x, y, s
  if (st == CF_INFEASIBLE) {
    sx = NAN; ss = NAN; sy = 1.0 / (-c->by);
  } else if (st == CF_UNBOUNDED) {
    sx = 1.0 / (-c->cx); ss = sx; sy = NAN;
  } else if (tau > 0.0) {
    sx = sy = ss = 1.0 / tau;
  } else {
    sx = sy = ss = NAN;
  }
  const double fx = sx / c->sigma, fy = sy / c->rho, fs = ss / c->sigma;
  GRID_STRIDE(i, n) out[i] = (double)ux[i] * (e ? (double)e[i] : 1.0) * fx;
  GRID_STRIDE(i, m) {
    out[n + i] = (double)uy[i] * (d ? (double)d[i] : 1.0) * fy;
    out[n + m + i] = (double)vs[i] * (dinv ? (double)dinv[i] : 1.0) * fs;
  }
}

__global__ void k_export_uv(const Ctl* c, int64_t n, int64_t m, const float* __restrict__ ux,
                            const float* __restrict__ uy, const float* __restrict__ vs,
                            double* __restrict__ uv) {
  const int64_t N = n + m + 1;
  GRID_STRIDE(i, n) {
    uv[i] = ux[i];
    uv[N + i] = 0.0;
  }
  GRID_STRIDE(i, m) {
    uv[n + i] = uy[i];
    uv[N + n + i] = vs[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uv[n + m] = c->tau;
    uv[N + n + m] = c->kappa;
  }
}

// ------------------------------------------------------------ graph building
namespace {

struct Seg {
  cudaStream_t s;
  std::vector<cudaGraphNode_t> tail;
};

// Launch with programmatic stream serialisation (see pdl_wait): the kernel
// may begin while the previous kernel on the stream finishes.  Inside a
// captured graph this becomes a programmatic edge.
template <class... KArgs, class... Args>
void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

cf_err seg_begin(cudaStream_t s, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps) {
  CF_CUDA(cudaStreamBeginCaptureToGraph(s, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                        deps.size(), cudaStreamCaptureModeRelaxed));
  return CF_OK;
}

cf_err seg_end(cudaStream_t s, std::vector<cudaGraphNode_t>* tail) {
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaGraph_t g;
  CF_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  std::vector<cudaGraphNode_t> t(deps, deps + nd);
  cudaGraph_t out;
  CF_CUDA(cudaStreamEndCapture(s, &out));
  if (tail) *tail = t;
  return CF_OK;
}

cf_err add_cond(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                cudaGraphNode_t* node, cudaGraph_t* body) {
  // zero-filled storage: the params union has no usable default constructor
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  CF_CUDA(cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
  *body = p.conditional.phGraph_out[0];
  return CF_OK;
}

int count_kernels(cudaGraph_t g) {
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Buffers of one CG run on (lam I + A^T A) z = rhs.  With folded diagonal
// blocks (fold.nb > 0), the Gram pass applies A's other blocks (skip) and the
// blocks' diagonal (fold.gd) enters through q's start value.
struct CgBufs {
  Ctl* ctl;
  const cf_op* A;
  int64_t n, m;
  float *z, *rhs, *r, *p, *q, *t, *ws;
  float *gz, *az;  // G z and A z carried along (az may be null)
  double* part;
  Fold fold = {};
  const uint8_t* skip = nullptr;
};

// Loop-decision handles of the graph being captured; in_graph == 0 when the
// kernels are launched directly by the host-driven loop.
struct Conds {
  cudaGraphConditionalHandle outer = 0, cg = 0, check = 0, refresh = 0;
  int in_graph = 1;
};

// Gram pass out = A^T A x (the CG kernels add lam x).  Folded: the other
// blocks only; acc: added onto out (the CG step's q starts at (lam + gd) p).
void gram(const CgBufs& b, const float* x, float* out, bool acc, cudaStream_t s) {
  op_apply(b.A, false, 1.f, x, b.t, false, b.ws, s, false, b.skip);
  op_apply(b.A, true, 1.f, b.t, out, acc, b.ws, s, false, b.skip);
}

// CG start at z with gz = G z already known (fresh = 0) or computed here
// from scratch (fresh = 1).
void emit_cg_start(const CgBufs& b, int mode, int fresh, const Conds& cd, cudaStream_t s) {
  if (fresh) gram(b, b.z, b.gz, false, s);
  k_cg_init<<<red_grid(b.n), kThreads, 0, s>>>(b.ctl, b.n, b.rhs, b.z, b.gz, b.r, b.p, b.part, mode, fresh,
                                               cd.cg, cd.in_graph, b.fold.gd, b.q);
}

// One CG step (body of the CG WHILE node).
void emit_cg_step(const CgBufs& b, int mode, const Conds& cd, cudaStream_t s) {
  const bool folded = b.fold.nb > 0;
  gram(b, b.p, b.q, folded, s);
  k_cg_dot<<<red_grid(b.n), kThreads, 0, s>>>(b.ctl, b.n, b.p, b.q, b.part, folded ? 1 : 0);
  launch_pdl(k_cg_update, (unsigned)red_grid(b.n), kThreads, s, b.ctl, b.n, b.m, b.z, b.r, (const float*)b.p,
             (const float*)b.q, b.gz, b.az, (const float*)b.t, b.part, mode, b.fold, folded ? 1 : 0);
  launch_pdl(k_cg_p, (unsigned)grid_for(b.n), kThreads, s, b.ctl, b.n, (const float*)b.r, b.p, mode, cd.cg,
             cd.in_graph, (const float*)b.fold.gd, b.q);
}

// CG buffers on z; the ADMM iterations' CG steps apply the inner operator
// when one is set (the setup's always apply A).  The folded blocks belong to
// A, so they apply whenever A does.
CgBufs cg_bufs(cf_problem* P, float* z, bool iter = false) {
  const cf_op* A = iter && P->inner ? P->inner : P->A;
  CgBufs b{P->ctl, A, P->n, P->m, z, P->rhs, P->r, P->p, P->qv, P->t, P->ws, P->gz, P->az, P->part};
  if (A == P->A && P->fold.nb > 0) {
    b.fold = P->fold;
    b.skip = P->fold_skip.data();
  }
  return b;
}

// ---- the pieces of the setup and of one ADMM iteration
void emit_setup_pre(cf_problem* P, const Conds& cd, cudaStream_t s) {
  const int64_t n = P->n, m = P->m;
  k_setup_init<<<grid_for(std::max(n, m)), kThreads, 0, s>>>(P->ctl, n, m, P->gx, P->gz, P->az, P->rhs, P->cf);
  op_apply(P->A, true, -1.f, P->bf, P->rhs, true, P->ws, s);  // rhs = c - A^T b
  emit_cg_start(cg_bufs(P, P->gx), CG_SETUP, 0, cd, s);        // g_x = 0, G g_x = 0
}

void emit_setup_post(cf_problem* P, cudaStream_t s) {
  const int64_t n = P->n, m = P->m;
  op_apply(P->A, false, 1.f, P->gx, P->gy, false, P->ws, s);  // exact A g_x
  k_setup_fin<<<red_grid(std::max(n, m)), kThreads, 0, s>>>(P->ctl, n, m, P->gx, P->gy, P->bf, P->cf, P->part);
}

void emit_init(cf_problem* P, cudaStream_t s) {
  const int64_t n = P->n, m = P->m;
  k_init<<<grid_for(std::max(n, m)), kThreads, 0, s>>>(P->ctl, n, m, P->ux, P->uy, P->vs, P->zx, P->gz, P->az,
                                                       P->warm_dev);
}

// w = u + v; rhs = w_x - A^T w_y; CG start at the previous z_x
void emit_pre_cg(cf_problem* P, const Conds& cd, cudaStream_t s) {
  const int64_t n = P->n, m = P->m;
  k_rhs<<<grid_for(std::max(n, m)), kThreads, 0, s>>>(P->ctl, n, m, P->ux, P->uy, P->vs, P->wy, P->rhs,
                                                       P->fold);
  op_apply(P->A, true, -1.f, P->wy, P->rhs, true, P->ws, s, false, P->fold.nb ? P->fold_skip.data() : nullptr);
  emit_cg_start(cg_bufs(P, P->zx, true), CG_ITER, 0, cd, s);
}

// subspace step, projection, dual update
void emit_post_cg(cf_problem* P, const Conds& cd, cudaStream_t s) {
  const int64_t n = P->n, m = P->m;
  k_utau<<<red_grid(std::max(n, m)), kThreads, 0, s>>>(P->ctl, n, m, P->zx, P->az, P->zy, P->wy, P->bf, P->cf,
                                                       P->part, P->fold);
  if (P->nchunk > 0)
    k_soc_norm<<<(unsigned)P->nchunk, kThreads, 0, s>>>(P->ctl, P->chunk_seg, P->chunk_r0, P->chunk_r1,
                                                        P->seg_head, P->seg_c0, P->seg_nc, P->zy, P->gy,
                                                        P->uy, P->vs, P->chunk_n2, P->seg_p0, P->seg_nrm,
                                                        P->seg_cnt);
  const int nlin = grid_for(std::max<int64_t>(n, P->z + P->l));
  k_apply<<<(unsigned)(nlin + P->nchunk), kThreads, 0, s>>>(
      P->ctl, n, m, P->z, P->l, nlin, P->ux, P->uy, P->vs, P->zx, P->zy, P->gx, P->gy, P->chunk_seg,
      P->chunk_r0, P->chunk_r1, P->seg_head, P->seg_nrm, P->seg_p0, cd.check, cd.refresh, cd.outer,
      cd.in_graph);
}

// residuals and certificates (every check_interval iterations)
void emit_check(cf_problem* P, const Conds& cd, cudaStream_t s) {
  const int64_t n = P->n, m = P->m;
  op_apply(P->A, false, 1.f, P->ux, P->cm, false, P->ws, s);
  op_apply(P->A, true, 1.f, P->uy, P->cn, false, P->ws, s);
  k_resid<<<red_grid(std::max(n, m)), kThreads, 0, s>>>(P->ctl, n, m, P->cm, P->cn, P->ux, P->uy, P->vs,
                                                        P->bf, P->cf, P->eq_dinv, P->eq_einv, P->part, cd.outer,
                                                        cd.in_graph);
}

// exact A z_x and G z_x (every kRefreshInterval iterations)
void emit_refresh(cf_problem* P, cudaStream_t s) {
  op_apply(P->A, false, 1.f, P->zx, P->az, false, P->ws, s);
  op_apply(P->A, true, 1.f, P->az, P->gz, false, P->ws, s);
  k_gz_shift<<<grid_for(P->n), kThreads, 0, s>>>(P->ctl, P->n, P->zx, P->gz);
}


cf_err build_setup_graph(cf_problem* P) {
  cudaStream_t s = P->stream;
  cudaGraph_t G;
  CF_CUDA(cudaGraphCreate(&G, 0));
  P->setup_graph = G;
  Conds cd;
  CF_CUDA(cudaGraphConditionalHandleCreate(&cd.cg, G, 0, 0));
  std::vector<cudaGraphNode_t> tail, tmp;
  CF_TRY(seg_begin(s, G, {}));
  emit_setup_pre(P, cd, s);
  CF_TRY(seg_end(s, &tail));
  cudaGraphNode_t wn;
  cudaGraph_t body = nullptr;
  CF_TRY(add_cond(G, tail, cd.cg, cudaGraphCondTypeWhile, &wn, &body));
  CF_TRY(seg_begin(s, body, {}));
  emit_cg_step(cg_bufs(P, P->gx), CG_SETUP, cd, s);
  CF_TRY(seg_end(s, &tmp));
  CF_TRY(seg_begin(s, G, {wn}));
  emit_setup_post(P, s);
  CF_TRY(seg_end(s, &tmp));
  CF_CUDA(cudaGetLastError());
  P->skc.top = count_kernels(G);
  P->skc.cg = count_kernels(body);
  CF_CUDA(cudaGraphInstantiate(&P->setup_exec, G, 0));
  return CF_OK;
}

cf_err build_iter_graph(cf_problem* P) {
  cudaStream_t s = P->stream;
  cudaGraph_t G;
  CF_CUDA(cudaGraphCreate(&G, 0));
  P->graph = G;
  Conds cd;
  CF_CUDA(cudaGraphConditionalHandleCreate(&cd.outer, G, 1, cudaGraphCondAssignDefault));
  std::vector<cudaGraphNode_t> tail, tmp;
  CF_TRY(seg_begin(s, G, {}));
  emit_init(P, s);
  CF_TRY(seg_end(s, &tail));
  cudaGraphNode_t wn;
  cudaGraph_t B = nullptr;
  CF_TRY(add_cond(G, tail, cd.outer, cudaGraphCondTypeWhile, &wn, &B));
  CF_CUDA(cudaGraphConditionalHandleCreate(&cd.cg, B, 0, 0));
  CF_CUDA(cudaGraphConditionalHandleCreate(&cd.check, B, 0, 0));
  CF_CUDA(cudaGraphConditionalHandleCreate(&cd.refresh, B, 0, 0));
  // body: rhs and CG start, CG loop, subspace step + projection (which also
  // decides the loop), residual check (which may revise it), refresh
  CF_TRY(seg_begin(s, B, {}));
  emit_pre_cg(P, cd, s);
  CF_TRY(seg_end(s, &tail));
  cudaGraphNode_t cgn;
  cudaGraph_t C = nullptr;
  CF_TRY(add_cond(B, tail, cd.cg, cudaGraphCondTypeWhile, &cgn, &C));
  CF_TRY(seg_begin(s, C, {}));
  emit_cg_step(cg_bufs(P, P->zx, true), CG_ITER, cd, s);
  CF_TRY(seg_end(s, &tmp));
  CF_TRY(seg_begin(s, B, {cgn}));
  emit_post_cg(P, cd, s);
  CF_TRY(seg_end(s, &tail));
  cudaGraphNode_t ifn;
  cudaGraph_t D = nullptr;
  CF_TRY(add_cond(B, tail, cd.check, cudaGraphCondTypeIf, &ifn, &D));
  CF_TRY(seg_begin(s, D, {}));
  emit_check(P, cd, s);
  CF_TRY(seg_end(s, &tmp));
  cudaGraphNode_t rfn;
  cudaGraph_t R = nullptr;
  CF_TRY(add_cond(B, {ifn}, cd.refresh, cudaGraphCondTypeIf, &rfn, &R));
  CF_TRY(seg_begin(s, R, {}));
  emit_refresh(P, s);
  CF_TRY(seg_end(s, &tmp));
  CF_CUDA(cudaGetLastError());
  P->kc.top = count_kernels(G);
  P->kc.body = count_kernels(B);
  P->kc.cg = count_kernels(C);
  P->kc.check = count_kernels(D);
  P->kc.refresh = count_kernels(R);
  CF_CUDA(cudaGraphInstantiate(&P->exec, G, 0));
  return CF_OK;
}

// ---- host-driven execution of the same kernels (no graph)
struct Flags {
  int cg_go, do_check, do_refresh, outer_go;
};

// Read the loop decisions the kernels stored (one small copy and a wait).
cf_err read_flags(cf_problem* P, Flags* f) {
  CF_CUDA(cudaMemcpyAsync(P->flags_host, &P->ctl->cg_go, sizeof(Flags), cudaMemcpyDeviceToHost, P->stream));
  CF_CUDA(cudaStreamSynchronize(P->stream));
  std::memcpy(f, P->flags_host, sizeof(Flags));
  return CF_OK;
}

// Runs the setup CG loop from the host; the loop is also capped on the host.
cf_err run_setup_host(cf_problem* P, int64_t* launches) {
  cudaStream_t s = P->stream;
  Conds cd;
  cd.in_graph = 0;
  const CgBufs cb = cg_bufs(P, P->gx);
  Flags f;
  int steps = 0;
  emit_setup_pre(P, cd, s);
  CF_CUDA(cudaGetLastError());
  CF_TRY(read_flags(P, &f));
  while (f.cg_go && steps < P->ctl_host->st.setup_cg_max) {
    emit_cg_step(cb, CG_SETUP, cd, s);
    CF_CUDA(cudaGetLastError());
    CF_TRY(read_flags(P, &f));
    ++steps;
  }
  emit_setup_post(P, s);
  CF_CUDA(cudaGetLastError());
  *launches += P->skc.top + (int64_t)steps * P->skc.cg;
  return CF_OK;
}

// Runs the ADMM iterations from the host: identical kernels, with each loop
// decision read back instead of evaluated by a conditional graph node.
cf_err run_iterations_host(cf_problem* P) {
  cudaStream_t s = P->stream;
  Conds cd;
  cd.in_graph = 0;
  const CgBufs cb = cg_bufs(P, P->zx, true);
  const Settings& st = P->ctl_host->st;
  const int cg_cap = st.cg_fixed > 0 ? st.cg_fixed : st.cg_max;
  Flags f;
  emit_init(P, s);
  for (int it = 0; it < st.max_iters; ++it) {
    emit_pre_cg(P, cd, s);
    CF_CUDA(cudaGetLastError());
    CF_TRY(read_flags(P, &f));
    for (int k = 0; f.cg_go && k < cg_cap; ++k) {
      emit_cg_step(cb, CG_ITER, cd, s);
      CF_CUDA(cudaGetLastError());
      CF_TRY(read_flags(P, &f));
    }
    emit_post_cg(P, cd, s);
    CF_TRY(read_flags(P, &f));
    const int refresh = f.do_refresh;
    if (f.do_check) {
      emit_check(P, cd, s);
      CF_TRY(read_flags(P, &f));
    }
    if (refresh) emit_refresh(P, s);
    CF_CUDA(cudaGetLastError());
    if (!f.outer_go) break;
  }
  return CF_OK;
}

}  // namespace

// ------------------------------------------------------------ state
size_t solver_ws_floats(const cf_problem* P) {
  size_t w = std::max(op_ws_floats(P->A, false), op_ws_floats(P->A, true));
  if (P->inner) w = std::max(w, std::max(op_ws_floats(P->inner, false), op_ws_floats(P->inner, true)));
  return w;
}

size_t problem_state_bytes(const cf_problem* P) {
  const size_t n = P->n, m = P->m, N = n + m + 1;
  auto f = [](size_t k) { return align_up(k * sizeof(float), 256); };
  auto d = [](size_t k) { return align_up(k * sizeof(double), 256); };
  size_t wsf = solver_ws_floats(P);
  size_t b = 0;
  b += 10 * f(n);           // ux zx rhs r p q gx cn gz, fold_gd
  b += 9 * f(m);            // uy vs wy t zy gy cm az, fold_s
  b += f(wsf);
  b += f(std::max<size_t>(team::scratch_floats(P), 1));
  b += d((size_t)kMaxRedBlocks * kRedSlots);
  b += d((size_t)std::max<int64_t>(P->nchunk, 1)) + 3 * d((size_t)std::max<int64_t>(P->nseg, 1));
  b += 2 * d(2 * N);        // warm_dev, uv_dev
  b += d(n + 2 * m);        // out_dev
  b += align_up(sizeof(Ctl), 256);
  return b;
}

cf_err ensure_state(cf_problem* P) {
  if (P->arena) return CF_OK;
  const size_t n = P->n, m = P->m, N = n + m + 1;
  size_t bytes = problem_state_bytes(P);
  void* a = nullptr;
  cudaError_t e = cudaMalloc(&a, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CF_E_OOM, std::string("solver state allocation failed: ") + cudaGetErrorString(e));
  }
  P->arena = a;
  P->state_bytes = bytes;
  char* cur = (char*)a;
  auto takef = [&](size_t k) { float* r = (float*)cur; cur += align_up(k * sizeof(float), 256); return r; };
  auto taked = [&](size_t k) { double* r = (double*)cur; cur += align_up(k * sizeof(double), 256); return r; };
  P->ux = takef(n); P->zx = takef(n); P->rhs = takef(n); P->r = takef(n);
  P->p = takef(n); P->qv = takef(n); P->gx = takef(n); P->cn = takef(n);
  P->uy = takef(m); P->vs = takef(m); P->wy = takef(m); P->t = takef(m);
  P->zy = takef(m); P->gy = takef(m); P->cm = takef(m);
  P->gz = takef(n); P->az = takef(m);
  P->fold_gd = takef(n); P->fold_s = takef(m);
  P->ws = takef(solver_ws_floats(P));
  P->team_scratch = takef(std::max<size_t>(team::scratch_floats(P), 1));
  P->part = taked((size_t)kMaxRedBlocks * kRedSlots);
  P->chunk_n2 = taked((size_t)std::max<int64_t>(P->nchunk, 1));
  P->seg_p0 = taked((size_t)std::max<int64_t>(P->nseg, 1));
  P->seg_nrm = taked((size_t)std::max<int64_t>(P->nseg, 1));
  P->seg_cnt = (unsigned int*)taked((size_t)std::max<int64_t>(P->nseg, 1));
  P->warm_dev = taked(2 * N);
  P->uv_dev = taked(2 * N);
  P->out_dev = taked(n + 2 * m);
  P->ctl = (Ctl*)cur;
  CF_CUDA(cudaMemsetAsync(P->ctl, 0, sizeof(Ctl), P->stream));
  // diagonal row blocks folded out of the graph engine's CG passes (not with
  // an inner operator: its CG steps carry A z from the inner copy); t is
  // zeroed so that the rows the folded passes never write stay zero
  CF_CUDA(cudaMemsetAsync(P->t, 0, m * sizeof(float), P->stream));
  P->fold = Fold{};
  P->fold_skip.clear();
  std::vector<DiagBlock> blocks;
  if (!P->inner && fold_diag_blocks(P->A, &blocks, &P->fold_skip)) {
    Fold f;
    FoldSrc src{};
    f.nb = (int)blocks.size();
    for (int b = 0; b < f.nb; ++b) {
      f.r0[b] = blocks[b].r0;
      f.c0[b] = blocks[b].c0;
      f.len[b] = blocks[b].len;
      src.alpha[b] = blocks[b].alpha;
      src.d[b] = blocks[b].d;
    }
    f.s = P->fold_s;
    f.gd = P->fold_gd;
    k_fold_prep<<<grid_for(std::max(n, m)), kThreads, 0, P->stream>>>(f, src, (int64_t)m, (int64_t)n, P->eq_d,
                                                                       P->eq_e, P->fold_s, P->fold_gd);
    CF_CUDA(cudaGetLastError());
    P->fold = f;
  } else {
    P->fold_skip.clear();
  }
  CF_CUDA(cudaMemsetAsync(P->seg_cnt, 0, sizeof(double) * std::max<int64_t>(P->nseg, 1), P->stream));
  CF_CUDA(cudaMemsetAsync(P->warm_dev, 0, 2 * N * sizeof(double), P->stream));
  CF_CUDA(cudaStreamSynchronize(P->stream));
  P->ctl_host->nb = P->nb;
  P->ctl_host->nc = P->nc;
  P->ctl_host->sigma = P->sigma;
  P->ctl_host->rho = P->rho;
  CF_CUDA(cudaMemcpy(&P->ctl->nb, &P->nb, sizeof(double), cudaMemcpyHostToDevice));
  CF_CUDA(cudaMemcpy(&P->ctl->nc, &P->nc, sizeof(double), cudaMemcpyHostToDevice));
  CF_CUDA(cudaMemcpy(&P->ctl->sigma, &P->sigma, sizeof(double), cudaMemcpyHostToDevice));
  CF_CUDA(cudaMemcpy(&P->ctl->rho, &P->rho, sizeof(double), cudaMemcpyHostToDevice));
  P->setup_done = false;
  return CF_OK;
}

void release_state(cf_problem* P) {
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->setup_exec) cudaGraphExecDestroy(P->setup_exec);
  if (P->setup_graph) cudaGraphDestroy(P->setup_graph);
  P->exec = nullptr;
  P->graph = nullptr;
  P->setup_exec = nullptr;
  P->setup_graph = nullptr;
  if (P->arena) cudaFree(P->arena);
  P->arena = nullptr;
  P->team_scratch = nullptr;
  P->fold = Fold{};
  P->fold_skip.clear();
  P->fold_s = P->fold_gd = nullptr;
  P->setup_done = false;
}

bool settings_valid(const cf_settings* st, std::string* why) {
  auto bad = [&](const char* w) { *why = w; return false; };
  if (!(st->eps > 0)) return bad("eps must be > 0");
  if (!(st->eps_infeas > 0)) return bad("eps_infeas must be > 0");
  if (!(st->alpha > 0 && st->alpha < 2)) return bad("alpha must be in (0, 2)");
  if (st->max_iters < 1) return bad("max_iters must be >= 1");
  if (st->check_interval < 1) return bad("check_interval must be >= 1");
  if (st->cg_max_iters < 0 || st->cg_max_iters > 100000) return bad("cg_max_iters must be in [0, 100000]");
  if (st->cg_fixed_iters < 0 || st->cg_fixed_iters > 100000) return bad("cg_fixed_iters must be in [0, 100000]");
  if (st->setup_cg_max_iters < 1 || st->setup_cg_max_iters > 1000000) return bad("setup_cg_max_iters must be in [1, 1e6]");
  if (!(st->setup_cg_tol > 0)) return bad("setup_cg_tol must be > 0");
  if (!(st->cg_tol_rel >= 0) || !(st->cg_tol_min >= 0) || !std::isfinite(st->cg_tol_exp))
    return bad("CG tolerance parameters must be >= 0");
  if (st->host_loop != 0 && st->host_loop != 1) return bad("host_loop must be 0 or 1");
  if (st->engine != CF_ENGINE_AUTO && st->engine != CF_ENGINE_GRAPH && st->engine != CF_ENGINE_TEAM &&
      st->engine != CF_ENGINE_GRID)
    return bad("engine must be CF_ENGINE_AUTO, CF_ENGINE_GRAPH, CF_ENGINE_TEAM or CF_ENGINE_GRID");
  if (st->host_loop && (st->engine == CF_ENGINE_TEAM || st->engine == CF_ENGINE_GRID))
    return bad("host_loop runs the graph engine's kernels");
  return true;
}

void write_settings(cf_problem* P, const cf_settings* st, bool warm) {
  Settings& s = P->ctl_host->st;
  s.alpha = st->alpha;
  s.eps = st->eps;
  s.eps_inf = st->eps_infeas;
  s.cg_tol_rel = st->cg_tol_rel;
  s.cg_tol_exp = st->cg_tol_exp;
  s.cg_tol_min = st->cg_tol_min;
  s.setup_tol = st->setup_cg_tol;
  s.max_iters = st->max_iters;
  s.check_interval = st->check_interval;
  s.cg_max = st->cg_max_iters;
  s.cg_fixed = st->cg_fixed_iters;
  s.setup_cg_max = st->setup_cg_max_iters;
  s.warm = warm ? 1 : 0;
}

// Setup (g = M^{-1} h) is stream-ordered before the iterations: nothing waits
// for it on the host, so fresh problems of a batch overlap their setups.  Its
// CG step count arrives with the control block copied back after the solve.
static cf_err run_setup(cf_problem* P, bool host_loop) {
  if (!P->setup_exec) CF_TRY(build_setup_graph(P));  // also gives the kernel counts
  P->setup_sig = 1;
  CF_CUDA(cudaMemcpyAsync(&P->ctl->st, &P->ctl_host->st, sizeof(Settings), cudaMemcpyHostToDevice, P->stream));
  if (host_loop) {
    int64_t dummy = 0;
    CF_TRY(run_setup_host(P, &dummy));
  } else {
    CF_CUDA(cudaGraphLaunch(P->setup_exec, P->stream));
  }
  P->setup_done = true;
  return CF_OK;
}

cf_err solve_launch(cf_problem* P, const cf_settings* st_in, double* x, double* y, double* s,
                    const double* warm_uv, double* uv_out, bool join_ctx) {
  cf_settings st;
  if (st_in)
    st = *st_in;
  else
    cf_settings_default(&st);
  std::string why;
  if (!settings_valid(&st, &why)) return fail(CF_E_INVALID, "solve: " + why);
  const int64_t t0 = now_ns();
  int engine = CF_ENGINE_GRAPH;
  CF_TRY(pick_engine(P, &st, &engine));
  CF_TRY(ensure_state(P));
  write_settings(P, &st, warm_uv != nullptr);
  P->ran_setup = false;
  if (engine == CF_ENGINE_TEAM || engine == CF_ENGINE_GRID) {
    P->x_out = x;
    P->y_out = y;
    P->s_out = s;
    P->uv_out = uv_out;
    if (engine == CF_ENGINE_GRID)
      CF_TRY(team::grid_launch(P, &st, warm_uv, join_ctx));
    else
      CF_TRY(team::solo_launch(P, &st, warm_uv, join_ctx));
    P->setup_ns_last = P->ran_setup ? now_ns() - t0 : 0;
    return CF_OK;
  }
  P->last_engine = CF_ENGINE_GRAPH;
  // order after earlier work on the context stream
  CF_CUDA(cudaEventRecord(P->ev_in, P->ctx->stream));
  CF_CUDA(cudaStreamWaitEvent(P->stream, P->ev_in, 0));
  if (!P->setup_done || P->setup_sig != 1) {
    CF_TRY(run_setup(P, st.host_loop != 0));
    P->ran_setup = true;
    P->setup_ns_last = now_ns() - t0;
  } else {
    P->setup_ns_last = 0;
  }
  if (!P->exec) CF_TRY(build_iter_graph(P));
  const int64_t N = P->n + P->m + 1;
  if (warm_uv) CF_TRY(copy_any(P->warm_dev, warm_uv, 2 * N * sizeof(double), P->stream));
  CF_CUDA(cudaMemcpyAsync(&P->ctl->st, &P->ctl_host->st, sizeof(Settings), cudaMemcpyHostToDevice, P->stream));
  P->t_launch = now_ns();
  if (st.host_loop)
    CF_TRY(run_iterations_host(P));
  else
    CF_CUDA(cudaGraphLaunch(P->exec, P->stream));
  P->x_out = x;
  P->y_out = y;
  P->s_out = s;
  P->uv_out = uv_out;
  if (x || y || s) {
    k_output<<<grid_for(std::max(P->n, P->m)), kThreads, 0, P->stream>>>(P->ctl, P->n, P->m, P->ux, P->uy,
                                                                       P->vs, P->eq_d, P->eq_e, P->eq_dinv,
                                                                       P->out_dev);
    CF_CUDA(cudaGetLastError());
  }
  if (uv_out) {
    k_export_uv<<<grid_for(std::max(P->n, P->m)), kThreads, 0, P->stream>>>(P->ctl, P->n, P->m, P->ux,
                                                                           P->uy, P->vs, P->uv_dev);
    CF_CUDA(cudaGetLastError());
  }
  CF_CUDA(cudaMemcpyAsync(P->ctl_host, P->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P->stream));
  CF_CUDA(cudaEventRecord(P->ev_out, P->stream));
  if (join_ctx) CF_CUDA(cudaStreamWaitEvent(P->ctx->stream, P->ev_out, 0));
  return CF_OK;
}

cf_err solve_finish(cf_problem* P, cf_info* info) {
  CF_CUDA(cudaStreamSynchronize(P->stream));
  const int64_t t1 = now_ns();
  const int64_t n = P->n, m = P->m, N = n + m + 1;
  if (P->x_out) CF_TRY(copy_any(P->x_out, P->out_dev, n * sizeof(double), P->stream));
  if (P->y_out) CF_TRY(copy_any(P->y_out, P->out_dev + n, m * sizeof(double), P->stream));
  if (P->s_out) CF_TRY(copy_any(P->s_out, P->out_dev + n + m, m * sizeof(double), P->stream));
  if (P->uv_out) CF_TRY(copy_any(P->uv_out, P->uv_dev, 2 * N * sizeof(double), P->stream));
  CF_CUDA(cudaStreamSynchronize(P->stream));
  const Ctl& c = *P->ctl_host;
  if (P->last_engine == CF_ENGINE_GRID && c.grid_abort) {
    P->setup_done = false;  // g = M^-1 h may be incomplete: the next solve recomputes it
    return fail(CF_E_CUDA, "solve: a grid-wide barrier wait of the grid engine gave up (the solve was abandoned)");
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = c.status;
    info->iters = c.k;
    info->cg_iters_total = c.cg_total;
    info->checks = c.checks;
    if (P->ran_setup) P->setup_iters_last = c.setup_iters;
    info->setup_cg_iters = P->ran_setup ? P->setup_iters_last : 0;
    info->pri_res = c.pri;
    info->dual_res = c.dual;
    info->gap = c.gap;
    const double tau = c.tau;
    info->pobj = tau > 0 ? c.cx / tau : NAN;
    info->dobj = tau > 0 ? -c.by / tau : NAN;
    info->tau = c.tau;
    info->kappa = c.kappa;
    info->setup_ns = P->setup_ns_last;
    info->solve_ns = t1 - P->t_launch;
    if (P->last_engine == CF_ENGINE_TEAM || P->last_engine == CF_ENGINE_GRID) {
      info->kernel_launches = P->team_launches;  // the whole solve is one persistent launch
      info->device_ns = c.t_end - c.t_start;
    } else {
      int64_t kl = P->kc.top + (int64_t)c.k * P->kc.body + c.cg_total * P->kc.cg +
                   (int64_t)c.checks * P->kc.check + (int64_t)c.refreshes * P->kc.refresh;
      if (P->x_out || P->y_out || P->s_out) kl += 1;
      if (P->uv_out) kl += 1;
      if (P->ran_setup) kl += P->skc.top + (int64_t)P->setup_iters_last * P->skc.cg;
      info->kernel_launches = kl;
    }
  }
  return CF_OK;
}

// k_cg_init/update with mode CG_SETUP read their threshold and cap from the
// setup fields; a standalone CG run sets those and the shift lam.
__global__ void k_cg_solo_init(Ctl* c, double lam, double tol, int max_iters) {
  c->lam = lam;
  c->st.setup_tol = tol;
  c->st.setup_cg_max = max_iters;
  c->setup_iters = 0;
  c->red_count = 0u;
}

cf_err cg_solve_impl(cf_op* A, double lam, const float* rhs_in, float* x, int32_t max_iters,
                     double tol, int32_t* iters, double* res_norm) {
  cf_ctx* ctx = A->ctx;
  const int64_t n = A->n, m = A->m;
  const size_t wsf = std::max(op_ws_floats(A, false), op_ws_floats(A, true));
  auto f = [](size_t k) { return align_up(k * sizeof(float), 256); };
  const size_t bytes = 6 * f(n) + f(m) + f(wsf) +
                       align_up(sizeof(double) * kMaxRedBlocks * kRedSlots, 256) + align_up(sizeof(Ctl), 256);
  char* arena = nullptr;
  cudaError_t e = cudaMalloc((void**)&arena, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CF_E_OOM, "cg_solve: allocation failed");
  }
  char* cur = arena;
  auto take = [&](size_t b) { char* r = cur; cur += align_up(b, 256); return r; };
  CgBufs b;
  b.A = A;
  b.n = n;
  b.m = m;
  b.z = (float*)take(n * 4);
  b.rhs = (float*)take(n * 4);
  b.r = (float*)take(n * 4);
  b.p = (float*)take(n * 4);
  b.q = (float*)take(n * 4);
  b.gz = (float*)take(n * 4);
  b.az = nullptr;
  b.t = (float*)take(m * 4);
  b.ws = (float*)take(wsf * 4);
  b.part = (double*)take(sizeof(double) * kMaxRedBlocks * kRedSlots);
  b.ctl = (Ctl*)take(sizeof(Ctl));
  cudaStream_t s = nullptr;
  cudaGraph_t G = nullptr;
  cudaGraphExec_t ex = nullptr;
  Ctl* hc = nullptr;
  cudaEvent_t ev = nullptr;
  auto run = [&]() -> cf_err {
    CF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    CF_CUDA(cudaMallocHost((void**)&hc, sizeof(Ctl)));
    CF_CUDA(cudaMemsetAsync(b.ctl, 0, sizeof(Ctl), s));
    CF_TRY(copy_any(b.rhs, rhs_in, n * sizeof(float), s));
    CF_TRY(copy_any(b.z, x, n * sizeof(float), s));
    CF_CUDA(cudaGraphCreate(&G, 0));
    Conds cd;
    CF_CUDA(cudaGraphConditionalHandleCreate(&cd.cg, G, 0, 0));
    std::vector<cudaGraphNode_t> tail, tmp;
    CF_TRY(seg_begin(s, G, {}));
    k_cg_solo_init<<<1, 1, 0, s>>>(b.ctl, lam, tol, max_iters);
    emit_cg_start(b, CG_SETUP, 1, cd, s);
    CF_TRY(seg_end(s, &tail));
    cudaGraphNode_t wn;
    cudaGraph_t body = nullptr;
    CF_TRY(add_cond(G, tail, cd.cg, cudaGraphCondTypeWhile, &wn, &body));
    CF_TRY(seg_begin(s, body, {}));
    emit_cg_step(b, CG_SETUP, cd, s);
    CF_TRY(seg_end(s, &tmp));
    CF_CUDA(cudaGetLastError());
    CF_CUDA(cudaGraphInstantiate(&ex, G, 0));
    CF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CF_CUDA(cudaEventRecord(ev, ctx->stream));
    CF_CUDA(cudaStreamWaitEvent(s, ev, 0));
    CF_CUDA(cudaGraphLaunch(ex, s));
    CF_CUDA(cudaMemcpyAsync(hc, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CF_TRY(copy_any(x, b.z, n * sizeof(float), s));
    CF_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = hc->setup_iters;
    if (res_norm) *res_norm = std::sqrt(hc->rr);
    return CF_OK;
  };
  cf_err r = run();
  if (ex) cudaGraphExecDestroy(ex);
  if (G) cudaGraphDestroy(G);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (hc) cudaFreeHost(hc);
  if (ev) cudaEventDestroy(ev);
  cudaFree(arena);
  return r;
}

}  // namespace cf

using namespace cf;

// ------------------------------------------------------------------ C ABI
extern "C" {

cf_err cone_problem_create(cf_ctx* ctx, const cf_op* A, const double* b, int64_t m,
                           const double* c, int64_t n, const cf_cone* K, cf_problem** out) {
  if (!ctx || !A || !b || !c || !K || !out) return fail(CF_E_INVALID, "cone_problem_create: NULL argument");
  if (A->m != m || A->n != n) return fail(CF_E_INVALID, "cone_problem_create: operator shape differs from (m, n)");
  if (K->z < 0 || K->l < 0 || K->nq < 0 || (K->nq > 0 && !K->q))
    return fail(CF_E_INVALID, "cone_problem_create: bad cone");
  int64_t tot = K->z + K->l;
  for (int64_t j = 0; j < K->nq; ++j) {
    if (K->q[j] < 1) return fail(CF_E_INVALID, "cone_problem_create: SOC size < 1");
    tot += K->q[j];
  }
  if (tot != m) return fail(CF_E_INVALID, "cone_problem_create: z + l + sum(q) != m");
  DevGuard guard(ctx->device);
  std::unique_ptr<cf_problem> P(new cf_problem());
  P->ctx = ctx;
  P->device = ctx->device;
  P->m = m;
  P->n = n;
  P->z = K->z;
  P->l = K->l;
  P->q.assign(K->q, K->q + K->nq);
  auto run = [&]() -> cf_err {
    // cone tables
    std::vector<int32_t> cseg, sc0, snc;
    std::vector<int64_t> cr0, cr1, shead;
    int64_t off = K->z + K->l;
    for (size_t j = 0; j < P->q.size(); ++j) {
      shead.push_back(off);
      sc0.push_back((int32_t)cr0.size());
      int32_t cnt = 0;
      for (int64_t r = off; r < off + P->q[j]; r += kSocChunk) {
        cseg.push_back((int32_t)j);
        cr0.push_back(r);
        cr1.push_back(std::min(r + kSocChunk, off + P->q[j]));
        ++cnt;
      }
      snc.push_back(cnt);
      off += P->q[j];
    }
    P->nseg = (int64_t)shead.size();
    P->nchunk = (int64_t)cr0.size();
    size_t bytes = align_up(m * 4, 256) + align_up(n * 4, 256) +
                   align_up(std::max<size_t>(P->nchunk, 1) * (4 + 8 + 8), 256) +
                   align_up(std::max<size_t>(P->nseg, 1) * (8 + 4 + 4), 256) + 1024;
    char* base = nullptr;
    cudaError_t e = cudaMalloc((void**)&base, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(CF_E_OOM, "cone_problem_create: allocation failed");
    }
    P->persist_bytes = bytes;
    char* cur = base;
    auto take = [&](size_t k) { char* r = cur; cur += align_up(k, 256); return r; };
    P->bf = (float*)take(m * 4);
    P->cf = (float*)take(n * 4);
    const size_t nch = std::max<size_t>(P->nchunk, 1), nsg = std::max<size_t>(P->nseg, 1);
    P->chunk_r0 = (int64_t*)take(nch * 8);
    P->chunk_r1 = (int64_t*)take(nch * 8);
    P->chunk_seg = (int32_t*)take(nch * 4);
    P->seg_head = (int64_t*)take(nsg * 8);
    P->seg_c0 = (int32_t*)take(nsg * 4);
    P->seg_nc = (int32_t*)take(nsg * 4);
    // b and c: float64 to the device (host or device source), converted,
    // normed and checked there
    {
      cudaStream_t st = ctx->stream;
      const size_t tb = align_up((size_t)(m + n) * 8, 256) + align_up(2 * kPrepGrid * 8, 256) + 256;
      char* tmp = nullptr;
      CF_CUDA(cudaMallocAsync((void**)&tmp, tb, st));
      double* bd = (double*)tmp;
      double* cd = bd + m;
      double* part = (double*)(tmp + align_up((size_t)(m + n) * 8, 256));
      int* bad = (int*)(tmp + align_up((size_t)(m + n) * 8, 256) + align_up(2 * kPrepGrid * 8, 256));
      std::vector<double> hp(2 * kPrepGrid);
      int hbad = 0;
      auto prep = [&]() -> cf_err {
        CF_CUDA(cudaMemcpyAsync(bd, b, m * sizeof(double), cudaMemcpyDefault, st));
        CF_CUDA(cudaMemcpyAsync(cd, c, n * sizeof(double), cudaMemcpyDefault, st));
        CF_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
        k_prep_data<<<kPrepGrid, kThreads, 0, st>>>(m, n, bd, cd, P->bf, P->cf, part, bad);
        CF_CUDA(cudaGetLastError());
        CF_CUDA(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CF_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        CF_CUDA(cudaStreamSynchronize(st));
        return CF_OK;
      };
      const cf_err pr = prep();
      cudaFreeAsync(tmp, st);
      if (pr != CF_OK) return pr;
      if (hbad) return fail(CF_E_INVALID, "cone_problem_create: b or c not finite");
      double nb = 0, nc = 0;
      for (int k = 0; k < kPrepGrid; ++k) {
        nb += hp[2 * k];
        nc += hp[2 * k + 1];
      }
      P->nb = std::sqrt(nb);
      P->nc = std::sqrt(nc);
    }
    if (P->nchunk) {
      CF_CUDA(cudaMemcpy(P->chunk_r0, cr0.data(), P->nchunk * 8, cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(P->chunk_r1, cr1.data(), P->nchunk * 8, cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(P->chunk_seg, cseg.data(), P->nchunk * 4, cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(P->seg_head, shead.data(), P->nseg * 8, cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(P->seg_c0, sc0.data(), P->nseg * 4, cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(P->seg_nc, snc.data(), P->nseg * 4, cudaMemcpyHostToDevice));
    }
    CF_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    CF_CUDA(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
    CF_CUDA(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
    // one pinned block: the control block's mirror, then the loop flags
    char* pin = nullptr;
    CF_CUDA(cudaMallocHost((void**)&pin, align_up(sizeof(Ctl), 64) + 64));
    std::memset(pin, 0, align_up(sizeof(Ctl), 64) + 64);
    P->ctl_host = (Ctl*)pin;
    P->flags_host = pin + align_up(sizeof(Ctl), 64);
    return CF_OK;
  };
  cf_err r = run();
  if (r != CF_OK) {
    cf_problem* raw = P.release();
    raw->A = nullptr;
    cf_problem_destroy(raw);
  } else {
    op_retain(const_cast<cf_op*>(A));
    P->A = const_cast<cf_op*>(A);
    r = team::plan_problem(P.get());
    if (r != CF_OK) {
      cf_problem_destroy(P.release());
      return r;
    }
    *out = P.release();
  }
  return r;
}

void cf_problem_destroy(cf_problem* P) {
  if (!P) return;
  DevGuard guard(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  release_state(P);
  team::release(P);
  if (P->eq) cudaFree(P->eq);
  if (P->A_orig) cf_op_destroy(P->A_orig);
  if (P->inner) cf_op_destroy(P->inner);
  if (P->inner_orig) cf_op_destroy(P->inner_orig);
  if (P->bf) cudaFree(P->bf);  // base of the persistent block
  if (P->ctl_host) cudaFreeHost(P->ctl_host);  // the flags share its block
  if (P->ev_in) cudaEventDestroy(P->ev_in);
  if (P->ev_out) cudaEventDestroy(P->ev_out);
  if (P->stream) cudaStreamDestroy(P->stream);
  if (P->A) cf_op_destroy(P->A);
  delete P;
}

cf_err cone_problem_set_inner(cf_problem* P, const cf_op* inner) {
  if (!P) return fail(CF_E_INVALID, "cone_problem_set_inner: NULL problem");
  if (inner && (inner->m != P->m || inner->n != P->n))
    return fail(CF_E_INVALID, "cone_problem_set_inner: inner operator is " + std::to_string(inner->m) + " x " +
                                  std::to_string(inner->n) + ", A is " + std::to_string(P->m) + " x " +
                                  std::to_string(P->n));
  if (inner && inner->ctx != P->ctx)
    return fail(CF_E_INVALID, "cone_problem_set_inner: inner operator belongs to another context");
  std::lock_guard<std::mutex> lk(P->mtx);
  DevGuard guard(P->device);
  if (P->stream) CF_CUDA(cudaStreamSynchronize(P->stream));
  cf_op* wrapped = nullptr;
  if (inner && P->A_orig) {
    // equilibrated: the same diagonals as A's (parts 0 and 2 of D A E)
    cf_op* parts[3] = {P->A->parts[0], const_cast<cf_op*>(inner), P->A->parts[2]};
    CF_TRY(operator_compose(P->ctx, CF_PRODUCT, parts, 3, 1.0, &wrapped));
  }
  if (P->inner) cf_op_destroy(P->inner);
  if (P->inner_orig) cf_op_destroy(P->inner_orig);
  P->inner = P->inner_orig = nullptr;
  if (inner) {
    op_retain(const_cast<cf_op*>(inner));
    if (wrapped) {
      P->inner = wrapped;
      P->inner_orig = const_cast<cf_op*>(inner);
    } else {
      P->inner = const_cast<cf_op*>(inner);
    }
  }
  // new workspace sizes and graphs; the team plan records the refusal
  release_state(P);
  team::release(P);
  cf_err r = team::plan_problem(P);
  P->setup_done = false;
  P->setup_sig = 0;
  return r;
}

cf_err solve(cf_problem* P, const cf_settings* st, double* x, double* y, double* s,
             const double* warm_uv, double* uv_out, cf_info* info) {
  if (!P) return fail(CF_E_INVALID, "solve: NULL problem");
  std::lock_guard<std::mutex> lk(P->mtx);
  DevGuard guard(P->device);
  cf_err r = solve_launch(P, st, x, y, s, warm_uv, uv_out);
  if (r == CF_OK) r = solve_finish(P, info);
  return r;
}

cf_err solve_batch(cf_problem* const* probs, int32_t count, const cf_settings* st,
                   double* const* xs, double* const* ys, double* const* ss, cf_info* infos) {
  if (count < 0 || (count > 0 && !probs)) return fail(CF_E_INVALID, "solve_batch: bad arguments");
  for (int32_t i = 0; i < count; ++i) {
    if (!probs[i]) return fail(CF_E_INVALID, "solve_batch: NULL problem");
    for (int32_t j = 0; j < i; ++j)
      if (probs[j] == probs[i]) return fail(CF_E_INVALID, "solve_batch: a problem appears twice");
  }
  std::vector<std::unique_lock<std::mutex>> locks;
  for (int32_t i = 0; i < count; ++i) locks.emplace_back(probs[i]->mtx);
  cf_err first = CF_OK;
  std::vector<char> launched(count, 0);
  DevGuard guard(count > 0 ? probs[0]->device : 0);
  cf_settings sv;
  if (st)
    sv = *st;
  else
    cf_settings_default(&sv);
  std::string why;
  if (!settings_valid(&sv, &why)) return fail(CF_E_INVALID, "solve_batch: " + why);
  // team-engine problems, grouped by context: one persistent launch each
  std::vector<std::pair<cf_ctx*, std::vector<int32_t>>> groups;
  for (int32_t i = 0; i < count; ++i) {
    cf_problem* P = probs[i];
    int engine = CF_ENGINE_GRAPH;
    cudaSetDevice(P->device);
    cf_err r = pick_engine(P, &sv, &engine, /*in_batch=*/true);
    if (r == CF_OK && engine == CF_ENGINE_TEAM) {
      r = ensure_state(P);
      if (r == CF_OK) {
        write_settings(P, &sv, false);
        P->x_out = xs ? xs[i] : nullptr;
        P->y_out = ys ? ys[i] : nullptr;
        P->s_out = ss ? ss[i] : nullptr;
        P->uv_out = nullptr;
        size_t g = 0;
        while (g < groups.size() && groups[g].first != P->ctx) ++g;
        if (g == groups.size()) groups.push_back({P->ctx, {}});
        groups[g].second.push_back(i);
        continue;
      }
    }
    if (r == CF_OK)
      r = solve_launch(P, &sv, xs ? xs[i] : nullptr, ys ? ys[i] : nullptr, ss ? ss[i] : nullptr, nullptr,
                       nullptr, /*join_ctx=*/false);
    launched[i] = r == CF_OK;
    if (r != CF_OK && first == CF_OK) first = r;
  }
  for (auto& g : groups) {
    std::vector<cf_problem*> ps;
    for (int32_t i : g.second) ps.push_back(probs[i]);
    cudaSetDevice(g.first->device);
    cf_err r = team::batch_launch(ps, &sv);
    for (int32_t i : g.second) launched[i] = r == CF_OK;
    if (r != CF_OK && first == CF_OK) first = r;
  }
  // every problem was enqueued before any join, so they run concurrently
  for (int32_t i = 0; i < count; ++i)
    if (launched[i]) cudaStreamWaitEvent(probs[i]->ctx->stream, probs[i]->ev_out, 0);
  for (int32_t i = 0; i < count; ++i) {
    if (!launched[i]) continue;
    cf_err r = solve_finish(probs[i], infos ? &infos[i] : nullptr);
    if (r != CF_OK && first == CF_OK) first = r;
  }
  return first;
}

cf_err cg_solve(cf_op* A, double lam, const float* rhs, float* x, int32_t max_iters, double tol,
                int32_t* iters, double* res_norm) {
  if (!A || !rhs || !x || max_iters < 0 || !(tol >= 0) || !(lam >= 0))
    return fail(CF_E_INVALID, "cg_solve: bad arguments");
  DevGuard guard(A->device);
  return cg_solve_impl(A, lam, rhs, x, max_iters, tol, iters, res_norm);
}

}  // extern "C"
