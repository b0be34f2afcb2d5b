// The team engine: the SCS iteration of solver.cu (Section 5.2, following the
// published SCS method the paper cites) run by one persistent kernel in
// which a team of CTAs carries a problem through its whole solve.
//
// A team is one CTA, or one thread-block cluster whose CTAs synchronise with
// the cluster barrier and add their partial sums through distributed shared
// memory.  Phases that the graph engine separates by kernel boundaries are
// separated here by team barriers, so a small problem's iteration costs
// barriers instead of launches.  A batch is one launch: cluster teams take
// the large problems and then every CTA takes small problems by itself, both
// from work queues ordered longest first; a finished problem retires and its
// team takes the next one.
//
// Partitions.  Vector phases give float4 group v of every vector to team
// thread v mod (team threads) and the scalar tail to the next threads in
// order, the same map for every vector, so a thread rereads only what it
// wrote.  Operator terms partition their outputs otherwise (rows to lane
// groups, tiles to CTAs); a team barrier separates them from the vector
// phases.
//
// Reductions are deterministic: compensated float32 per thread, double-float
// across a warp, float64 across the warps (one warp) and across the CTAs of
// the team in rank order, so all CTAs hold the same totals and take the same
// loop decisions.  The scalar recurrences (CG step sizes, tau, kappa,
// stopping tests) run once per CTA on thread 0; float64 is never spread over
// every thread, since one SM's float64 rate is a small fraction of its
// float32 rate.
// Every loop is bounded by counters (max_iters, the CG caps, the queues); the
// batch kernel has no spin-waits.
//
// The grid team (CF_ENGINE_GRID) is the same solve with every CTA of a
// cooperative launch (one per SM) as one team: barriers are a grid-wide
// arrive/wait on a global arrival counter, and the CTAs add their partial
// sums from global memory.  The cooperative launch makes the
// runtime check that every CTA is resident, so every barrier completes; each
// wait is still bounded (kGridSpinLimit polls), after which the CTA raises an
// abort flag, every later barrier returns at once, the loops end, and the
// host reports the solve as failed.  It carries one large problem through a
// whole solve in one launch (no per-kernel launches, no graph control flow).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "devutil.cuh"
#include "fftconv.cuh"
#include "solver.cuh"

namespace cgr = cooperative_groups;

namespace cf {
namespace team {

// ------------------------------------------------------------ table entry
struct __align__(16) Prob {
  Settings st;
  Ctl* ctl;
  const Term *fwd, *adj, *adj_m;
  int32_t nfwd, nadj, nadj_m, nseg;
  int32_t lanes;     // CSR lanes per row
  int32_t do_setup;  // compute g = M^{-1} h first
  int32_t tune;      // timing run: g = 0, no setup, no outputs
  int32_t want_out, want_uv, pad0;
  int64_t n, m, z, l;
  int64_t seg_head[kMaxSeg], seg_end[kMaxSeg];
  double nb, nc;
  const float *bf, *cf;
  float *ux, *uy, *vs, *zx, *rhs, *r, *p, *q, *gx, *gy, *wy, *t, *zy, *cm, *cn, *gz, *az, *scratch;
  const double* warm;
  double *out, *uv;
  const float *eq_d, *eq_e, *eq_dinv, *eq_einv;  // equilibration (null: none)
  double sigma, rho;
};
static_assert(sizeof(Prob) % 16 == 0, "Prob is copied as 16-byte words");

// Barrier words of a grid team (zeroed before each launch).
struct GridBar {
  unsigned long long count;  // arrivals since the launch: barrier b completes at C (b + 1)
  int abort;                 // a wait gave up: every later barrier returns at once
  int pad;
};

constexpr unsigned int kGridSpinLimit = 1u << 22;  // polls (~0.5 us apart) before a wait gives up

struct Team {
  int C;     // CTAs in the team (1: this CTA alone)
  int rank;  // this CTA's rank in the team
  int tt;    // thread index in the team
  int TT;    // threads in the team
  int grid = 0;            // the team is every CTA of a cooperative launch
  GridBar* gb = nullptr;   // grid team: barrier words
  float* gpart = nullptr;  // grid team: partial sums, [2][C][32] floats
  unsigned int spin_limit = kGridSpinLimit;  // grid team: polls before a wait gives up
};

// Scalar state of a solve.  Thread 0 of every CTA of the team updates it from
// the team's sums (all CTAs hold the same sums, so they hold the same state);
// the other threads read it after the barrier that ends each sum.
struct __align__(16) Scal {
  double tau, kappa, hg, rr, tol2, pri, dual, gap, cx, by, sx, sy, ss;
  long long cg_total;
  int k, checks, refreshes, status, stop, chk, ref, go;
  int cg_it, cg_guard, cg_cont, cg_cap, cg_cap2, cg_fixed, setup_iters;
  float alpha_f, beta_f, ut_f, tau_f;
  int seg_mode[kMaxSeg];       // 0 keep, 1 zero, 2 scale onto the boundary
  float seg_head[kMaxSeg];     // projected head value (mode 2)
  float seg_scale[kMaxSeg];    // tail scale (mode 2)
};

struct __align__(16) Shared {
  Prob P;              // the problem being solved
  Scal sc;             // its scalar state
  float part[2][16];   // this CTA's partials (hi, lo pairs), double-buffered across sums
  float bh[8][32];     // block-sum scratch (double-float), one column per warp
  float bl[8][32];
  int item;            // work-queue slot taken by the team's rank 0
};

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a grid team: every write of any CTA before it is
// visible to every CTA after it.  Thread 0 of each CTA publishes the CTA's
// writes (the CTA barrier, then a fence) and adds one to the arrival count;
// the barrier its arrival belongs to completes when the count reaches the
// next multiple of C, which it polls with acquire loads, at most spin_limit
// times.  One atomic and the polls: no reset, no second word.
__device__ __noinline__ void grid_sync(const Team& tm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    GridBar* g = tm.gb;
    if (!*(volatile int*)&g->abort) {
      __threadfence();
      const unsigned long long C = (unsigned long long)tm.C;
      const unsigned long long target = (atomicAdd(&g->count, 1ull) / C + 1ull) * C;
      unsigned int k = 0;
      while (ld_acquire_gpu(&g->count) < target) {
        if (++k > tm.spin_limit || ((k & 255u) == 0u && *(volatile int*)&g->abort)) {
          atomicExch(&g->abort, 1);
          break;
        }
        if (k > 32u) __nanosleep(32);
      }
    }
  }
  __syncthreads();
}

// Whether a grid team's barrier gave up (loops end early; the solve fails).
__device__ __forceinline__ bool team_aborted(const Team& tm) {
  return tm.grid && *(volatile int*)&tm.gb->abort != 0;
}

__device__ __forceinline__ void tsync(const Team& tm) {
  if (tm.grid)
    grid_sync(tm);
  else if (tm.C > 1)
    cgr::this_cluster().sync();
  else
    __syncthreads();
}

// Vectors written during the solve are read with ordinary (L1-cached)
// loads: a barrier of the team (CTA barrier, or the cluster barrier's
// release/acquire) orders every write before it with every read after it.
__device__ __forceinline__ float4 ld4v(const float* p, int64_t v) { return reinterpret_cast<const float4*>(p)[v]; }

#define TV4(v, n) for (int64_t v = tm.tt; v < ((n) >> 2); v += tm.TT)
#define TTAIL(i, n) for (int64_t i = ((n) & ~(int64_t)3) + tm.tt; i < (n); i += tm.TT)

// f(i) for every index of [0, n) this thread owns under the vector partition.
template <class F>
__device__ __forceinline__ void each(const Team& tm, int64_t n, F&& f) {
  for (int64_t v = tm.tt; v < (n >> 2); v += tm.TT) {
    f(4 * v);
    f(4 * v + 1);
    f(4 * v + 2);
    f(4 * v + 3);
  }
  TTAIL(i, n) f(i);
}

// (hi, lo) + (hi2, lo2) in double-float: TwoSum of the heads, then the
// error and the tails, renormalised.
__device__ __forceinline__ void df_add(float& hi, float& lo, float hi2, float lo2) {
  const float s = __fadd_rn(hi, hi2);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(hi2, bb));
  const float t = __fadd_rn(__fadd_rn(lo, lo2), e);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// Team-wide deterministic sum of NV compensated per-thread sums, in
// double-float throughout (float shuffles and float arithmetic; one SM's
// float64 rate is a small fraction of its float32 rate): across each warp,
// across the warps of a CTA (warp 0), then across the CTAs of the team (lane
// j of warp 0 adds value j of every CTA's partial in rank order).  Thread 0
// of each CTA then runs fin(totals) -- the totals as float64 -- which updates
// the scalar state, and a barrier makes it visible to the CTA.
template <int NV, class F>
__device__ void team_sum(const Team& tm, Shared& sh, int& ph, Acc2 (&a)[NV], F&& fin) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float hi = a[j].hi, lo = a[j].lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
      const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
      df_add(hi, lo, h2, l2);
    }
    if (lane == 0) {
      sh.bh[j][wid] = hi;
      sh.bl[j][wid] = lo;
    }
  }
  __syncthreads();
  if (wid == 0) {
    float th[NV], tl[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      float hi = lane < nw ? sh.bh[j][lane] : 0.f, lo = lane < nw ? sh.bl[j][lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        df_add(hi, lo, h2, l2);
      }
      th[j] = hi;  // lane 0's values are the CTA's sums
      tl[j] = lo;
    }
    if (tm.grid) {
      if (lane == 0) {
        float* gp = tm.gpart + ((size_t)ph * tm.C + tm.rank) * 32;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          gp[2 * j] = th[j];
          gp[2 * j + 1] = tl[j];
        }
      }
    } else if (tm.C > 1) {
      if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          sh.part[ph][2 * j] = th[j];
          sh.part[ph][2 * j + 1] = tl[j];
        }
      }
    } else if (lane == 0) {
      double tv[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) tv[j] = (double)th[j] + (double)tl[j];
      fin(tv);
    }
  }
  if (tm.grid) {
    // every CTA adds the C partials of each value in the same order: warp j
    // takes value j, lane l the ranks l, l + 32, ..., then a fixed shuffle
    // tree; thread 0 finishes with the totals
    grid_sync(tm);
    __shared__ double gtot[16];
    if (wid < NV) {
      float hi = 0.f, lo = 0.f;
      const float* gp = tm.gpart + (size_t)ph * tm.C * 32 + 2 * wid;
      for (int r = lane; r < tm.C; r += 32) df_add(hi, lo, __ldcg(gp + (size_t)r * 32), __ldcg(gp + (size_t)r * 32 + 1));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        df_add(hi, lo, h2, l2);
      }
      if (lane == 0) gtot[wid] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tv[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) tv[j] = gtot[j];
      fin(tv);
    }
  } else if (tm.C > 1) {
    cgr::cluster_group cl = cgr::this_cluster();
    cl.sync();
    if (wid == 0) {
      float hi = 0.f, lo = 0.f;
      if (lane < NV)
        for (int r = 0; r < tm.C; ++r) {
          const float* pr = cl.map_shared_rank(&sh.part[ph][2 * lane], r);
          df_add(hi, lo, pr[0], pr[1]);
        }
      double tv[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j)
        tv[j] = (double)__shfl_sync(0xffffffffu, hi, j) + (double)__shfl_sync(0xffffffffu, lo, j);
      if (lane == 0) fin(tv);
    }
  }
  __syncthreads();
  ph ^= 1;
}

// ------------------------------------------------------------ operator terms
__device__ void term_diag(const Team& tm, const Term& t, const float* x, float* y) {
  const float* d = (const float*)t.a;
  for (int64_t i = tm.tt; i < t.rows; i += tm.TT) {
    const float xv = t.sin ? t.sin[i] * x[t.xo + i] : x[t.xo + i];
    const float a = t.sout ? t.alpha * t.sout[i] : t.alpha;
    float* yp = y + t.yo + i;
    *yp = fmaf(a, d ? __ldg(d + i) * xv : xv, t.acc ? *yp : 0.f);
  }
}

template <bool BF16>
__device__ __forceinline__ float tval(const void* __restrict__ val, int32_t k) {
  return BF16 ? __bfloat162float(__ldg(((const __nv_bfloat16*)val) + k)) : __ldg(((const float*)val) + k);
}

// CSR rows to groups of L lanes (L a power of two).  A lane takes aligned
// chunks of 8 entries of its row (the arrays are padded to whole chunks):
// two 16-byte loads of column indices and one (BF16) or two (FP32) of values
// per chunk, UC chunks issued before any is used, entries outside the row
// masked.  The input vector is staged in the CTA's shared memory when it
// fits, so the gathers never leave the SM.  The row pointers of a warp's
// next rows are loaded while it works on the current ones.
template <bool BF16, int UC>
__device__ void term_csr(const Team& tm, const Term& t, const float* x, float* y, int L, float* dsm) {
  const bool staged = t.cols <= kCsrStageFloats;
  if (staged) {
    __syncthreads();  // earlier users of the shared buffer are done
    for (int64_t i = threadIdx.x; i < t.cols; i += blockDim.x)
      dsm[i] = t.sin ? t.sin[i] * x[t.xo + i] : x[t.xo + i];
    __syncthreads();
  }
  const float* xs = staged ? dsm : x + t.xo;
  const float* sx = staged ? nullptr : t.sin;  // input scale still to apply
  const int lane = threadIdx.x & 31;
  const int rpw = 32 / L;
  const int sub = lane / L, l = lane & (L - 1);
  const int64_t warp = tm.tt >> 5, nwarps = tm.TT >> 5;
  const int64_t step = nwarps * rpw;
  const int32_t* __restrict__ rp = t.rowptr;
  const int32_t* __restrict__ col = t.col;
  const char* __restrict__ val = (const char*)t.a;
  constexpr int VB = BF16 ? 2 : 4;  // bytes per value
  int64_t r = warp * rpw + sub;
  int32_t b = r < t.rows ? __ldg(rp + r) : 0, e = r < t.rows ? __ldg(rp + r + 1) : 0;
  for (int64_t rb = warp * rpw; rb < t.rows; rb += step) {
    const int64_t rn = r + step;
    const int32_t nb = rn < t.rows ? __ldg(rp + rn) : 0, ne = rn < t.rows ? __ldg(rp + rn + 1) : 0;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int32_t k = (b & ~7) + 8 * l; k < e; k += 8 * L * UC) {
      int4 ca[UC], cb[UC];
      uint4 va[UC], vb[UC];
#pragma unroll
      for (int j = 0; j < UC; ++j) {
        const int32_t kk = k + 8 * L * j;
        if (kk < e) {
          ca[j] = ld_stream_i4(col + kk);
          cb[j] = ld_stream_i4(col + kk + 4);
          va[j] = ld_stream_u4(val + (size_t)kk * VB);
          if (!BF16) vb[j] = ld_stream_u4(val + (size_t)kk * VB + 16);
        }
      }
#pragma unroll
      for (int j = 0; j < UC; ++j) {
        const int32_t kk = k + 8 * L * j;
        if (kk < e) {
          const int32_t c8[8] = {ca[j].x, ca[j].y, ca[j].z, ca[j].w, cb[j].x, cb[j].y, cb[j].z, cb[j].w};
          float v8[8];
          if (BF16) {
            Vec<__nv_bfloat16>::unpack(va[j], v8);
          } else {
            Vec<float>::unpack(va[j], v8);
            Vec<float>::unpack(vb[j], v8 + 4);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int32_t idx = kk + u;
            if (idx >= b && idx < e) acc[u & 3] = fmaf(v8[u], sx ? sx[c8[u]] * xs[c8[u]] : xs[c8[u]], acc[u & 3]);
          }
        }
      }
    }
    float s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    for (int o = L >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0 && r < t.rows) {
      const float out = (t.sout ? t.alpha * t.sout[r] : t.alpha) * s;
      float* yp = y + t.yo + r;
      *yp = t.acc ? *yp + out : out;
    }
    r = rn;
    b = nb;
    e = ne;
  }
}

// y = alpha D x, D row-major (rows x cols, leading dimension lda): x is staged
// in each CTA's shared memory, a warp takes four rows at a time and its lanes
// read 16-byte pieces of them.
template <typename TS>
__device__ void term_dense_n(const Team& tm, const Term& t, const float* x, float* y, float* dsm) {
  constexpr int V = Vec<TS>::N;
  constexpr int RW = 4;
  const int64_t n = t.cols, m = t.rows, lda = t.lda;
  const int64_t npad = (n + 15) & ~(int64_t)15;
  __syncthreads();  // earlier users of the shared buffer are done
  for (int64_t i = threadIdx.x; i < npad; i += blockDim.x)
    dsm[i] = i < n ? (t.sin ? t.sin[i] * x[t.xo + i] : x[t.xo + i]) : 0.f;
  __syncthreads();
  const TS* A = (const TS*)t.a;
  const int lane = threadIdx.x & 31;
  const int64_t warp = tm.tt >> 5, nw = tm.TT >> 5;
  for (int64_t r0 = warp * RW; r0 < m; r0 += nw * RW) {
    float acc[RW];
#pragma unroll
    for (int rr = 0; rr < RW; ++rr) acc[rr] = 0.f;
    for (int64_t k = (int64_t)lane * V; k < n; k += 32 * V) {
      float xv[V];
#pragma unroll
      for (int q = 0; q < V; q += 4) {
        const float4 f4 = *reinterpret_cast<const float4*>(dsm + k + q);
        xv[q] = f4.x; xv[q + 1] = f4.y; xv[q + 2] = f4.z; xv[q + 3] = f4.w;
      }
      uint4 u[RW];
#pragma unroll
      for (int rr = 0; rr < RW; ++rr)
        if (r0 + rr < m) u[rr] = __ldg(reinterpret_cast<const uint4*>(A + (r0 + rr) * lda + k));
#pragma unroll
      for (int rr = 0; rr < RW; ++rr) {
        if (r0 + rr < m) {
          float f[V];
          Vec<TS>::unpack(u[rr], f);
          // padding columns (>= n) meet x = 0 and are finite (zero-filled)
#pragma unroll
          for (int q = 0; q < V; ++q) acc[rr] = fmaf(f[q], xv[q], acc[rr]);
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < RW; ++rr) {
      float s = acc[rr];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      acc[rr] = s;
    }
    if (lane < RW && r0 + lane < m) {
      float s = acc[0];
#pragma unroll
      for (int rr = 1; rr < RW; ++rr)
        if (lane == rr) s = acc[rr];
      const int64_t r = r0 + lane;
      float out = (t.sout ? t.alpha * t.sout[r] : t.alpha) * (t.scale ? __ldg(t.scale + r) * s : s);
      float* yp = y + t.yo + r;
      *yp = t.acc ? *yp + out : out;
    }
  }
}

// y = alpha D^T x: warps take (column piece, row group) items; with several
// row groups the partials go to scratch and are added in group order after a
// team barrier.
template <typename TS>
__device__ void term_dense_t(const Team& tm, const Term& t, const float* x, float* y, float* scratch) {
  constexpr int V = Vec<TS>::N;
  const int64_t nout = t.rows, nin = t.cols, lda = t.lda;
  const int64_t piece = 32 * V;
  const int64_t npc = (nout + piece - 1) / piece;
  const int64_t nw = tm.TT >> 5, warp = tm.tt >> 5;
  int64_t R = nw / npc;
  R = R < 1 ? 1 : (R > kDenseTGroups ? kDenseTGroups : R);
  if (R > 1) tsync(tm);  // an earlier term's readers of the scratch are done
  const TS* A = (const TS*)t.a;
  const int lane = threadIdx.x & 31;
  for (int64_t it = warp; it < npc * R; it += nw) {
    const int64_t c = it % npc, g = it / npc;
    const int64_t r0 = g * nin / R, r1 = (g + 1) * nin / R;
    const int64_t col0 = c * piece + (int64_t)lane * V;
    float acc[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = 0.f;
    if (col0 < nout) {
      int64_t i = r0;
      for (; i + 4 <= r1; i += 4) {
        uint4 u[4];
        float xi[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          u[j] = __ldg(reinterpret_cast<const uint4*>(A + (i + j) * lda + col0));
          xi[j] = x[t.xo + i + j];
          if (t.scale) xi[j] *= __ldg(t.scale + i + j);
          if (t.sin) xi[j] *= t.sin[i + j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float f[V];
          Vec<TS>::unpack(u[j], f);
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] = fmaf(xi[j], f[q], acc[q]);
        }
      }
      for (; i < r1; ++i) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(A + i * lda + col0));
        float xi = x[t.xo + i];
        if (t.scale) xi *= __ldg(t.scale + i);
        if (t.sin) xi *= t.sin[i];
        float f[V];
        Vec<TS>::unpack(u, f);
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] = fmaf(xi, f[q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int64_t j = col0 + q;
        if (j < nout) {
          if (R == 1) {
            float* yp = y + t.yo + j;
            const float out = (t.sout ? t.alpha * t.sout[j] : t.alpha) * acc[q];
            *yp = t.acc ? *yp + out : out;
          } else {
            scratch[g * nout + j] = acc[q];
          }
        }
      }
    }
  }
  if (R > 1) {
    tsync(tm);
    for (int64_t j = tm.tt; j < nout; j += tm.TT) {
      float s = 0.f;
      for (int64_t g = 0; g < R; ++g) s += scratch[g * nout + j];
      float* yp = y + t.yo + j;
      const float out = (t.sout ? t.alpha * t.sout[j] : t.alpha) * s;
      *yp = t.acc ? *yp + out : out;
    }
  }
}

// out[i] = sum_{j < Lp} wrev[j] x[i + shift - (Lp - 1) + j] (x = 0 outside
// [0, cols)): output tiles go to the team's CTAs in turn; each tile's input
// window and the taps sit in shared memory, and a thread computes kConvR
// consecutive outputs from a register window of 2 kConvR inputs, so that
// every 8 taps cost 6 shared-memory loads for 64 multiply-adds.
constexpr int kConvR = 8;

__device__ void term_conv(const Team& tm, const Term& t, const float* x, float* y, float* dsm) {
  const int64_t n_out = t.rows, n_in = t.cols, Lp = t.Lp;
  float* w_s = dsm;
  float* in_s = dsm + Lp;  // 64-byte aligned: Lp is a multiple of 16
  __syncthreads();  // earlier users of the shared buffer are done
  for (int64_t j = threadIdx.x; j < Lp; j += blockDim.x) w_s[j] = __ldg((const float*)t.a + j);
  const int64_t ntile = (n_out + kConvTile - 1) / kConvTile;
  for (int64_t tile = tm.rank; tile < ntile; tile += tm.C) {
    const int64_t o0 = tile * kConvTile;
    const int64_t cnt = (n_out - o0) < kConvTile ? (n_out - o0) : (int64_t)kConvTile;
    const int64_t base = o0 + t.shift - (Lp - 1);
    __syncthreads();
    // window [0, cnt + Lp + kConvR): the last register window of the last
    // thread reaches index (cnt - 1) + Lp + kConvR - 2 at most
    for (int64_t j = threadIdx.x; j < cnt + Lp + kConvR; j += blockDim.x) {
      const int64_t g = base + j;
      in_s[j] = (g >= 0 && g < n_in) ? (t.sin ? t.sin[g] * x[t.xo + g] : x[t.xo + g]) : 0.f;
    }
    __syncthreads();
    const float4* w4 = reinterpret_cast<const float4*>(w_s);
    for (int64_t ob = (int64_t)threadIdx.x * kConvR; ob < cnt; ob += (int64_t)blockDim.x * kConvR) {
      float acc[kConvR];
#pragma unroll
      for (int r = 0; r < kConvR; ++r) acc[r] = 0.f;
      const float4* x4 = reinterpret_cast<const float4*>(in_s + ob);
      for (int64_t j = 0; j < Lp; j += 8) {
        float xw[16], w[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 v = x4[(j >> 2) + q];
          xw[4 * q] = v.x; xw[4 * q + 1] = v.y; xw[4 * q + 2] = v.z; xw[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float4 v = w4[(j >> 2) + q];
          w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
#pragma unroll
          for (int r = 0; r < kConvR; ++r) acc[r] = fmaf(w[jj], xw[r + jj], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < kConvR; ++r) {
        if (ob + r < cnt) {
          const float out = (t.sout ? t.alpha * t.sout[o0 + ob + r] : t.alpha) * acc[r];
          float* yp = y + t.yo + o0 + ob + r;
          *yp = t.acc ? *yp + out : out;
        }
      }
    }
  }
}

// The 1-D convolution by overlap-save FFTs (fftconv.cuh): each N/16 threads
// of a CTA take pairs of segments in turn (pair g + groups x rank, + groups x
// C), with a transform buffer of their own in the CTA's shared memory and a
// named barrier of their own.  The input was written by other CTAs before a
// team barrier, so it is read through L2 (no read-only path).
__device__ __forceinline__ void group_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int N, bool SC>
__device__ __noinline__ void term_fft(const Team& tm, const Term& t, const float* x, float* y, float* dsm) {
  constexpr int T = N / 16;
  const int ng = blockDim.x / T, g = threadIdx.x / T, tl = threadIdx.x % T;
  const int Lp = (int)t.Lp;
  const int64_t V = N - Lp + 1;
  const int64_t npairs = (t.rows + 2 * V - 1) / (2 * V);
  const int64_t D = Lp - 1 - t.shift;
  float2* buf = reinterpret_cast<float2*>(dsm) + (size_t)g * fftc::buf_f2<N>();
  __syncthreads();  // earlier users of the shared buffer are done
  for (int64_t pr = (int64_t)tm.rank * ng + g; pr < npairs; pr += (int64_t)tm.C * ng)
    fftc::pair<N, SC, false, false>(tl, pr, t.rows, t.cols, Lp, D, static_cast<const float2*>(t.a), t.tw, t.alpha,
                                    x + t.xo, y + t.yo, t.acc != 0, t.sin, t.sout, buf, nullptr, nullptr,
                                    [g] { group_bar(1 + g, T); });
}

// y = the flattened operator applied to x (terms in order).  Compiled once
// per CTA size (not inlined at each call) so that the term loops get
// registers of their own; with 64 registers a thread (1024 threads on an SM)
// a lane keeps one CSR chunk (8 entries) in flight, with 128 or more two.
template <int MaxT, int MinB>
__device__ __noinline__ void apply(const Team& tm, const Term* terms, int nt, const float* x, float* y,
                                   float* scratch, float* dsm, int lanes) {
  constexpr int UC = 65536 / (MaxT * MinB) >= 128 ? 2 : 1;  // CSR chunks in flight per lane
  for (int k = 0; k < nt; ++k) {
    const Term& t = terms[k];
    if (t.sync) tsync(tm);
    switch (t.kind) {
      case T_FILL:
        for (int64_t i = tm.tt; i < t.rows; i += tm.TT) y[t.yo + i] = 0.f;
        break;
      case T_DIAG:
        term_diag(tm, t, x, y);
        break;
      case T_CSR:
        if (t.prec == CF_BF16)
          term_csr<true, UC>(tm, t, x, y, lanes, dsm);
        else
          term_csr<false, UC>(tm, t, x, y, lanes, dsm);
        break;
      case T_DENSE_N:
        if (t.prec == CF_BF16)
          term_dense_n<__nv_bfloat16>(tm, t, x, y, dsm);
        else if (t.prec == CF_FP8_E4M3)
          term_dense_n<__nv_fp8_e4m3>(tm, t, x, y, dsm);
        else
          term_dense_n<float>(tm, t, x, y, dsm);
        break;
      case T_DENSE_T:
        if (t.prec == CF_BF16)
          term_dense_t<__nv_bfloat16>(tm, t, x, y, scratch);
        else if (t.prec == CF_FP8_E4M3)
          term_dense_t<__nv_fp8_e4m3>(tm, t, x, y, scratch);
        else
          term_dense_t<float>(tm, t, x, y, scratch);
        break;
      case T_CONV:
        term_conv(tm, t, x, y, dsm);
        break;
      case T_FFT:
        if (t.fftn == 2048) {
          if (t.sin)
            term_fft<2048, true>(tm, t, x, y, dsm);
          else
            term_fft<2048, false>(tm, t, x, y, dsm);
        } else {
          if (t.sin)
            term_fft<4096, true>(tm, t, x, y, dsm);
          else
            term_fft<4096, false>(tm, t, x, y, dsm);
        }
        break;
    }
  }
}

// ------------------------------------------------------------ CG (Section 4.2)
// CG on (I + A^T A) z = rhs from the z held, with gz = G z carried (setup
// starts at z = 0; iterations warm-start with the carried G z).  mode
// CG_ITER also carries az = A z.  k_outer: the ADMM iteration (tolerance).
template <int MaxT, int MinB>
__device__ __noinline__ void cg_run(const Team& tm, Shared& sh, int& ph, float* dsm, int mode, float* z,
                                    int k_outer) {
  const Prob& P = sh.P;
  const int64_t n = P.n, m = P.m;
  float *r = P.r, *p = P.p, *q = P.q, *gz = P.gz, *az = P.az, *t = P.t;
  const float* rhs = P.rhs;
  {
    Acc2 a[2];
    TV4(v, n) {
      const float4 g = ld4v(gz, v), rh = ld4v(rhs, v);
      float4 rv;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        el(rv, k) = elc(rh, k) - elc(g, k);
        a[0].add_prod(elc(rv, k), elc(rv, k));
        a[1].add_prod(elc(rh, k), elc(rh, k));
      }
      st4(r, v, rv);
      st4(p, v, rv);
    }
    TTAIL(i, n) {
      const float rh = rhs[i];
      const float ri = rh - gz[i];
      r[i] = ri;
      p[i] = ri;
      a[0].add_prod(ri, ri);
      a[1].add_prod(rh, rh);
    }
    team_sum<2>(tm, sh, ph, a, [&](const double* tv) {
      Scal& c = sh.sc;
      const Settings& st = sh.P.st;
      const double nrhs = sqrt(tv[1]);
      double tol;
      if (mode == CG_SETUP) {
        tol = st.setup_tol * nrhs;
        c.cg_cap = st.setup_cg_max;
        c.cg_fixed = 0;
      } else {
        tol = st.cg_tol_rel * nrhs * (double)powf((float)k_outer + 1.0f, -(float)st.cg_tol_exp);
        tol = fmax(tol, st.cg_tol_min);
        c.cg_cap = st.cg_max;
        c.cg_fixed = st.cg_fixed;
      }
      c.rr = tv[0];
      c.tol2 = tol * tol;
      c.cg_it = 0;
      c.cg_guard = 0;
      c.cg_cap2 = mode == CG_SETUP ? st.setup_cg_max : (st.cg_fixed > 0 ? st.cg_fixed : st.cg_max);
      c.cg_cont = c.cg_fixed > 0 ? 1 : ((c.rr > c.tol2 && c.cg_cap > 0) ? 1 : 0);
    });
  }
  bool cont = sh.sc.cg_cont != 0;
  while (cont && !team_aborted(tm)) {
    // p (vector partition, followed by a sum or a barrier) -> t = A p -> q = A^T t
    apply<MaxT, MinB>(tm, P.fwd, P.nfwd, p, t, P.scratch, dsm, P.lanes);
    tsync(tm);
    apply<MaxT, MinB>(tm, P.adj, P.nadj, t, q, P.scratch, dsm, P.lanes);
    tsync(tm);
    {
      Acc2 b[1];
      TV4(v, n) {
        const float4 pp = ld4v(p, v);
        float4 qq = ld4v(q, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          el(qq, k) = el(qq, k) + elc(pp, k);  // q += lam p, lam = 1
          b[0].add_prod(elc(pp, k), elc(qq, k));
        }
        st4(q, v, qq);
      }
      TTAIL(i, n) {
        const float pi = p[i];
        const float qi = q[i] + pi;
        q[i] = qi;
        b[0].add_prod(pi, qi);
      }
      team_sum<1>(tm, sh, ph, b, [&](const double* tv) {
        // the step length is a float32 quantity; float64 stays in the CG test
        const float pq = (float)tv[0];
        sh.sc.alpha_f = pq > 0.f ? (float)sh.sc.rr / pq : 0.f;
      });
    }
    const float a = sh.sc.alpha_f;
    {
      Acc2 c0[1];
      TV4(v, n) {
        const float4 qq = ld4v(q, v), pp = ld4v(p, v);
        float4 zz = ld4v(z, v), gg = ld4v(gz, v), rv = ld4v(r, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          el(zz, k) = fmaf(a, elc(pp, k), el(zz, k));
          el(gg, k) = fmaf(a, elc(qq, k), el(gg, k));
          el(rv, k) = fmaf(-a, elc(qq, k), el(rv, k));
          c0[0].add_prod(elc(rv, k), elc(rv, k));
        }
        st4(z, v, zz);
        st4(gz, v, gg);
        st4(r, v, rv);
      }
      TTAIL(i, n) {
        const float qi = q[i];
        z[i] = fmaf(a, p[i], z[i]);
        gz[i] = fmaf(a, qi, gz[i]);
        const float ri = fmaf(-a, qi, r[i]);
        r[i] = ri;
        c0[0].add_prod(ri, ri);
      }
      if (mode == CG_ITER) {
        TV4(v, m) {
          const float4 tv = ld4v(t, v);
          float4 aa = ld4v(az, v);
#pragma unroll
          for (int k = 0; k < 4; ++k) el(aa, k) = fmaf(a, elc(tv, k), el(aa, k));
          st4(az, v, aa);
        }
        TTAIL(i, m) az[i] = fmaf(a, t[i], az[i]);
      }
      team_sum<1>(tm, sh, ph, c0, [&](const double* tv) {
        Scal& c = sh.sc;
        const double rr_new = tv[0];
        c.beta_f = c.rr > 0.0 ? (float)rr_new / (float)c.rr : 0.f;
        c.rr = rr_new;
        ++c.cg_it;
        if (mode == CG_SETUP)
          ++c.setup_iters;
        else
          ++c.cg_total;
        const bool more = c.cg_fixed > 0 ? (c.cg_it < c.cg_fixed) : (rr_new > c.tol2 && c.cg_it < c.cg_cap);
        ++c.cg_guard;
        c.cg_cont = (more && c.cg_guard < c.cg_cap2) ? 1 : 0;
      });
    }
    const float b = sh.sc.beta_f;
    cont = sh.sc.cg_cont != 0;
    TV4(v, n) {
      const float4 rv = ld4v(r, v);
      float4 pp = ld4v(p, v);
#pragma unroll
      for (int k = 0; k < 4; ++k) el(pp, k) = fmaf(b, el(pp, k), elc(rv, k));
      st4(p, v, pp);
    }
    TTAIL(i, n) p[i] = fmaf(b, p[i], r[i]);
    if (cont) tsync(tm);  // the next forward term reads p under its own partition
  }
}

// ------------------------------------------------------------ one solve
__device__ __forceinline__ int seg_of(const Prob& P, int64_t i) {
  int s = 0;
  while (s + 1 < P.nseg && i >= P.seg_end[s]) ++s;
  return s;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Head value p0 and tail norm of each of the NS second-order cone blocks of
// the point to project; the projection constants of each block (float32:
// the projection is a float32 step) go to the scalar state.
template <int NS>
__device__ void soc_norms(const Team& tm, Shared& sh, int& ph, float af, float a1, float utf) {
  const Prob& P = sh.P;
  const int64_t nl = P.z + P.l;
  Acc2 acc[2 * NS];
  each(tm, P.m, [&](int64_t i) {
    if (i < nl) return;
    const float pi = y_pre(af, a1, utf, P.zy[i], P.gy[i], P.uy[i], P.vs[i]);
    const int s = seg_of(P, i);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      if (j == s) {
        if (i == P.seg_head[j])
          acc[2 * j].add(pi);
        else
          acc[2 * j + 1].add_prod(pi, pi);
      }
    }
  });
  team_sum<2 * NS>(tm, sh, ph, acc, [&](const double* tv) {
    Scal& c = sh.sc;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const float p0 = (float)tv[2 * j], nrm = sqrtf((float)tv[2 * j + 1]);
      const float ah = 0.5f * (p0 + nrm);
      c.seg_mode[j] = nrm <= p0 ? 0 : (nrm <= -p0 ? 1 : 2);
      c.seg_head[j] = ah;
      c.seg_scale[j] = c.seg_mode[j] == 2 ? ah / nrm : 0.f;
    }
  });
}

template <int MaxT, int MinB>
__device__ void solve_one(const Team& tm, Shared& sh, float* dsm) {
  const unsigned long long t_start = gtimer();
  const Prob& P = sh.P;
  const Settings& st = P.st;
  const int64_t n = P.n, m = P.m, N = n + m + 1;
  int ph = 0;
  const bool warm = st.warm != 0 && !P.tune;
  if (threadIdx.x == 0) {
    Scal& c = sh.sc;
    c.cg_total = 0;
    c.k = c.checks = c.refreshes = 0;
    c.status = CF_MAX_ITERS;
    c.stop = 0;
    c.pri = c.dual = c.gap = INFINITY;
    c.cx = c.by = 0.0;
    c.setup_iters = 0;
    c.hg = P.tune ? 0.0 : (P.do_setup ? 0.0 : P.ctl->hg);
    c.tau = warm ? P.warm[n + m] : 1.0;
    c.kappa = warm ? P.warm[N + n + m] : 1.0;
  }
  __syncthreads();

  // ---- setup: g = M^{-1} h, h^T g
  if (P.tune) {
    each(tm, n, [&](int64_t i) { P.gx[i] = 0.f; });
    each(tm, m, [&](int64_t i) { P.gy[i] = 0.f; });
  } else if (P.do_setup) {
    each(tm, n, [&](int64_t i) {
      P.gx[i] = 0.f;
      P.gz[i] = 0.f;
      P.rhs[i] = __ldg(P.cf + i);
    });
    tsync(tm);
    apply<MaxT, MinB>(tm, P.adj_m, P.nadj_m, P.bf, P.rhs, P.scratch, dsm, P.lanes);  // rhs = c - A^T b
    tsync(tm);
    cg_run<MaxT, MinB>(tm, sh, ph, dsm, CG_SETUP, P.gx, 0);
    tsync(tm);
    apply<MaxT, MinB>(tm, P.fwd, P.nfwd, P.gx, P.gy, P.scratch, dsm, P.lanes);  // A g_x
    tsync(tm);
    Acc2 a[1];
    each(tm, m, [&](int64_t i) {
      const float bi = __ldg(P.bf + i);
      const float gi = P.gy[i] + bi;
      P.gy[i] = gi;
      a[0].add_prod(bi, gi);
    });
    each(tm, n, [&](int64_t i) { a[0].add_prod(__ldg(P.cf + i), P.gx[i]); });
    team_sum<1>(tm, sh, ph, a, [&](const double* tv) { sh.sc.hg = tv[0]; });
  }

  // ---- initial point u = v = (0, 0, 1) or the warm start
  each(tm, n, [&](int64_t i) {
    P.ux[i] = warm ? (float)P.warm[i] : 0.f;
    P.zx[i] = 0.f;
    P.gz[i] = 0.f;
  });
  each(tm, m, [&](int64_t i) {
    P.uy[i] = warm ? (float)P.warm[n + i] : 0.f;
    P.vs[i] = warm ? (float)P.warm[N + n + i] : 0.f;
    P.az[i] = 0.f;
  });
  const double al = st.alpha;
  const float af = (float)al, a1 = (float)(1.0 - al);
  const int64_t z = P.z, nl = P.z + P.l;

  for (int guard = 0; guard < st.max_iters && !team_aborted(tm); ++guard) {
    // ---- w = u + v; rhs = w_x - A^T w_y
    TV4(v, m) {
      const float4 a = ld4v(P.uy, v), b = ld4v(P.vs, v);
      st4(P.wy, v, make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w));
    }
    TTAIL(i, m) P.wy[i] = P.uy[i] + P.vs[i];
    TV4(v, n) st4(P.rhs, v, ld4v(P.ux, v));
    TTAIL(i, n) P.rhs[i] = P.ux[i];
    tsync(tm);
    apply<MaxT, MinB>(tm, P.adj_m, P.nadj_m, P.wy, P.rhs, P.scratch, dsm, P.lanes);
    tsync(tm);
    // ---- z_x by CG, warm-started at the previous z_x
    cg_run<MaxT, MinB>(tm, sh, ph, dsm, CG_ITER, P.zx, sh.sc.k);
    // ---- z_y = w_y + A z_x (carried); u~_tau; then tau, kappa, the
    // iteration counter and this iteration's decisions
    {
      Acc2 a[1];
      TV4(v, m) {
        const float4 aa = ld4v(P.az, v), ww = ld4v(P.wy, v), bb = __ldg(reinterpret_cast<const float4*>(P.bf) + v);
        float4 zz;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          el(zz, j) = elc(aa, j) + elc(ww, j);
          a[0].add_prod(elc(bb, j), elc(zz, j));
        }
        st4(P.zy, v, zz);
      }
      TTAIL(i, m) {
        const float zi = P.az[i] + P.wy[i];
        P.zy[i] = zi;
        a[0].add_prod(__ldg(P.bf + i), zi);
      }
      TV4(v, n) {
        const float4 cc = __ldg(reinterpret_cast<const float4*>(P.cf) + v), xx = ld4v(P.zx, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) a[0].add_prod(elc(cc, j), elc(xx, j));
      }
      TTAIL(i, n) a[0].add_prod(__ldg(P.cf + i), P.zx[i]);
      team_sum<1>(tm, sh, ph, a, [&](const double* tv) {
        Scal& c = sh.sc;
        const Settings& s = sh.P.st;
        const double ut = (c.tau + c.kappa + tv[0]) / (1.0 + c.hg);  // w_tau = tau + kappa
        c.ut_f = (float)ut;
        const double uhat = s.alpha * ut + (1.0 - s.alpha) * c.tau;
        const double pt = uhat - c.kappa;
        const double tn = pt > 0.0 ? pt : 0.0;
        c.tau = tn;
        c.kappa = tn - pt;
        c.tau_f = (float)tn;
        const int k = ++c.k;
        c.chk = ((k % s.check_interval == 0) || (k >= s.max_iters)) ? 1 : 0;
        c.ref = ((k % 50 == 0) && (k < s.max_iters)) ? 1 : 0;
        if (!isfinite(c.tau) || !isfinite(c.kappa)) {
          c.status = CF_NUMERICAL;
          c.stop = 1;
        }
        c.go = (!c.stop && k < s.max_iters) ? 1 : 0;
      });
    }
    const float utf = sh.sc.ut_f;
    // ---- second-order cones: head value and tail norm of each block
    switch (P.nseg) {
      case 1: soc_norms<1>(tm, sh, ph, af, a1, utf); break;
      case 2: soc_norms<2>(tm, sh, ph, af, a1, utf); break;
      case 3: soc_norms<3>(tm, sh, ph, af, a1, utf); break;
      case 4: soc_norms<4>(tm, sh, ph, af, a1, utf); break;
      default: break;
    }
    // ---- projection onto C and dual update (u+ = Pi(u_hat - v), v+ = v - u_hat + u+)
    TV4(v, n) {
      const float4 zz = ld4v(P.zx, v), gg = ld4v(P.gx, v);
      float4 uu = ld4v(P.ux, v);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        el(uu, j) = __fadd_rn(__fmul_rn(af, __fsub_rn(elc(zz, j), __fmul_rn(utf, elc(gg, j)))),
                              __fmul_rn(a1, el(uu, j)));
      st4(P.ux, v, uu);
    }
    TTAIL(i, n) P.ux[i] = __fadd_rn(__fmul_rn(af, __fsub_rn(P.zx[i], __fmul_rn(utf, P.gx[i]))),
                                    __fmul_rn(a1, P.ux[i]));
    each(tm, m, [&](int64_t i) {
      const float pi = y_pre(af, a1, utf, P.zy[i], P.gy[i], P.uy[i], P.vs[i]);
      float ui;
      if (i < z) {
        ui = pi;
      } else if (i < nl) {
        ui = fmaxf(pi, 0.f);
      } else {
        const int s = seg_of(P, i);
        const int md = sh.sc.seg_mode[s];
        ui = md == 0 ? pi : (md == 1 ? 0.f : (i == P.seg_head[s] ? sh.sc.seg_head[s] : __fmul_rn(sh.sc.seg_scale[s], pi)));
      }
      P.uy[i] = ui;
      P.vs[i] = __fsub_rn(ui, pi);
    });
    const bool chk = sh.sc.chk != 0, ref = sh.sc.ref != 0;
    bool go = sh.sc.go != 0;
    // ---- residuals and certificates
    if (chk && !sh.sc.stop) {
      tsync(tm);
      apply<MaxT, MinB>(tm, P.fwd, P.nfwd, P.ux, P.cm, P.scratch, dsm, P.lanes);
      apply<MaxT, MinB>(tm, P.adj, P.nadj, P.uy, P.cn, P.scratch, dsm, P.lanes);
      tsync(tm);
      // sums of k_resid (solver.cu): weighted by 1/D, 1/E when equilibrated
      const float tf = sh.sc.tau_f;
      Acc2 s[6];
      each(tm, m, [&](int64_t i) {
        const float bi = __ldg(P.bf + i);
        const float w = P.eq_dinv ? P.eq_dinv[i] : 1.f;
        const float e = P.cm[i] + P.vs[i];
        const float d = w * fmaf(-bi, tf, e);
        const float we = w * e;
        s[0].add_prod(d, d);
        s[1].add_prod(we, we);
        s[2].add_prod(bi, P.uy[i]);
      });
      each(tm, n, [&](int64_t i) {
        const float ci = __ldg(P.cf + i), cn = P.cn[i];
        const float w = P.eq_einv ? P.eq_einv[i] : 1.f;
        const float d = w * fmaf(ci, tf, cn);
        const float wc = w * cn;
        s[3].add_prod(d, d);
        s[4].add_prod(wc, wc);
        s[5].add_prod(ci, P.ux[i]);
      });
      team_sum<6>(tm, sh, ph, s, [&](const double* v) {
        Scal& c = sh.sc;
        const Settings& st2 = sh.P.st;
        const double tau = c.tau, sig = sh.P.sigma, rho = sh.P.rho;
        ++c.checks;
        c.cx = v[5] / (rho * sig);
        c.by = v[2] / (rho * sig);
        bool bad = false;
        for (int j = 0; j < 6; ++j) bad |= !isfinite(v[j]);
        if (bad) {
          c.status = CF_NUMERICAL;
          c.stop = 1;
        } else {
          if (tau > 0.0) {
            c.pri = sqrt(v[0]) / (sig * tau) / (1.0 + sh.P.nb);
            c.dual = sqrt(v[3]) / (rho * tau) / (1.0 + sh.P.nc);
            const double cxt = c.cx / tau, byt = c.by / tau;
            c.gap = fabs(cxt + byt) / (1.0 + fabs(cxt) + fabs(byt));
            if (c.pri <= st2.eps && c.dual <= st2.eps && c.gap <= st2.eps) {
              c.status = CF_SOLVED;
              c.stop = 1;
            }
          }
          if (!c.stop) {
            if (-v[2] > 0.0 && sig * sqrt(v[4]) <= st2.eps_inf * (-v[2])) {
              c.status = CF_INFEASIBLE;
              c.stop = 1;
            } else if (-v[5] > 0.0 && rho * sqrt(v[1]) <= st2.eps_inf * (-v[5])) {
              c.status = CF_UNBOUNDED;
              c.stop = 1;
            }
          }
        }
        c.go = (!c.stop && c.k < st2.max_iters) ? 1 : 0;
      });
      go = sh.sc.go != 0;
    }
    if (!go) break;
    // ---- exact A z_x and G z_x every 50 iterations
    if (ref) {
      if (threadIdx.x == 0) ++sh.sc.refreshes;
      tsync(tm);
      apply<MaxT, MinB>(tm, P.fwd, P.nfwd, P.zx, P.az, P.scratch, dsm, P.lanes);
      tsync(tm);
      apply<MaxT, MinB>(tm, P.adj, P.nadj, P.az, P.gz, P.scratch, dsm, P.lanes);
      tsync(tm);
      each(tm, n, [&](int64_t i) { P.gz[i] = P.zx[i] + P.gz[i]; });  // G z = lam z + A^T A z, lam = 1
    }
  }

  // ---- outputs
  if (threadIdx.x == 0) {
    Scal& c = sh.sc;
    if (c.status == CF_INFEASIBLE) {
      c.sx = NAN; c.ss = NAN; c.sy = 1.0 / (-c.by);
    } else if (c.status == CF_UNBOUNDED) {
      c.sx = 1.0 / (-c.cx); c.ss = c.sx; c.sy = NAN;
    } else if (c.tau > 0.0) {
      c.sx = c.sy = c.ss = 1.0 / c.tau;
    } else {
      c.sx = c.sy = c.ss = NAN;
    }
  }
  __syncthreads();
  if (!P.tune) {
    if (P.want_out) {
      // the original problem's point (see k_output in solver.cu)
      const double sx = sh.sc.sx / P.sigma, sy = sh.sc.sy / P.rho, ss = sh.sc.ss / P.sigma;
      each(tm, n, [&](int64_t i) { P.out[i] = (double)P.ux[i] * (P.eq_e ? (double)P.eq_e[i] : 1.0) * sx; });
      each(tm, m, [&](int64_t i) {
        P.out[n + i] = (double)P.uy[i] * (P.eq_d ? (double)P.eq_d[i] : 1.0) * sy;
        P.out[n + m + i] = (double)P.vs[i] * (P.eq_dinv ? (double)P.eq_dinv[i] : 1.0) * ss;
      });
    }
    if (P.want_uv) {
      each(tm, n, [&](int64_t i) {
        P.uv[i] = P.ux[i];
        P.uv[N + i] = 0.0;
      });
      each(tm, m, [&](int64_t i) {
        P.uv[n + i] = P.uy[i];
        P.uv[N + n + i] = P.vs[i];
      });
      if (tm.tt == 0) {
        P.uv[n + m] = sh.sc.tau;
        P.uv[N + n + m] = sh.sc.kappa;
      }
    }
  }
  if (tm.tt == 0) {
    const Scal& s = sh.sc;
    Ctl* c = P.ctl;
    c->lam = 1.0;
    c->hg = s.hg;
    c->tau = s.tau;
    c->kappa = s.kappa;
    c->pri = s.pri;
    c->dual = s.dual;
    c->gap = s.gap;
    c->cx = s.cx;
    c->by = s.by;
    c->cg_total = s.cg_total;
    c->k = s.k;
    c->checks = s.checks;
    c->refreshes = s.refreshes;
    c->status = s.status;
    c->stop = 1;
    c->grid_abort = team_aborted(tm) ? 1 : 0;
    if (P.do_setup && !P.tune) c->setup_iters = s.setup_iters;
    c->t_start = (long long)t_start;
    c->t_end = (long long)gtimer();
  }
}

__device__ void load_prob(Shared& sh, const Prob* src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&sh.P);
  for (int i = threadIdx.x; i < (int)(sizeof(Prob) / 16); i += blockDim.x) d[i] = __ldg(s + i);
  __syncthreads();
}

// Persistent kernel: cluster teams take problems order[0, nbig), then every
// CTA takes problems order[nbig, nbig + nsmall) alone.
template <int MaxT, int MinB>
__global__ void __launch_bounds__(MaxT, MinB) k_team(const Prob* __restrict__ probs, const int32_t* __restrict__ order,
                                               int32_t nbig, int32_t nsmall, unsigned int* counters,
                                               int32_t cluster) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ Shared sh;
  Team tm;
  if (cluster > 1) {
    cgr::cluster_group cl = cgr::this_cluster();
    tm.C = cluster;
    tm.rank = (int)cl.block_rank();
    tm.TT = cluster * (int)blockDim.x;
    tm.tt = tm.rank * (int)blockDim.x + (int)threadIdx.x;
    for (;;) {
      if (tm.rank == 0 && threadIdx.x == 0) sh.item = (int)atomicAdd(&counters[0], 1u);
      cl.sync();
      const int it = *cl.map_shared_rank(&sh.item, 0);
      cl.sync();
      if (it >= nbig) break;
      load_prob(sh, probs + order[it]);
      solve_one<MaxT, MinB>(tm, sh, dsm);
    }
  }
  tm.C = 1;
  tm.rank = 0;
  tm.TT = (int)blockDim.x;
  tm.tt = (int)threadIdx.x;
  for (;;) {
    if (threadIdx.x == 0) sh.item = (int)atomicAdd(&counters[1], 1u);
    __syncthreads();
    const int it = sh.item;
    __syncthreads();
    if (it >= nsmall) break;
    load_prob(sh, probs + order[nbig + it]);
    solve_one<MaxT, MinB>(tm, sh, dsm);
  }
}

// Grid team: every CTA of this cooperative launch carries the one problem.
template <int MaxT, int MinB>
__global__ void __launch_bounds__(MaxT, MinB) k_team_grid(const Prob* __restrict__ prob, GridBar* gb,
                                                        float* gpart, unsigned int spin_limit) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ Shared sh;
  Team tm;
  tm.grid = 1;
  tm.gb = gb;
  tm.gpart = gpart;
  tm.spin_limit = spin_limit;
  tm.C = (int)gridDim.x;
  tm.rank = (int)blockIdx.x;
  tm.TT = (int)(gridDim.x * blockDim.x);
  tm.tt = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  load_prob(sh, prob);
  solve_one<MaxT, MinB>(tm, sh, dsm);
}

// ------------------------------------------------------------ host: planning
namespace {

int64_t out_len(const cf_op* op, bool trans) { return trans ? op->n : op->m; }

// Mirrors op_apply_rec (ops.cu): the same walk, emitting terms instead of
// launches.
bool flatten(const cf_op* op, bool trans, float alpha, int64_t xo, int64_t yo, bool acc,
             std::vector<Term>& out, std::string* why) {
  Term t{};
  t.alpha = alpha;
  t.acc = acc ? 1 : 0;
  t.xo = xo;
  t.yo = yo;
  switch (op->kind) {
    case OP_ZERO:
      if (!acc) {
        t.kind = T_FILL;
        t.rows = out_len(op, trans);
        out.push_back(t);
      }
      return true;
    case OP_DIAG:
      t.kind = T_DIAG;
      t.rows = t.cols = op->n;
      t.a = op->d;
      out.push_back(t);
      return true;
    case OP_DENSE:
      if (!trans && op->n > kDenseMaxCols) {
        *why = "dense leaf wider than " + std::to_string(kDenseMaxCols) + " columns";
        return false;
      }
      t.kind = trans ? T_DENSE_T : T_DENSE_N;
      t.prec = op->prec;
      t.rows = trans ? op->n : op->m;
      t.cols = trans ? op->m : op->n;
      t.a = op->a;
      t.scale = op->row_scale;
      t.lda = op->lda;
      out.push_back(t);
      return true;
    case OP_CSR:
      t.kind = T_CSR;
      t.prec = op->prec;
      t.rows = trans ? op->n : op->m;
      t.cols = trans ? op->m : op->n;
      t.rowptr = trans ? op->t_rowptr : op->rowptr;
      t.col = trans ? op->t_col : op->col;
      t.a = trans ? op->t_val : op->val;
      out.push_back(t);
      return true;
    case OP_CONV1D:
      if (op->fft_tw) {  // the leaf is evaluated by overlap-save FFTs
        t.kind = T_FFT;
        t.rows = trans ? op->n : op->m;
        t.cols = trans ? op->m : op->n;
        t.Lp = op->Lp;
        t.shift = trans ? op->Lp - 1 : 0;
        t.a = trans ? op->fft_ha : op->fft_hf;
        t.tw = op->fft_tw;
        t.fftn = op->fft_n;
        out.push_back(t);
        return true;
      }
      if (op->Lp > kConvMaxLp) {
        *why = "convolution longer than " + std::to_string(kConvMaxLp) + " taps";
        return false;
      }
      t.kind = T_CONV;
      t.rows = trans ? op->n : op->m;
      t.cols = trans ? op->m : op->n;
      t.Lp = op->Lp;
      t.shift = trans ? op->Lp - 1 : 0;
      t.a = trans ? op->w_adj : op->w_fwd;
      out.push_back(t);
      return true;
    case OP_CONV2D:
      *why = "2-D convolution leaf";
      return false;
    case OP_SCALE:
      return flatten(op->parts[0], trans, (float)(alpha * op->alpha), xo, yo, acc, out, why);
    case OP_ADJOINT:
      return flatten(op->parts[0], !trans, alpha, xo, yo, acc, out, why);
    case OP_VSTACK:
    case OP_HSTACK: {
      const bool split_out = (op->kind == OP_VSTACK) != trans;
      int64_t off = 0;
      bool first = true;
      for (const cf_op* p : op->parts) {
        if (split_out) {
          if (!flatten(p, trans, alpha, xo, yo + off, acc, out, why)) return false;
          off += trans ? p->n : p->m;
        } else {
          if (!flatten(p, trans, alpha, xo + off, yo, first ? acc : true, out, why)) return false;
          off += trans ? p->m : p->n;
          first = false;
        }
      }
      return true;
    }
    case OP_BLOCKDIAG: {
      int64_t ro = 0, co = 0;
      for (const cf_op* p : op->parts) {
        const int64_t din = trans ? p->m : p->n, dout = trans ? p->n : p->m;
        if (!flatten(p, trans, alpha, xo + ro, yo + co, acc, out, why)) return false;
        ro += din;
        co += dout;
      }
      return true;
    }
    case OP_SUM: {
      bool first = true;
      for (const cf_op* p : op->parts) {
        if (!flatten(p, trans, alpha, xo, yo, first ? acc : true, out, why)) return false;
        first = false;
      }
      return true;
    }
    case OP_PRODUCT:
      *why = "operator product";
      return false;
    case OP_KRON:
      *why = "Kronecker operator";
      return false;
  }
  *why = "unknown operator";
  return false;
}

// A term whose outputs overlap an output written since the last barrier
// (under another row partition) needs a barrier first.
void mark_syncs(std::vector<Term>& ts) {
  std::vector<std::pair<int64_t, int64_t>> win;
  for (Term& t : ts) {
    const int64_t a = t.yo, b = t.yo + t.rows;
    bool hit = false;
    for (auto& w : win) hit |= a < w.second && w.first < b;
    t.sync = hit ? 1 : 0;
    if (hit) win.clear();
    win.push_back({a, b});
  }
}

double term_bytes(const Term& t) {
  switch (t.kind) {
    case T_FILL: return 4.0 * t.rows;
    case T_DIAG: return (t.a ? 12.0 : 8.0) * t.rows;
    case T_CSR: {
      return 0.0;  // filled in by plan_problem from the leaf's nnz
    }
    case T_DENSE_N: case T_DENSE_T: {
      const double esz = t.prec == CF_FP32 ? 4 : (t.prec == CF_BF16 ? 2 : 1);
      const double mrows = t.kind == T_DENSE_N ? t.rows : t.cols;
      return mrows * t.lda * esz + (t.scale ? 4.0 * mrows : 0.0);
    }
    case T_CONV:
      // input + output, and the multiply-adds at 16 flops per byte (one SM's
      // FP32 rate over its share of the memory bandwidth)
      return 4.0 * (t.rows + t.cols) + 2.0 * t.Lp * t.rows / 16.0;
    case T_FFT:
      // input + output, and ~90 transform flops per output at 16 per byte
      return 4.0 * (t.rows + t.cols) + 90.0 * t.rows / 16.0;
  }
  return 0.0;
}

}  // namespace

cf_err plan_problem(cf_problem* P) {
  Plan& pl = P->plan;
  pl = Plan();
  std::string why;
  if ((int64_t)P->q.size() > kMaxSeg) {
    pl.why = "more than " + std::to_string(kMaxSeg) + " second-order cones";
    return CF_OK;
  }
  if (P->inner) {
    pl.why = "an inner operator (mixed-precision refinement) runs on the graph engine";
    return CF_OK;
  }
  // an equilibrated operator diag(D) A diag(E): A's terms with the scalings
  // folded in (inputs scaled by E forward / D adjoint, outputs by D / E)
  const cf_op* core = P->A;
  const float *dsc = nullptr, *esc = nullptr;
  if (P->A->kind == OP_PRODUCT && P->A->parts.size() == 3 && P->A->parts[0]->kind == OP_DIAG &&
      P->A->parts[2]->kind == OP_DIAG) {
    core = P->A->parts[1];
    dsc = P->A->parts[0]->d;
    esc = P->A->parts[2]->d;
  }
  auto scale = [](std::vector<Term>& ts, const float* in, const float* out) {
    for (Term& t : ts) {
      t.sin = in ? in + t.xo : nullptr;
      t.sout = out ? out + t.yo : nullptr;
    }
  };
  if (!flatten(core, false, 1.f, 0, 0, false, pl.fwd, &why) ||
      !flatten(core, true, 1.f, 0, 0, false, pl.adj, &why) ||
      !flatten(core, true, -1.f, 0, 0, true, pl.adj_m, &why)) {
    pl.fwd.clear();
    pl.adj.clear();
    pl.adj_m.clear();
    pl.why = why;
    return CF_OK;
  }
  scale(pl.fwd, esc, dsc);
  scale(pl.adj, dsc, esc);
  scale(pl.adj_m, dsc, esc);
  mark_syncs(pl.fwd);
  mark_syncs(pl.adj);
  mark_syncs(pl.adj_m);
  // sizes: bytes of a forward pass (CSR from the leaf's nnz), CSR rows,
  // adjoint dense widths, shared memory
  double bytes = 0.0, nnz = 0.0, rows = 0.0;
  int64_t smem = 0;
  for (const Term& t : pl.fwd) {
    if (t.kind == T_CSR) {
      std::vector<int32_t> ends(2);
      // nnz of the leaf: rowptr[rows] (host copy of one entry)
      cudaMemcpy(ends.data(), t.rowptr + t.rows, sizeof(int32_t), cudaMemcpyDeviceToHost);
      const double esz = t.prec == CF_BF16 ? 2.0 : 4.0;
      bytes += ends[0] * (4.0 + esz) + 4.0 * (t.rows + 1);
      nnz += ends[0];
      rows += t.rows;
    } else {
      bytes += term_bytes(t);
    }
  }
  for (const std::vector<Term>* lst : {&pl.fwd, &pl.adj, &pl.adj_m})
    for (const Term& t : *lst) {
      if (t.kind == T_FFT) {
        if ((t.sin == nullptr) != (t.sout == nullptr)) {
          pl.fwd.clear();
          pl.adj.clear();
          pl.adj_m.clear();
          pl.why = "FFT convolution term with one of its two scalings";
          return CF_OK;
        }
        pl.has_fft = true;
      }
      if (t.kind == T_DENSE_N) smem = std::max<int64_t>(smem, (t.cols + 15) & ~(int64_t)15);
      if (t.kind == T_CONV) smem = std::max<int64_t>(smem, 2 * t.Lp + kConvTile + 2 * kConvR);
      if (t.kind == T_DENSE_T) pl.dense_t_cols = std::max(pl.dense_t_cols, t.rows);
      if (t.kind == T_CSR && t.cols <= kCsrStageFloats) smem = std::max<int64_t>(smem, t.cols);
    }
  pl.pass_bytes = bytes + 4.0 * (P->n + P->m);
  pl.avg_row_nnz = rows > 0 ? nnz / rows : 0.0;
  pl.smem_floats = smem;
  // device copy of the three lists
  const size_t nt = pl.fwd.size() + pl.adj.size() + pl.adj_m.size();
  std::vector<Term> all;
  all.reserve(nt);
  all.insert(all.end(), pl.fwd.begin(), pl.fwd.end());
  all.insert(all.end(), pl.adj.begin(), pl.adj.end());
  all.insert(all.end(), pl.adj_m.begin(), pl.adj_m.end());
  cudaError_t e = cudaMalloc((void**)&P->team_terms, std::max<size_t>(nt, 1) * sizeof(Term));
  if (e != cudaSuccess) {
    cudaGetLastError();
    P->team_terms = nullptr;
    return fail(CF_E_OOM, "cone_problem_create: allocation failed");
  }
  if (nt) CF_CUDA(cudaMemcpy(P->team_terms, all.data(), nt * sizeof(Term), cudaMemcpyHostToDevice));
  pl.ok = true;
  return CF_OK;
}

size_t scratch_floats(const cf_problem* P) {
  return P->plan.ok ? (size_t)kDenseTGroups * (size_t)P->plan.dense_t_cols : 0;
}

void release(cf_problem* P) {
  if (P->team_terms) cudaFree(P->team_terms);
  if (P->team_buf) cudaFree(P->team_buf);
  if (P->grid_buf) cudaFree(P->grid_buf);
  P->grid_buf = nullptr;
  if (P->team_buf_host) cudaFreeHost(P->team_buf_host);
  P->team_terms = nullptr;
  P->team_buf = nullptr;
  P->team_buf_host = nullptr;
}

// ------------------------------------------------------------ host: launches
namespace {

int lanes_for(const Plan& pl, const cf_schedule& s) {
  int L = 1;
  while (L < 32 && (double)L * s.csr_nnz_per_lane < pl.avg_row_nnz) L *= 2;
  return L;
}

bool is_big(const cf_problem* P, const cf_schedule& s) {
  return s.cluster > 1 && P->plan.pass_bytes >= s.team_bytes;
}

// Identifies the reduction partitions a problem runs with (>= 2; 1 is the
// graph engine).
int sig_for(const cf_problem* P, const cf_schedule& s) {
  const int C = is_big(P, s) ? s.cluster : 1;
  return 2 + (C * 4096 + s.threads) * 64 + lanes_for(P->plan, s);
}

void fill_prob(cf_problem* P, const cf_schedule& s, bool do_setup, bool tune, Prob* o) {
  std::memset(o, 0, sizeof(Prob));
  o->st = P->ctl_host->st;
  o->ctl = P->ctl;
  const Plan& pl = P->plan;
  o->fwd = P->team_terms;
  o->adj = P->team_terms + pl.fwd.size();
  o->adj_m = P->team_terms + pl.fwd.size() + pl.adj.size();
  o->nfwd = (int32_t)pl.fwd.size();
  o->nadj = (int32_t)pl.adj.size();
  o->nadj_m = (int32_t)pl.adj_m.size();
  o->nseg = (int32_t)P->q.size();
  o->lanes = lanes_for(pl, s);
  o->do_setup = do_setup ? 1 : 0;
  o->tune = tune ? 1 : 0;
  o->want_out = (!tune && (P->x_out || P->y_out || P->s_out)) ? 1 : 0;
  o->want_uv = (!tune && P->uv_out) ? 1 : 0;
  o->n = P->n;
  o->m = P->m;
  o->z = P->z;
  o->l = P->l;
  int64_t off = P->z + P->l;
  for (size_t j = 0; j < P->q.size(); ++j) {
    o->seg_head[j] = off;
    off += P->q[j];
    o->seg_end[j] = off;
  }
  o->nb = P->nb;
  o->nc = P->nc;
  o->bf = P->bf;
  o->cf = P->cf;
  o->ux = P->ux; o->uy = P->uy; o->vs = P->vs; o->zx = P->zx; o->rhs = P->rhs; o->r = P->r;
  o->p = P->p; o->q = P->qv; o->gx = P->gx; o->gy = P->gy; o->wy = P->wy; o->t = P->t;
  o->zy = P->zy; o->cm = P->cm; o->cn = P->cn; o->gz = P->gz; o->az = P->az;
  o->scratch = P->team_scratch;
  o->warm = P->warm_dev;
  o->out = P->out_dev;
  o->uv = P->uv_dev;
  o->eq_d = P->eq_d;
  o->eq_e = P->eq_e;
  o->eq_dinv = P->eq_dinv;
  o->eq_einv = P->eq_einv;
  o->sigma = P->sigma;
  o->rho = P->rho;
}

struct Launch {
  int C = 1, T = 512, B = 1;  // cluster size, threads per CTA, CTAs per SM the registers allow
  int64_t grid = 1;
  size_t smem = 0;
};

template <int MaxT, int MinB>
cf_err launch_k(const Launch& L, const Prob* probs, const int32_t* order, int32_t nbig, int32_t nsmall,
                unsigned int* counters, cudaStream_t s) {
  auto kern = k_team<MaxT, MinB>;
  if (L.smem > 48 * 1024) CF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)L.grid);
  cfg.blockDim = dim3((unsigned)L.T);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (L.C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  CF_CUDA(cudaLaunchKernelEx(&cfg, kern, probs, order, nbig, nsmall, counters, (int32_t)L.C));
  return CF_OK;
}

template <int MaxT, int MinB>
cf_err max_grid(const Launch& L, int sm_count, int64_t* out) {
  auto kern = k_team<MaxT, MinB>;
  if (L.smem > 48 * 1024) CF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
  if (L.C == 1) {
    int nb = 0;
    CF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, L.T, L.smem));
    *out = (int64_t)std::max(nb, 1) * sm_count;
    return CF_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(L.C * sm_count));
  cfg.blockDim = dim3((unsigned)L.T);
  cfg.dynamicSmemBytes = L.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)L.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  CF_CUDA(cudaOccupancyMaxActiveClusters(&nc, kern, &cfg));
  *out = (int64_t)std::max(nc, 1) * L.C;
  return CF_OK;
}

template <int T, int B>
cf_err dispatch_tb(const Launch& L, bool query, int sm_count, int64_t* grid, const Prob* probs,
                   const int32_t* order, int32_t nbig, int32_t nsmall, unsigned int* counters, cudaStream_t s) {
  return query ? max_grid<T, B>(L, sm_count, grid) : launch_k<T, B>(L, probs, order, nbig, nsmall, counters, s);
}

cf_err dispatch(const Launch& L, bool query, int sm_count, int64_t* grid, const Prob* probs,
                const int32_t* order, int32_t nbig, int32_t nsmall, unsigned int* counters, cudaStream_t s) {
  const int key = L.T * 8 + L.B;
  switch (key) {
    case 256 * 8 + 1: return dispatch_tb<256, 1>(L, query, sm_count, grid, probs, order, nbig, nsmall, counters, s);
    case 256 * 8 + 2: return dispatch_tb<256, 2>(L, query, sm_count, grid, probs, order, nbig, nsmall, counters, s);
    case 256 * 8 + 4: return dispatch_tb<256, 4>(L, query, sm_count, grid, probs, order, nbig, nsmall, counters, s);
    case 512 * 8 + 1: return dispatch_tb<512, 1>(L, query, sm_count, grid, probs, order, nbig, nsmall, counters, s);
    case 512 * 8 + 2: return dispatch_tb<512, 2>(L, query, sm_count, grid, probs, order, nbig, nsmall, counters, s);
    case 1024 * 8 + 1: return dispatch_tb<1024, 1>(L, query, sm_count, grid, probs, order, nbig, nsmall, counters, s);
  }
  return fail(CF_E_INVALID, "team engine: unsupported threads per CTA x CTAs per SM");
}

// Launch table layout: counters (2), order (count), then the entries.
size_t table_bytes(size_t count) {
  return 256 + align_up(count * sizeof(int32_t), 256) + count * sizeof(Prob);
}

// Builds the table for `probs` under schedule s into host memory `h` (of
// table_bytes(count)), orders big problems then small ones, longest first.
void build_table(const std::vector<cf_problem*>& probs, const cf_schedule& s, bool tune, char* h,
                 int32_t* nbig_out, int32_t* nsmall_out, size_t* smem_out, std::vector<int>* setups) {
  const size_t count = probs.size();
  std::memset(h, 0, 256);
  int32_t* order = (int32_t*)(h + 256);
  Prob* ents = (Prob*)(h + 256 + align_up(count * sizeof(int32_t), 256));
  std::vector<int32_t> big, small;
  size_t smem = 0;
  setups->assign(count, 0);
  for (size_t i = 0; i < count; ++i) {
    cf_problem* P = probs[i];
    const int sig = sig_for(P, s);
    const bool do_setup = !tune && !(P->setup_done && P->setup_sig == sig);
    (*setups)[i] = do_setup ? 1 : 0;
    fill_prob(P, s, do_setup, tune, &ents[i]);
    (is_big(P, s) ? big : small).push_back((int32_t)i);
    smem = std::max(smem, (size_t)P->plan.smem_floats * sizeof(float));
    if (P->plan.has_fft) smem = std::max(smem, (size_t)s.threads * 17 * sizeof(float2));  // (N + N/16) float2 per N/16 threads
  }
  auto longer = [&](int32_t a, int32_t b) {
    const double wa = probs[a]->plan.pass_bytes, wb = probs[b]->plan.pass_bytes;
    return wa != wb ? wa > wb : a < b;
  };
  std::sort(big.begin(), big.end(), longer);
  std::sort(small.begin(), small.end(), longer);
  size_t k = 0;
  for (int32_t i : big) order[k++] = i;
  for (int32_t i : small) order[k++] = i;
  *nbig_out = (int32_t)big.size();
  *nsmall_out = (int32_t)small.size();
  *smem_out = smem;
}

// Enqueues the launch of a table already on the device at `dev` (same
// layout) on stream s.
cf_err enqueue(cf_ctx* ctx, const cf_schedule& s, char* dev, size_t count, int32_t nbig, int32_t nsmall,
               size_t smem, cudaStream_t st) {
  Launch L;
  L.T = s.threads;
  L.B = s.ctas_per_sm;
  L.C = nbig > 0 ? s.cluster : 1;
  L.smem = smem;
  int64_t cap = 1;
  CF_TRY(dispatch(L, true, ctx->sm_count, &cap, nullptr, nullptr, 0, 0, nullptr, nullptr));
  const int64_t need = (int64_t)nbig * L.C + nsmall;  // CTAs that can be busy at once
  int64_t g = std::min<int64_t>(cap, std::max<int64_t>(need, 1));
  g = std::max<int64_t>((g + L.C - 1) / L.C * L.C, L.C);
  if (g > cap) g = std::max<int64_t>(cap / L.C * L.C, L.C);
  L.grid = g;
  unsigned int* counters = (unsigned int*)dev;
  const int32_t* order = (const int32_t*)(dev + 256);
  const Prob* ents = (const Prob*)(dev + 256 + align_up(count * sizeof(int32_t), 256));
  return dispatch(L, false, ctx->sm_count, nullptr, ents, order, nbig, nsmall, counters, st);
}

cf_schedule sched_of(cf_ctx* ctx) {
  std::lock_guard<std::mutex> lk(ctx->sched_mu);
  return ctx->sched;
}

}  // namespace

cf_err solo_launch(cf_problem* P, const cf_settings* st, const double* warm_uv, bool join_ctx) {
  const cf_schedule s = sched_of(P->ctx);
  const size_t bytes = table_bytes(1);
  if (!P->team_buf) {
    cudaError_t e = cudaMalloc(&P->team_buf, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      P->team_buf = nullptr;
      return fail(CF_E_OOM, "solve: team launch table allocation failed");
    }
    CF_CUDA(cudaMallocHost(&P->team_buf_host, bytes));
  }
  const int64_t N = P->n + P->m + 1;
  CF_CUDA(cudaEventRecord(P->ev_in, P->ctx->stream));
  CF_CUDA(cudaStreamWaitEvent(P->stream, P->ev_in, 0));
  if (warm_uv) CF_TRY(copy_any(P->warm_dev, warm_uv, 2 * N * sizeof(double), P->stream));
  int32_t nbig = 0, nsmall = 0;
  size_t smem = 0;
  std::vector<int> setups;
  // the pinned staging buffer is free: the previous solve of P finished
  build_table({P}, s, false, (char*)P->team_buf_host, &nbig, &nsmall, &smem, &setups);
  CF_CUDA(cudaMemcpyAsync(P->team_buf, P->team_buf_host, bytes, cudaMemcpyHostToDevice, P->stream));
  P->t_launch = now_ns();
  CF_TRY(enqueue(P->ctx, s, (char*)P->team_buf, 1, nbig, nsmall, smem, P->stream));
  CF_CUDA(cudaMemcpyAsync(P->ctl_host, P->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P->stream));
  CF_CUDA(cudaEventRecord(P->ev_out, P->stream));
  if (join_ctx) CF_CUDA(cudaStreamWaitEvent(P->ctx->stream, P->ev_out, 0));
  P->ran_setup = setups[0] != 0;
  P->setup_done = true;
  P->setup_sig = sig_for(P, s);
  P->last_engine = CF_ENGINE_TEAM;
  P->team_launches = 1;
  (void)st;
  return CF_OK;
}

namespace {

constexpr int kGridThreads = 512;  // threads per CTA of a grid team (two FFT transforms at a time)

// Identifies the grid team's reduction partitions (distinct from every
// batch schedule's).
int grid_sig(int C, int lanes) { return 2 + ((1000 + C) * 4096 + kGridThreads) * 64 + lanes; }

}  // namespace

cf_err grid_launch(cf_problem* P, const cf_settings* st, const double* warm_uv, bool join_ctx) {
  cf_schedule s = sched_of(P->ctx);
  s.cluster = 1;
  s.threads = kGridThreads;
  s.ctas_per_sm = 1;
  const int C = P->ctx->sm_count;  // one CTA per SM
  size_t smem = (size_t)P->plan.smem_floats * sizeof(float);
  if (P->plan.has_fft) smem = std::max(smem, (size_t)kGridThreads * 17 * sizeof(float2));
  auto kern = k_team_grid<kGridThreads, 1>;
  if (smem > 48 * 1024) CF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGridThreads, smem));
  if (per_sm < 1) return fail(CF_E_INVALID, "solve: the grid engine's kernel does not fit on an SM");
  const size_t bytes = table_bytes(1);
  if (!P->team_buf) {
    cudaError_t e = cudaMalloc(&P->team_buf, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      P->team_buf = nullptr;
      return fail(CF_E_OOM, "solve: team launch table allocation failed");
    }
    CF_CUDA(cudaMallocHost(&P->team_buf_host, bytes));
  }
  const size_t gbytes = 256 + (size_t)2 * C * 32 * sizeof(float);
  if (!P->grid_buf) {
    cudaError_t e = cudaMalloc(&P->grid_buf, gbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      P->grid_buf = nullptr;
      return fail(CF_E_OOM, "solve: grid barrier allocation failed");
    }
  }
  const int64_t N = P->n + P->m + 1;
  CF_CUDA(cudaEventRecord(P->ev_in, P->ctx->stream));
  CF_CUDA(cudaStreamWaitEvent(P->stream, P->ev_in, 0));
  if (warm_uv) CF_TRY(copy_any(P->warm_dev, warm_uv, 2 * N * sizeof(double), P->stream));
  const int sig = grid_sig(C, lanes_for(P->plan, s));
  const bool do_setup = !(P->setup_done && P->setup_sig == sig);
  // the pinned staging buffer is free: the previous solve of P finished
  Prob* ph = (Prob*)P->team_buf_host;
  fill_prob(P, s, do_setup, false, ph);
  CF_CUDA(cudaMemcpyAsync(P->team_buf, ph, sizeof(Prob), cudaMemcpyHostToDevice, P->stream));
  CF_CUDA(cudaMemsetAsync(P->grid_buf, 0, sizeof(GridBar), P->stream));
  P->t_launch = now_ns();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3((unsigned)kGridThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = P->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // CVXB300_GRID_SPIN_LIMIT (tests of the give-up path) lowers the poll limit
  unsigned int spin = kGridSpinLimit;
  if (const char* ev = std::getenv("CVXB300_GRID_SPIN_LIMIT")) spin = (unsigned int)std::strtoul(ev, nullptr, 10);
  CF_CUDA(cudaLaunchKernelEx(&cfg, kern, (const Prob*)P->team_buf, (GridBar*)P->grid_buf,
                             (float*)((char*)P->grid_buf + 256), spin));
  CF_CUDA(cudaMemcpyAsync(P->ctl_host, P->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P->stream));
  CF_CUDA(cudaEventRecord(P->ev_out, P->stream));
  if (join_ctx) CF_CUDA(cudaStreamWaitEvent(P->ctx->stream, P->ev_out, 0));
  P->ran_setup = do_setup;
  P->setup_done = true;
  P->setup_sig = sig;
  P->last_engine = CF_ENGINE_GRID;
  P->team_launches = 1;
  (void)st;
  return CF_OK;
}

namespace {

// One launch of `probs` (one context) on stream s; table memory from the
// stream-ordered allocator, freed after the launch.
cf_err launch_group(const std::vector<cf_problem*>& probs, const cf_schedule& s, bool tune, cudaStream_t st,
                    std::vector<int>* setups) {
  cf_ctx* ctx = probs[0]->ctx;
  const size_t bytes = table_bytes(probs.size());
  std::vector<char> host(bytes);
  int32_t nbig = 0, nsmall = 0;
  size_t smem = 0;
  build_table(probs, s, tune, host.data(), &nbig, &nsmall, &smem, setups);
  char* dev = nullptr;
  CF_CUDA(cudaMallocAsync((void**)&dev, bytes, st));
  CF_CUDA(cudaMemcpyAsync(dev, host.data(), bytes, cudaMemcpyHostToDevice, st));
  cf_err r = enqueue(ctx, s, dev, probs.size(), nbig, nsmall, smem, st);
  cudaFreeAsync(dev, st);
  return r;
}

}  // namespace

cf_err batch_launch(const std::vector<cf_problem*>& probs, const cf_settings* st) {
  if (probs.empty()) return CF_OK;
  (void)st;
  cf_ctx* ctx = probs[0]->ctx;
  const cf_schedule s = sched_of(ctx);
  cudaStream_t bs = nullptr;
  cudaEvent_t ev = nullptr;
  CF_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  cf_err r = [&]() -> cf_err {
    CF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CF_CUDA(cudaEventRecord(ev, ctx->stream));
    CF_CUDA(cudaStreamWaitEvent(bs, ev, 0));
    const int64_t t0 = now_ns();
    std::vector<int> setups;
    CF_TRY(launch_group(probs, s, false, bs, &setups));
    CF_CUDA(cudaEventRecord(ev, bs));
    for (size_t i = 0; i < probs.size(); ++i) {
      cf_problem* P = probs[i];
      P->t_launch = t0;
      CF_CUDA(cudaStreamWaitEvent(P->stream, ev, 0));
      CF_CUDA(cudaMemcpyAsync(P->ctl_host, P->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, P->stream));
      CF_CUDA(cudaEventRecord(P->ev_out, P->stream));
      P->ran_setup = setups[i] != 0;
      P->setup_done = true;
      P->setup_sig = sig_for(P, s);
      P->last_engine = CF_ENGINE_TEAM;
      P->team_launches = i == 0 ? 1 : 0;
    }
    return CF_OK;
  }();
  if (ev) cudaEventDestroy(ev);
  cudaStreamDestroy(bs);  // released once its work is done
  return r;
}

}  // namespace team

// ------------------------------------------------------------ schedules
cf_schedule default_schedule() {
  cf_schedule s{};
  s.cluster = 4;
  s.threads = 512;
  s.csr_nnz_per_lane = 16;
  s.ctas_per_sm = 1;
  s.team_bytes = 256e3;
  s.auto_max_bytes = 1e6;
  s.batch_max_bytes = 48e6;
  return s;
}

bool schedule_valid(const cf_schedule& s, std::string* why) {
  if (s.cluster != 1 && s.cluster != 2 && s.cluster != 4 && s.cluster != 8) {
    *why = "cluster must be 1, 2, 4 or 8";
    return false;
  }
  if (s.threads != 256 && s.threads != 512 && s.threads != 1024) {
    *why = "threads must be 256, 512 or 1024";
    return false;
  }
  if (!((s.ctas_per_sm == 1) || (s.ctas_per_sm == 2 && s.threads <= 512) ||
        (s.ctas_per_sm == 4 && s.threads == 256))) {
    *why = "ctas_per_sm must be 1, 2 (threads <= 512) or 4 (threads 256)";
    return false;
  }
  if (s.csr_nnz_per_lane < 1 || s.csr_nnz_per_lane > 64) {
    *why = "csr_nnz_per_lane must be in [1, 64]";
    return false;
  }
  if (!(s.team_bytes >= 0) || !(s.auto_max_bytes >= 0) || !(s.batch_max_bytes >= 0)) {
    *why = "team_bytes, auto_max_bytes and batch_max_bytes must be >= 0";
    return false;
  }
  return true;
}

cf_err pick_engine(cf_problem* P, const cf_settings* st, int* engine, bool in_batch) {
  if (st->host_loop || st->engine == CF_ENGINE_GRAPH) {
    *engine = CF_ENGINE_GRAPH;
    return CF_OK;
  }
  if (st->engine == CF_ENGINE_TEAM || (st->engine == CF_ENGINE_GRID && in_batch)) {
    if (!P->plan.ok) return fail(CF_E_INVALID, "solve: the team engine does not support this problem: " + P->plan.why);
    *engine = CF_ENGINE_TEAM;
    return CF_OK;
  }
  if (st->engine == CF_ENGINE_GRID) {
    if (!P->plan.ok) return fail(CF_E_INVALID, "solve: the grid engine does not support this problem: " + P->plan.why);
    *engine = CF_ENGINE_GRID;
    return CF_OK;
  }
  double lim;
  {
    std::lock_guard<std::mutex> lk(P->ctx->sched_mu);
    lim = in_batch ? std::max(P->ctx->sched.auto_max_bytes, P->ctx->sched.batch_max_bytes)
                   : P->ctx->sched.auto_max_bytes;
  }
  *engine = (P->plan.ok && P->plan.pass_bytes <= lim) ? CF_ENGINE_TEAM : CF_ENGINE_GRAPH;
  return CF_OK;
}

}  // namespace cf

using namespace cf;

// ------------------------------------------------------------------ C ABI
extern "C" cf_err cf_problem_team_info(const cf_problem* p, int32_t* supported, double* pass_bytes, char* why,
                                       size_t why_len) {
  if (!p) return fail(CF_E_INVALID, "cf_problem_team_info: NULL problem");
  if (supported) *supported = p->plan.ok ? 1 : 0;
  if (pass_bytes) *pass_bytes = p->plan.ok ? p->plan.pass_bytes : 0.0;
  if (why && why_len > 0) {
    const size_t k = std::min(why_len - 1, p->plan.why.size());
    std::memcpy(why, p->plan.why.data(), k);
    why[k] = 0;
  }
  return CF_OK;
}

extern "C" cf_err solve_batch_tune(cf_problem* const* probs, int32_t count, int32_t iters, cf_tune_info* info) {
  if (count < 0 || (count > 0 && !probs) || iters < 1 || iters > 100000)
    return fail(CF_E_INVALID, "solve_batch_tune: bad arguments");
  if (info) std::memset(info, 0, sizeof(*info));
  if (count == 0) return CF_OK;
  for (int32_t i = 0; i < count; ++i) {
    if (!probs[i]) return fail(CF_E_INVALID, "solve_batch_tune: NULL problem");
    if (probs[i]->ctx != probs[0]->ctx) return fail(CF_E_INVALID, "solve_batch_tune: problems of different contexts");
    for (int32_t j = 0; j < i; ++j)
      if (probs[j] == probs[i]) return fail(CF_E_INVALID, "solve_batch_tune: a problem appears twice");
  }
  cf_ctx* ctx = probs[0]->ctx;
  const int64_t t0 = now_ns();
  std::vector<std::unique_lock<std::mutex>> locks;
  for (int32_t i = 0; i < count; ++i) locks.emplace_back(probs[i]->mtx);
  DevGuard guard(ctx->device);
  cf_schedule held;
  {
    std::lock_guard<std::mutex> lk(ctx->sched_mu);
    held = ctx->sched;
  }
  cf_settings st;
  cf_settings_default(&st);
  st.max_iters = iters;
  st.check_interval = 1 << 30;
  st.cg_fixed_iters = 2;
  std::vector<cf_problem*> tp;
  for (int32_t i = 0; i < count; ++i) {
    cf_problem* P = probs[i];
    if (!P->plan.ok || P->plan.pass_bytes > std::max(held.auto_max_bytes, held.batch_max_bytes)) continue;
    CF_TRY(ensure_state(P));
    write_settings(P, &st, false);
    P->x_out = P->y_out = P->s_out = P->uv_out = nullptr;
    tp.push_back(P);
  }
  if (tp.empty()) return CF_OK;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  int ncand = 0;
  auto timed = [&](const cf_schedule& sc, double* ms) -> cf_err {
    std::vector<int> setups;
    CF_CUDA(cudaEventRecord(e0, s));
    CF_TRY(team::launch_group(tp, sc, true, s, &setups));
    CF_CUDA(cudaEventRecord(e1, s));
    CF_CUDA(cudaEventSynchronize(e1));
    float f = 0.f;
    CF_CUDA(cudaEventElapsedTime(&f, e0, e1));
    *ms = f;
    ++ncand;
    return CF_OK;
  };
  cf_schedule best = held;
  double best_ms = 0.0, held_ms = 0.0;
  cf_err r = [&]() -> cf_err {
    CF_CUDA(cudaEventCreate(&e0));
    CF_CUDA(cudaEventCreate(&e1));
    CF_CUDA(cudaEventRecord(e0, ctx->stream));
    CF_CUDA(cudaStreamWaitEvent(s, e0, 0));
    double ms = 0.0;
    CF_TRY(timed(held, &ms));  // warm-up (module load, caches)
    CF_TRY(timed(held, &held_ms));
    best_ms = held_ms;
    // stage 1: one-CTA teams; threads per CTA and CSR lanes per row
    cf_schedule b1 = held;
    b1.cluster = 1;
    double b1_ms = 1e300;
    const int shapes[6][2] = {{256, 1}, {256, 2}, {256, 4}, {512, 1}, {512, 2}, {1024, 1}};
    for (const auto& tb : shapes)
      for (int npl : {8, 16, 32, 64}) {
        cf_schedule c = held;
        c.cluster = 1;
        c.threads = tb[0];
        c.ctas_per_sm = tb[1];
        c.csr_nnz_per_lane = npl;
        CF_TRY(timed(c, &ms));
        if (ms < b1_ms) {
          b1_ms = ms;
          b1 = c;
        }
      }
    if (b1_ms < best_ms) {
      best_ms = b1_ms;
      best = b1;
    }
    // stage 2: cluster teams for the largest problems
    std::vector<double> w;
    for (cf_problem* P : tp) w.push_back(P->plan.pass_bytes);
    std::sort(w.begin(), w.end(), std::greater<double>());
    for (int C : {2, 4, 8})
      for (double f : {0.02, 0.06, 0.15}) {
        const size_t k = std::min(w.size() - 1, (size_t)std::floor(f * (double)w.size()));
        cf_schedule c = b1;
        c.cluster = C;
        c.team_bytes = w[k];
        CF_TRY(timed(c, &ms));
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    return CF_OK;
  }();
  cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  // the timing runs zeroed g: every problem redoes its setup
  for (cf_problem* P : tp) P->setup_done = false;
  if (r != CF_OK) return r;
  best.auto_max_bytes = held.auto_max_bytes;
  best.batch_max_bytes = held.batch_max_bytes;
  {
    std::lock_guard<std::mutex> lk(ctx->sched_mu);
    ctx->sched = best;
  }
  if (info) {
    info->candidates = ncand;
    info->problems = (int32_t)tp.size();
    info->seconds = (now_ns() - t0) * 1e-9;
    info->default_ms = held_ms;
    info->best_ms = best_ms;
    info->best = best;
  }
  return CF_OK;
}
