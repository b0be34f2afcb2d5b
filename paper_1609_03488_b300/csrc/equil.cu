// Matrix-free data equilibration (Section 3: forward and adjoint evaluations
// suffice to precondition a problem, after stochastic matrix-free
// equilibration).  Squared row and column norms of D A E are estimated from
// random-sign probes ((D A E s)_i^2 averages to sum_j (D A E)_ij^2 over signs
// s), then every row / column is divided by the square root of its estimated
// norm (a Ruiz step), with one factor per second-order cone block so that the
// cone is kept; rows and columns with a zero estimated norm keep their
// factor.  b and c are scaled to unit norm afterwards.  The problem's
// operator becomes diag(D) A diag(E); stopping tests and returned points are
// taken back to the original problem by the check and output kernels.
//
// The signs come from SplitMix64 (Steele, Lea, Flood 2014) used as a
// counter-based generator: output mix of seed + (k + 1) * 0x9E3779B97F4A7C15
// for counter k; top bit set gives -1.  Probe p of iteration t uses counters
// (t * probes + p) * 2^32 + j for the column signs (j < n) and
// (t * probes + p) * 2^32 + n + i for the row signs (i < m).
#include <cmath>
#include <cstring>

#include "solver.cuh"

namespace cf {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr float kScaleMin = 1e-4f, kScaleMax = 1e4f;
constexpr double kNormFloor = 1e-3;
constexpr float kZeroNorm2 = 1e-18f;

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// out[j] = scale[j] * sign(counter base + j)
__global__ void k_probe(int64_t n, uint64_t seed, uint64_t base, const float* __restrict__ scale,
                        float* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t v = sm64_mix(seed + (base + (uint64_t)j + 1ull) * kGamma);
    out[j] = (v >> 63) ? -scale[j] : scale[j];
  }
}

// acc[i] += (scale[i] v[i])^2
__global__ void k_sqacc(int64_t n, const float* __restrict__ scale, const float* __restrict__ v,
                        float* __restrict__ acc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float t = scale[i] * v[i];
    acc[i] = fmaf(t, t, acc[i]);
  }
}

// Every row of a second-order cone block gets the block's mean, in three
// launches over chunks of at most kMeanChunk rows (chunk c: rows
// [ch[3c], ch[3c + 1]) of block ch[3c + 2]): per-chunk FP64 sums, per-block
// sums of its chunks in chunk order, then the fill.
constexpr int64_t kMeanChunk = 16384;

__global__ void k_block_part(const int64_t* __restrict__ ch, const float* __restrict__ acc,
                             double* __restrict__ part) {
  const int64_t lo = ch[3 * blockIdx.x], hi = ch[3 * blockIdx.x + 1];
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += (double)acc[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// bk[3b], bk[3b + 1]: first chunk and chunk count of block b; bk[3b + 2]: rows
__global__ void k_block_final(int64_t nblk, const int64_t* __restrict__ bk, const double* __restrict__ part,
                              float* __restrict__ mean) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  double s = 0.0;
  for (int64_t c = bk[3 * b]; c < bk[3 * b] + bk[3 * b + 1]; ++c) s += part[c];
  mean[b] = (float)(s / (double)bk[3 * b + 2]);
}

__global__ void k_block_fill(const int64_t* __restrict__ ch, const float* __restrict__ mean,
                             float* __restrict__ acc) {
  const int64_t lo = ch[3 * blockIdx.x], hi = ch[3 * blockIdx.x + 1];
  const float v = mean[ch[3 * blockIdx.x + 2]];
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc[i] = v;
}

// s[i] <- clip(s[i] / (acc[i] / K)^(1/4)); a row / column whose estimated
// squared norm is zero (an empty row of a sparse operator) keeps its factor
__global__ void k_ruiz(int64_t n, float inv_k, const float* __restrict__ acc, float* __restrict__ s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = acc[i] * inv_k;
    if (r > kZeroNorm2) s[i] = fminf(fmaxf(s[i] / sqrtf(sqrtf(r)), kScaleMin), kScaleMax);
  }
}

// per-CTA partial sums of (s[i] v[i])^2 (added on the host in CTA order)
__global__ void k_sqnorm_part(int64_t n, const float* __restrict__ s, const float* __restrict__ v,
                              double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = (double)s[i] * (double)v[i];
    acc += t * t;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// v[i] = f s[i] v[i]; inv[i] = 1 / s[i]
__global__ void k_scale_vec(int64_t n, float f, const float* __restrict__ s, float* __restrict__ v,
                            float* __restrict__ inv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    v[i] = f * s[i] * v[i];
    inv[i] = 1.f / s[i];
  }
}

__global__ void k_fill1(int64_t n, float* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 1.f;
}

constexpr int kNormGrid = 256;

cf_err sqnorm(int64_t n, const float* s, const float* v, double* part_dev, double* out, cudaStream_t st) {
  k_sqnorm_part<<<kNormGrid, 256, 0, st>>>(n, s, v, part_dev);
  CF_CUDA(cudaGetLastError());
  double h[kNormGrid];
  CF_CUDA(cudaMemcpyAsync(h, part_dev, sizeof(h), cudaMemcpyDeviceToHost, st));
  CF_CUDA(cudaStreamSynchronize(st));
  double t = 0.0;
  for (int k = 0; k < kNormGrid; ++k) t += h[k];
  *out = t;
  return CF_OK;
}

}  // namespace
}  // namespace cf

using namespace cf;

extern "C" cf_err cone_problem_equilibrate(cf_problem* P, int32_t iters, int32_t probes, uint64_t seed) {
  if (!P || iters < 0 || iters > 100 || probes < 1 || probes > 1024)
    return fail(CF_E_INVALID, "cone_problem_equilibrate: bad arguments");
  std::lock_guard<std::mutex> lk(P->mtx);
  if (P->eq) return fail(CF_E_STATE, "cone_problem_equilibrate: the problem is already equilibrated");
  DevGuard guard(P->device);
  const int64_t m = P->m, n = P->n;
  cudaStream_t st = P->stream;
  CF_CUDA(cudaEventRecord(P->ev_in, P->ctx->stream));
  CF_CUDA(cudaStreamWaitEvent(st, P->ev_in, 0));
  CF_CUDA(cudaStreamSynchronize(st));
  // persistent: D, E, 1/D, 1/E; temporaries: probes, products, accumulators
  const size_t eq_floats = align_up(m, 64) * 2 + align_up(n, 64) * 2;
  float* eq = nullptr;
  cudaError_t e = cudaMalloc((void**)&eq, eq_floats * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CF_E_OOM, "cone_problem_equilibrate: allocation failed");
  }
  float* d = eq;
  float* dinv = d + align_up(m, 64);
  float* ev = dinv + align_up(m, 64);
  float* einv = ev + align_up(n, 64);
  const size_t wsf = std::max(op_ws_floats(P->A, false), op_ws_floats(P->A, true));
  const size_t tmp_floats = align_up(n, 64) * 3 + align_up(m, 64) * 3 + align_up(wsf, 64) + 2 * kNormGrid + 64;
  float* tmp = nullptr;
  cf_op *dD = nullptr, *dE = nullptr, *prod = nullptr;
  auto run = [&]() -> cf_err {
    e = cudaMalloc((void**)&tmp, tmp_floats * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      tmp = nullptr;
      return fail(CF_E_OOM, "cone_problem_equilibrate: allocation failed");
    }
    float* xin = tmp;
    float* xout = xin + align_up(n, 64);
    float* cacc = xout + align_up(n, 64);
    float* yin = cacc + align_up(n, 64);
    float* yout = yin + align_up(m, 64);
    float* racc = yout + align_up(m, 64);
    float* ws = racc + align_up(m, 64);
    double* part = (double*)(ws + align_up(wsf, 64));
    // second-order cone blocks, in chunks: table ch (lo, hi, block) per
    // chunk, bk (first chunk, chunks, rows) per block, then the per-chunk
    // sums (double) and per-block means (float) -- one allocation
    std::vector<int64_t> ch, bk;
    int64_t off = P->z + P->l;
    for (size_t b = 0; b < P->q.size(); ++b) {
      const int64_t q = P->q[b];
      bk.push_back((int64_t)ch.size() / 3);
      for (int64_t s = 0; s < q; s += kMeanChunk) {
        ch.push_back(off + s);
        ch.push_back(off + std::min(q, s + kMeanChunk));
        ch.push_back((int64_t)b);
      }
      bk.push_back((int64_t)ch.size() / 3 - bk.back());
      bk.push_back(q);
      off += q;
    }
    const int64_t nchunk = (int64_t)ch.size() / 3, nblk = (int64_t)P->q.size();
    int64_t* lohi_dev = nullptr;
    int64_t *ch_dev = nullptr, *bk_dev = nullptr;
    double* part_dev = nullptr;
    float* mean_dev = nullptr;
    if (nblk > 0) {
      const size_t words = ch.size() + bk.size() + (size_t)nchunk + (size_t)nblk;  // 8-byte words
      CF_CUDA(cudaMalloc((void**)&lohi_dev, words * sizeof(int64_t)));
      ch_dev = lohi_dev;
      bk_dev = ch_dev + ch.size();
      part_dev = (double*)(bk_dev + bk.size());
      mean_dev = (float*)(part_dev + nchunk);
      CF_CUDA(cudaMemcpy(ch_dev, ch.data(), ch.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
      CF_CUDA(cudaMemcpy(bk_dev, bk.data(), bk.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
    const unsigned gm = (unsigned)grid_for(m), gn = (unsigned)grid_for(n);
    k_fill1<<<gm, kThreads, 0, st>>>(m, d);
    k_fill1<<<gn, kThreads, 0, st>>>(n, ev);
    for (int t = 0; t < iters; ++t) {
      CF_CUDA(cudaMemsetAsync(racc, 0, m * sizeof(float), st));
      CF_CUDA(cudaMemsetAsync(cacc, 0, n * sizeof(float), st));
      for (int k = 0; k < probes; ++k) {
        const uint64_t base = (uint64_t)(t * probes + k) << 32;
        // the probes' products are squared and summed into row / column
        // norm estimates: convolutions by the direct sum, whose float32 error
        // is bounded entry by entry (an FFT's is bounded per segment, which
        // on the small entries of a random-sign product of a wide kernel is
        // ~1e-5 relative and moves the scalings by as much)
        k_probe<<<gn, kThreads, 0, st>>>(n, seed, base, ev, xin);
        op_apply(P->A, false, 1.f, xin, yout, false, ws, st, /*direct_conv=*/true);
        k_sqacc<<<gm, kThreads, 0, st>>>(m, d, yout, racc);
        k_probe<<<gm, kThreads, 0, st>>>(m, seed, base + (uint64_t)n, d, yin);
        op_apply(P->A, true, 1.f, yin, xout, false, ws, st, /*direct_conv=*/true);
        k_sqacc<<<gn, kThreads, 0, st>>>(n, ev, xout, cacc);
      }
      if (nblk > 0) {
        k_block_part<<<(unsigned)nchunk, 256, 0, st>>>(ch_dev, racc, part_dev);
        k_block_final<<<(unsigned)((nblk + 127) / 128), 128, 0, st>>>(nblk, bk_dev, part_dev, mean_dev);
        k_block_fill<<<(unsigned)nchunk, 256, 0, st>>>(ch_dev, mean_dev, racc);
      }
      k_ruiz<<<gm, kThreads, 0, st>>>(m, 1.f / (float)probes, racc, d);
      k_ruiz<<<gn, kThreads, 0, st>>>(n, 1.f / (float)probes, cacc, ev);
      CF_CUDA(cudaGetLastError());
    }
    double nb2 = 0, nc2 = 0;
    CF_TRY(sqnorm(m, d, P->bf, part, &nb2, st));
    CF_TRY(sqnorm(n, ev, P->cf, part, &nc2, st));
    const double sigma = 1.0 / std::max(std::sqrt(nb2), kNormFloor);
    const double rho = 1.0 / std::max(std::sqrt(nc2), kNormFloor);
    k_scale_vec<<<gm, kThreads, 0, st>>>(m, (float)sigma, d, P->bf, dinv);
    k_scale_vec<<<gn, kThreads, 0, st>>>(n, (float)rho, ev, P->cf, einv);
    CF_CUDA(cudaGetLastError());
    CF_CUDA(cudaStreamSynchronize(st));
    if (lohi_dev) cudaFree(lohi_dev);
    // the solver's operator becomes diag(D) A diag(E)
    CF_TRY(cf_op_diag(P->ctx, m, d, &dD));
    CF_TRY(cf_op_diag(P->ctx, n, ev, &dE));
    cf_op* parts[3] = {dD, P->A, dE};
    CF_TRY(operator_compose(P->ctx, CF_PRODUCT, parts, 3, 1.0, &prod));
    P->sigma = sigma;
    P->rho = rho;
    return CF_OK;
  };
  cf_err r = run();
  if (tmp) cudaFree(tmp);
  if (dD) cf_op_destroy(dD);  // the product holds its own references
  if (dE) cf_op_destroy(dE);
  if (r != CF_OK) {
    if (prod) cf_op_destroy(prod);
    cudaFree(eq);
    P->sigma = P->rho = 1.0;
    return r;
  }
  P->eq = eq;
  P->eq_d = d;
  P->eq_e = ev;
  P->eq_dinv = dinv;
  P->eq_einv = einv;
  P->A_orig = P->A;  // keeps its reference
  P->A = prod;
  if (P->inner) {
    // refinement: the inner operator takes the same diagonals
    cf_op* parts[3] = {prod->parts[0], P->inner, prod->parts[2]};
    cf_op* wrapped = nullptr;
    r = operator_compose(P->ctx, CF_PRODUCT, parts, 3, 1.0, &wrapped);
    if (r != CF_OK) return r;
    P->inner_orig = P->inner;  // keeps its reference
    P->inner = wrapped;
  }
  // new operator: new workspace sizes, graphs, team plan and setup
  release_state(P);
  team::release(P);
  r = team::plan_problem(P);
  P->setup_done = false;
  P->setup_sig = 0;
  return r;
}

extern "C" cf_err cf_problem_scaling(const cf_problem* P, float* D, float* E, double* sigma, double* rho) {
  if (!P) return fail(CF_E_INVALID, "cf_problem_scaling: NULL problem");
  DevGuard guard(P->device);
  if (sigma) *sigma = P->sigma;
  if (rho) *rho = P->rho;
  if (D) {
    if (P->eq_d) {
      CF_TRY(copy_any(D, P->eq_d, P->m * sizeof(float), P->ctx->stream));
    } else {
      std::vector<float> one(P->m, 1.f);
      CF_TRY(copy_any(D, one.data(), P->m * sizeof(float), P->ctx->stream));
    }
  }
  if (E) {
    if (P->eq_e) {
      CF_TRY(copy_any(E, P->eq_e, P->n * sizeof(float), P->ctx->stream));
    } else {
      std::vector<float> one(P->n, 1.f);
      CF_TRY(copy_any(E, one.data(), P->n * sizeof(float), P->ctx->stream));
    }
  }
  return CF_OK;
}
