// Solver state shared by the solver and the server translation units.
#pragma once

#include <mutex>

#include "internal.cuh"
#include "team.cuh"

namespace cf {

enum CgMode { CG_ITER = 0, CG_SETUP = 1 };

// Device control block of one problem.  The host writes the settings block
// before each launch; everything else is written by kernels.
struct Settings {
  double alpha, eps, eps_inf, cg_tol_rel, cg_tol_exp, cg_tol_min, setup_tol;
  int max_iters, check_interval, cg_max, cg_fixed, setup_cg_max, warm;
};

struct Ctl {
  Settings st;
  double lam;            // Gram shift: CG solves (lam I + A^T A) z = rhs
  double hg, nb, nc;     // h^T g, ||b||, ||c|| (original data)
  double sigma, rho;     // equilibration: b^ = sigma D b, c^ = rho E c (1 without)
  double tau, kappa, w_tau, ut_tau;
  double rr, tol2, alpha_cg, beta_cg;
  double pri, dual, gap, cx, by;
  long long cg_total;
  int k, cg_it, cg_guard, checks, refreshes, status, stop, cg_cont, setup_iters;
  // loop decisions, also set as graph conditions inside a graph
  int cg_go, do_check, do_refresh, outer_go;
  unsigned int red_count;
  long long t_start, t_end;  // team engine: device clock (ns) at the solve's start and end
  int grid_abort;            // grid team: a barrier wait gave up (the solve failed)
};

struct KernelCounts {
  int top = 0, body = 0, cg = 0, check = 0, refresh = 0;
};

// Diagonal row blocks folded out of the graph engine's CG passes (see
// fold_diag_blocks): block b covers rows [r0[b], r0[b] + len[b]) and columns
// [c0[b], c0[b] + len[b]); s holds the (equilibrated) diagonal on its rows,
// gd the sum of s^2 over the blocks covering each column.  nb == 0: none.
struct Fold {
  int nb = 0;
  int64_t r0[kMaxFold] = {}, c0[kMaxFold] = {}, len[kMaxFold] = {};
  const float* s = nullptr;
  const float* gd = nullptr;
};

}  // namespace cf

struct cf_problem {
  cf_ctx* ctx = nullptr;
  int device = 0;
  cf_op* A = nullptr;
  int64_t m = 0, n = 0, z = 0, l = 0;
  std::vector<int64_t> q;
  double nb = 0, nc = 0;
  std::mutex mtx;  // one solve at a time per problem
  // persistent device data
  float *bf = nullptr, *cf = nullptr;
  int64_t nseg = 0, nchunk = 0;
  int32_t *chunk_seg = nullptr;
  int64_t *chunk_r0 = nullptr, *chunk_r1 = nullptr, *seg_head = nullptr;
  int32_t *seg_c0 = nullptr, *seg_nc = nullptr;
  size_t persist_bytes = 0;
  // solver state (allocated on first use, released by release_state)
  void* arena = nullptr;
  size_t state_bytes = 0;
  float *ux, *uy, *vs, *zx, *rhs, *r, *p, *qv, *wy, *t, *zy, *gx, *gy, *cm, *cn, *ws;
  float *gz, *az;  // G z_x and A z_x, carried by the CG updates
  double *part, *chunk_n2, *seg_p0, *seg_nrm, *warm_dev, *out_dev, *uv_dev;
  unsigned int* seg_cnt = nullptr;  // per-segment tickets of the SOC norm
  cf::Ctl* ctl = nullptr;       // device
  cf::Ctl* ctl_host = nullptr;  // pinned mirror
  void* flags_host = nullptr;   // pinned copy of the loop decisions (host-driven mode)
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr, setup_graph = nullptr;
  cudaGraphExec_t exec = nullptr, setup_exec = nullptr;
  cf::KernelCounts kc, skc;
  bool setup_done = false;
  int setup_iters_last = 0;
  int64_t setup_ns_last = 0;
  // per-call bookkeeping between launch and finish
  double *x_out = nullptr, *y_out = nullptr, *s_out = nullptr, *uv_out = nullptr;
  int64_t t_launch = 0;
  bool ran_setup = false;
  // team engine
  cf::team::Plan plan;            // flattened operator (plan.ok: supported)
  cf::team::Term* team_terms = nullptr;  // device copy of plan.fwd, adj, adj_m
  float* team_scratch = nullptr;  // adjoint dense partials (in the state arena)
  void* team_buf = nullptr;       // device launch table of solo launches
  void* team_buf_host = nullptr;  // pinned staging of that table
  void* grid_buf = nullptr;       // grid team: barrier words and partial sums
  int setup_sig = 0;              // program that computed g: 0 none, 1 graph, >= 2 team
  int last_engine = 0;            // CF_ENGINE_GRAPH, CF_ENGINE_TEAM or CF_ENGINE_GRID
  int64_t team_launches = 0;      // kernels attributed to this problem's last solve
  // equilibration (cone_problem_equilibrate): the solver's A is then
  // diag(D) A_orig diag(E), bf / cf hold sigma D b / rho E c
  float* eq = nullptr;            // one allocation: D, 1/D, E, 1/E
  float *eq_d = nullptr, *eq_dinv = nullptr, *eq_e = nullptr, *eq_einv = nullptr;
  double sigma = 1.0, rho = 1.0;
  cf_op* A_orig = nullptr;
  // mixed-precision refinement: the operator the ADMM iterations' CG steps
  // apply (nullptr: A); equilibrated, diag(D) inner diag(E) with the user's
  // operator kept in inner_orig
  cf_op* inner = nullptr;
  cf_op* inner_orig = nullptr;
  // graph engine: diagonal row blocks of A folded out of the CG passes
  // (planned with the state; s and gd live in the state arena)
  cf::Fold fold;
  std::vector<uint8_t> fold_skip;
  float *fold_s = nullptr, *fold_gd = nullptr;
};

namespace cf {
size_t problem_state_bytes(const cf_problem* p);
// Workspace floats of every operator the solver applies (A and inner).
size_t solver_ws_floats(const cf_problem* p);
cf_err ensure_state(cf_problem* p);
void release_state(cf_problem* p);
// join_ctx: make the context stream wait for this solve right away (single
// solves); batches join after launching every problem, servers never do.
cf_err solve_launch(cf_problem* p, const cf_settings* st, double* x, double* y, double* s,
                    const double* warm_uv, double* uv_out, bool join_ctx = true);
cf_err solve_finish(cf_problem* p, cf_info* info);
bool settings_valid(const cf_settings* st, std::string* why);
void write_settings(cf_problem* p, const cf_settings* st, bool warm);
// Engine a solve of p with st runs on (CF_ENGINE_GRAPH, CF_ENGINE_TEAM or
// CF_ENGINE_GRID), or CF_E_INVALID when st asks for a team program and p is
// not supported.
cf_err pick_engine(cf_problem* p, const cf_settings* st, int* engine, bool in_batch = false);
namespace team {
// Flattens p's operator (at problem creation) and uploads the term lists.
cf_err plan_problem(cf_problem* p);
size_t scratch_floats(const cf_problem* p);
cf_err solo_launch(cf_problem* p, const cf_settings* st, const double* warm_uv, bool join_ctx);
// One cooperative launch in which every CTA (one per SM) carries p's solve.
cf_err grid_launch(cf_problem* p, const cf_settings* st, const double* warm_uv, bool join_ctx);
// Launches every problem of `probs` (all on the team engine, one context) in
// one persistent kernel; each problem's stream is made to wait for it and
// then copies the control block back and records ev_out.
cf_err batch_launch(const std::vector<cf_problem*>& probs, const cf_settings* st);
void release(cf_problem* p);
}  // namespace team
int64_t now_ns();
}  // namespace cf
