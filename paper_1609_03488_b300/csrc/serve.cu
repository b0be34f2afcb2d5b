// Serving loop: continuous batching of cone-program solves on one GPU.
//
// A host thread admits queued requests in arrival order as soon as a slot is
// free and the request's device memory fits in the budget, launches each
// admitted solve (one CUDA graph on the problem's own stream, so admitted
// solves of different sizes run concurrently and finish independently),
// polls running solves, and retires them.  A problem's iterates, operator and
// setup stay resident between requests; idle resident problems are evicted
// (least recently used first) when a new one needs the memory.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "solver.cuh"

using namespace cf;

namespace {

enum ReqState { Q_QUEUED, Q_RUNNING, Q_DONE };

struct Req {
  cf_ticket id;
  cf_problem* p;
  cf_settings st;
  ReqState state = Q_QUEUED;
  cf_err err = CF_OK;
  cf_info info{};
  std::vector<double> x, y, s;
  int64_t t_submit = 0, t_start = 0;
  std::unique_lock<std::mutex> plock;
};

size_t problem_bytes(cf_problem* p) {
  return problem_state_bytes(p) + p->persist_bytes + op_tree_bytes(p->A) +
         (p->inner ? op_tree_bytes(p->inner) : 0);
}

}  // namespace

struct cf_server {
  cf_ctx* ctx = nullptr;
  size_t budget = 0;
  int max_slots = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::vector<Req*> running;
  std::unordered_map<cf_ticket, Req*> all;
  std::vector<cf_problem*> resident;  // LRU order: front = oldest
  // bytes charged to `used` for each resident problem, recorded when it was
  // admitted; eviction returns exactly this amount even if the problem's
  // size changed since (equilibration or an inner operator set in between)
  std::unordered_map<cf_problem*, size_t> charged;
  size_t used = 0;
  bool stopping = false;
  cf_ticket next = 1;
  std::thread th;

  bool is_running(cf_problem* p) {
    for (Req* r : running)
      if (r->p == p) return true;
    return false;
  }
  bool is_resident(cf_problem* p) {
    return std::find(resident.begin(), resident.end(), p) != resident.end();
  }
  void touch(cf_problem* p) {
    auto it = std::find(resident.begin(), resident.end(), p);
    if (it != resident.end()) resident.erase(it);
    resident.push_back(p);
  }

  // Drop p from the resident set, returning the bytes it was charged.
  void uncharge(cf_problem* p) {
    auto it = std::find(resident.begin(), resident.end(), p);
    if (it != resident.end()) resident.erase(it);
    auto c = charged.find(p);
    if (c != charged.end()) {
      used -= std::min(used, c->second);
      charged.erase(c);
    }
  }

  // Make room for p; true if it fits (after evicting idle residents).  A
  // resident problem whose size changed since it was charged is re-charged
  // at its current size.
  bool make_room(cf_problem* p) {
    const size_t need = problem_bytes(p);
    if (is_resident(p)) {
      auto c = charged.find(p);
      if (c != charged.end() && c->second == need) return true;
      uncharge(p);                     // its state stays allocated until re-admitted
    }
    while (used + need > budget) {
      cf_problem* victim = nullptr;
      for (cf_problem* q : resident)
        if (!is_running(q)) {
          victim = q;
          break;
        }
      if (!victim) return false;
      uncharge(victim);
      std::lock_guard<std::mutex> lk(victim->mtx);
      release_state(victim);
    }
    return true;
  }

  void admit(std::unique_lock<std::mutex>& lk) {
    (void)lk;
    while (!queue.empty() && (int)running.size() < max_slots) {
      Req* r = queue.front();
      if (is_running(r->p)) break;  // same problem: wait for its previous request
      if (!make_room(r->p)) break;
      queue.pop_front();
      if (!is_resident(r->p)) {
        const size_t b = problem_bytes(r->p);
        charged[r->p] = b;
        used += b;
      }
      touch(r->p);
      r->plock = std::unique_lock<std::mutex>(r->p->mtx);
      cudaSetDevice(ctx->device);
      const int64_t n = r->p->n, m = r->p->m;
      r->x.resize(n);
      r->y.resize(m);
      r->s.resize(m);
      r->t_start = now_ns();
      r->err = solve_launch(r->p, &r->st, r->x.data(), r->y.data(), r->s.data(), nullptr, nullptr,
                            /*join_ctx=*/false);
      if (r->err != CF_OK) {
        r->plock.unlock();
        r->state = Q_DONE;
        cv_done.notify_all();
        continue;
      }
      r->state = Q_RUNNING;
      running.push_back(r);
    }
  }

  void retire() {
    for (size_t i = 0; i < running.size();) {
      Req* r = running[i];
      cudaError_t q = cudaStreamQuery(r->p->stream);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (q != cudaSuccess) cudaGetLastError();
      r->err = solve_finish(r->p, &r->info);
      r->info.queue_ns = r->t_start - r->t_submit;
      r->plock.unlock();
      r->state = Q_DONE;
      running.erase(running.begin() + i);
      cv_done.notify_all();
    }
  }

  void loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      admit(lk);
      retire();
      if (stopping && running.empty() && queue.empty()) break;
      if (running.empty() && (queue.empty() || stopping))
        cv_work.wait(lk);
      else
        cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
};

extern "C" {

cf_err serve_create(cf_ctx* ctx, size_t mem_budget_bytes, int32_t max_slots, cf_server** out) {
  if (!ctx || !out || max_slots < 1 || mem_budget_bytes == 0)
    return fail(CF_E_INVALID, "serve_create: bad arguments");
  cf_server* s = new cf_server();
  s->ctx = ctx;
  s->budget = mem_budget_bytes;
  s->max_slots = max_slots;
  s->th = std::thread([s]() { s->loop(); });
  *out = s;
  return CF_OK;
}

cf_err serve_submit(cf_server* s, cf_problem* p, const cf_settings* st, cf_ticket* out) {
  if (!s || !p || !out) return fail(CF_E_INVALID, "serve_submit: bad arguments");
  cf_settings cs;
  if (st)
    cs = *st;
  else
    cf_settings_default(&cs);
  std::string why;
  if (!settings_valid(&cs, &why)) return fail(CF_E_INVALID, "serve_submit: " + why);
  // a grid-engine solve holds every SM: served solves overlap, so they run
  // on the other programs
  if (cs.engine == CF_ENGINE_GRID) cs.engine = CF_ENGINE_AUTO;
  if (problem_bytes(p) > s->budget) return fail(CF_E_INVALID, "serve_submit: problem exceeds the memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return fail(CF_E_STATE, "serve_submit: server is stopping");
  if (s->queue.size() >= 4096) return fail(CF_E_BUSY, "serve_submit: queue full");
  Req* r = new Req();
  r->id = s->next++;
  r->p = p;
  r->st = cs;
  r->t_submit = now_ns();
  s->queue.push_back(r);
  s->all[r->id] = r;
  *out = r->id;
  s->cv_work.notify_all();
  return CF_OK;
}

cf_err serve_wait(cf_server* s, cf_ticket t, int64_t timeout_ns, double* x, double* y, double* sv,
                  cf_info* info) {
  if (!s) return fail(CF_E_INVALID, "serve_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(t);
  if (it == s->all.end()) return fail(CF_E_STATE, "serve_wait: unknown ticket");
  Req* r = it->second;
  auto done = [&]() { return r->state == Q_DONE; };
  if (timeout_ns < 0)
    s->cv_done.wait(lk, done);
  else if (!s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done))
    return fail(CF_E_TIMEOUT, "serve_wait: timed out");
  if (x && !r->x.empty()) std::copy(r->x.begin(), r->x.end(), x);
  if (y && !r->y.empty()) std::copy(r->y.begin(), r->y.end(), y);
  if (sv && !r->s.empty()) std::copy(r->s.begin(), r->s.end(), sv);
  if (info) *info = r->info;
  cf_err e = r->err;
  s->all.erase(it);
  delete r;
  return e;
}

void serve_destroy(cf_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    for (Req* r : s->queue) {
      r->state = Q_DONE;
      r->info.status = CF_CANCELLED;
    }
    s->queue.clear();
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

}  // extern "C"
