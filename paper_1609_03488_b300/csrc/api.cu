// Context, error reporting, copies and defaults of the C ABI.
#include <cstdio>
#include <cstring>

#include "internal.cuh"

namespace cf {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

cf_err fail(cf_err code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

cf_err cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  cudaGetLastError();  // clear a non-sticky error
  g_last_error = buf;
  return CF_E_CUDA;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stream-ordered copy between any host/device addresses; returns after the
// copy finished when either side is host memory, so the caller may reuse it.
cf_err copy_any(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return CF_OK;
  CF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  if (!is_device_ptr(dst) || !is_device_ptr(src)) CF_CUDA(cudaStreamSynchronize(s));
  return CF_OK;
}

}  // namespace cf

using namespace cf;

extern "C" {

void cf_settings_default(cf_settings* s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->eps = 1e-4;
  s->eps_infeas = 1e-4;
  s->alpha = 1.5;
  s->max_iters = 100000;
  s->check_interval = 10;
  s->cg_max_iters = 50;
  s->cg_fixed_iters = 0;
  s->cg_tol_rel = 1.0;
  s->cg_tol_exp = 1.5;
  s->cg_tol_min = 1e-9;
  s->setup_cg_max_iters = 2000;
  s->setup_cg_tol = 1e-7;
  s->engine = CF_ENGINE_AUTO;
}

cf_err cf_ctx_create(int device, void* cuda_stream, cf_ctx** out) {
  if (!out) return fail(CF_E_INVALID, "cf_ctx_create: NULL out");
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    return fail(CF_E_CUDA, std::string("cf_ctx_create: no CUDA device: ") + cudaGetErrorString(e));
  }
  if (device < 0 || device >= count) return fail(CF_E_INVALID, "cf_ctx_create: bad device index");
  CF_CUDA(cudaSetDevice(device));
  cf_ctx* c = new cf_ctx();
  c->device = device;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
    }
    c->own_stream = true;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  c->sm_count = sms;
  c->sched = default_schedule();
  *out = c;
  return CF_OK;
}

void cf_ctx_destroy(cf_ctx* c) {
  if (!c) return;
  if (c->own_stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  delete c;
}

int cf_ctx_sm_count(const cf_ctx* c) { return c ? c->sm_count : 0; }

cf_err cf_ctx_get_schedule(const cf_ctx* c, cf_schedule* out) {
  if (!c || !out) return fail(CF_E_INVALID, "cf_ctx_get_schedule: NULL argument");
  std::lock_guard<std::mutex> lk(const_cast<cf_ctx*>(c)->sched_mu);
  *out = c->sched;
  return CF_OK;
}

cf_err cf_ctx_set_schedule(cf_ctx* c, const cf_schedule* s) {
  if (!c || !s) return fail(CF_E_INVALID, "cf_ctx_set_schedule: NULL argument");
  std::string why;
  if (!schedule_valid(*s, &why)) return fail(CF_E_INVALID, "cf_ctx_set_schedule: " + why);
  std::lock_guard<std::mutex> lk(c->sched_mu);
  c->sched = *s;
  return CF_OK;
}

const char* cf_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
