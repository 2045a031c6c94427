// extern "C" entry points declared in include/sor.h.  Argument checking and
// device bookkeeping only; the work happens in sor_runtime.cu / sor_batch.cu.
#include <cmath>
#include <cstring>
#include <new>

#include "sor_runtime.h"

using namespace sorgb;

struct sor_ctx {
  Ctx impl;
};

namespace {

// Makes ctx->device current for the duration of an API call and restores the
// caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    ok = cudaSetDevice(dev) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

double sor_omega_opt(int32_t n) {
  if (n < 1) return 0.0;
  return 2.0 / (1.0 + std::sin(M_PI / (double)(n + 1)));
}

const char* sor_status_string(int32_t s) {
  switch (s) {
    case SOR_OK: return "ok";
    case SOR_NOT_READY: return "not ready";
    case SOR_ERR_INVALID_ARG: return "invalid argument";
    case SOR_ERR_BUDGET: return "over the device-memory budget";
    case SOR_ERR_OOM: return "out of memory";
    case SOR_ERR_CUDA: return "CUDA error";
    case SOR_ERR_TIMEOUT: return "timed out";
    case SOR_ERR_INTERNAL: return "internal error";
    case SOR_ERR_UNKNOWN_TICKET: return "unknown ticket";
    case SOR_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

sor_status sor_create(sor_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream, sor_alloc_fn alloc,
                      sor_free_fn free_, void* alloc_user) {
  if (!out) return SOR_ERR_INVALID_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (free_ == nullptr)) return SOR_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return SOR_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return SOR_ERR_INVALID_ARG;
  DeviceGuard dg(device);
  if (!dg.ok) return SOR_ERR_CUDA;
  sor_ctx* h = new (std::nothrow) sor_ctx();
  if (!h) return SOR_ERR_OOM;
  Ctx* c = &h->impl;
  c->device = device;
  c->alloc = alloc;
  c->free_ = free_;
  c->alloc_user = alloc_user;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SOR_ERR_CUDA;
  }
  c->sm_count = prop.multiProcessorCount;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SOR_ERR_CUDA;
  }
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return SOR_ERR_CUDA;
    }
    c->own_stream = true;
  }
  load_tune_cache(c);
  *out = h;
  return SOR_OK;
}

sor_status sor_destroy(sor_ctx* h) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  {
    DeviceGuard dg(c->device);
    batch_shutdown(c);
    {
      std::lock_guard<std::mutex> g(c->solve_mu);
      if (c->stream) cudaStreamSynchronize(c->stream);
      release_solve_workspace(c);
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  }
  delete h;
  return SOR_OK;
}

static sor_status check_inputs(Ctx* c, const sor_params* params, const double* u0, const double* f, double* u_out,
                               Plan* plan) {
  if (!params || !u0 || !u_out) {
    c->set_error("params, u0 and u_out must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  std::string why;
  sor_status rs = make_plan(params, f != nullptr, plan, &why);
  if (rs != SOR_OK) c->set_error(why);
  return rs;
}

sor_status sor_solve(sor_ctx* h, const sor_params* params, const double* u0, const double* f, double* u_out,
                     sor_result* res) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  Plan plan;
  sor_status rs = check_inputs(c, params, u0, f, u_out, &plan);
  if (rs != SOR_OK) return rs;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  return solve_blocking(c, plan, u0, f, u_out, res);
}

sor_status sor_solve3d(sor_ctx* h, const sor_params* params, const double* u0, const double* f, double* u_out,
                       sor_result* res) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  std::lock_guard<std::mutex> g(c->solve_mu);
  return solve3d_blocking(c, params, u0, f, u_out, res);
}

sor_status sor_solve9(sor_ctx* h, const sor_params* params, const double* u0, const double* f, double* u_out,
                      sor_result* res) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  std::lock_guard<std::mutex> g(c->solve_mu);
  return solve9_blocking(c, params, u0, f, u_out, res);
}

sor_status sor_solve_block(sor_ctx* h, const sor_params* params, int32_t block_rows, int32_t block_cols,
                           const double* u0, const double* f, double* u_out, sor_result* res) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  std::lock_guard<std::mutex> g(c->solve_mu);
  return solve_block_blocking(c, params, block_rows, block_cols, u0, f, u_out, res);
}

sor_status sor_diag_flow_wait(sor_ctx* h, int polls, int preset, int* timed_out) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  std::lock_guard<std::mutex> g(c->solve_mu);
  return diag_flow_wait(c, polls, preset, timed_out);
}

sor_status sor_diag_fp64_rate(sor_ctx* h, int kind, double* ops_per_s) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  std::lock_guard<std::mutex> g(c->solve_mu);
  return diag_fp64_rate(c, kind, ops_per_s);
}

sor_status sor_diag_bounds(sor_ctx* h, int* fired) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  std::lock_guard<std::mutex> g(c->solve_mu);
  return diag_bounds(c, fired);
}

sor_status sor_batch_submit(sor_ctx* h, const sor_params* params, const double* u0, const double* f, double* u_out,
                            uint64_t* ticket) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  if (!ticket) {
    c->set_error("ticket must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  Plan plan;
  sor_status rs = check_inputs(c, params, u0, f, u_out, &plan);
  if (rs != SOR_OK) return rs;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  return batch_submit(c, plan, u0, f, u_out, ticket);
}

sor_status sor_batch_submit3d(sor_ctx* h, const sor_params* params, const double* u0, const double* f,
                              double* u_out, uint64_t* ticket) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  DeviceGuard dg(c->device);
  if (!dg.ok) return SOR_ERR_CUDA;
  return batch_submit3d(c, params, u0, f, u_out, ticket);
}

sor_status sor_poll(sor_ctx* h, uint64_t ticket, sor_result* res) {
  if (!h) return SOR_ERR_INVALID_ARG;
  return batch_poll(&h->impl, ticket, 0.0, res);
}

sor_status sor_wait(sor_ctx* h, uint64_t ticket, double timeout_s, sor_result* res) {
  if (!h) return SOR_ERR_INVALID_ARG;
  if (std::isnan(timeout_s)) return SOR_ERR_INVALID_ARG;
  if (timeout_s == 0.0) timeout_s = 1e-9;
  return batch_poll(&h->impl, ticket, timeout_s, res);
}

sor_status sor_set_option(sor_ctx* h, int32_t option, int64_t value) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  if (value < 0 || value > (1 << 30)) return SOR_ERR_INVALID_ARG;
  const int v = (int)value;
  switch (option) {
    case SOR_OPT_TIMING: c->opt_timing = v ? 1 : 0; return SOR_OK;
    case SOR_OPT_GRAPHS: c->opt_graphs = v ? 1 : 0; return SOR_OK;
    case SOR_OPT_CHUNK: c->opt_chunk = v; return SOR_OK;
    case SOR_OPT_TEMPORAL_DEPTH: c->opt_tdepth = v; return SOR_OK;
    case SOR_OPT_AUTOTUNE: c->opt_autotune = v ? 1 : 0; return SOR_OK;
    case SOR_OPT_BATCH_MAX_SLOTS: c->opt_max_slots = v; return SOR_OK;
    case SOR_OPT_CLUSTER:
      if (v < 0 || v > 3) return SOR_ERR_INVALID_ARG;
      c->opt_cluster = v;
      return SOR_OK;
    case SOR_OPT_FAST_CHAIN: c->opt_fast_chain = v ? 1 : 0; return SOR_OK;
    case SOR_OPT_FUSED_KERNEL:
      if (v > 2) return SOR_ERR_INVALID_ARG;
      c->opt_fused_kernel = v;
      return SOR_OK;
    case SOR_OPT_BATCH_PLAIN_STEP:
      if (v > 4096) return SOR_ERR_INVALID_ARG;
      c->opt_plain_step = v;
      return SOR_OK;
    case SOR_OPT_CUBE_DEPTH:
      if (v < 0 || v > 2) return SOR_ERR_INVALID_ARG;
      c->opt_cube_depth = v;
      return SOR_OK;
    case SOR_OPT_BLOCK_CHAIN:
      if (v > (1 << 20)) return SOR_ERR_INVALID_ARG;
      c->opt_block_chain = v;
      return SOR_OK;
    default: return SOR_ERR_INVALID_ARG;
  }
}

sor_status sor_get_option(sor_ctx* h, int32_t option, int64_t* value) {
  if (!h || !value) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  switch (option) {
    case SOR_OPT_TIMING: *value = c->opt_timing.load(); return SOR_OK;
    case SOR_OPT_GRAPHS: *value = c->opt_graphs.load(); return SOR_OK;
    case SOR_OPT_CHUNK: *value = c->opt_chunk.load(); return SOR_OK;
    case SOR_OPT_TEMPORAL_DEPTH: *value = c->opt_tdepth.load(); return SOR_OK;
    case SOR_OPT_AUTOTUNE: *value = c->opt_autotune.load(); return SOR_OK;
    case SOR_OPT_BATCH_MAX_SLOTS: *value = c->opt_max_slots.load(); return SOR_OK;
    case SOR_OPT_CLUSTER: *value = c->opt_cluster.load(); return SOR_OK;
    case SOR_OPT_FAST_CHAIN: *value = c->opt_fast_chain.load(); return SOR_OK;
    case SOR_OPT_FUSED_KERNEL: *value = c->opt_fused_kernel.load(); return SOR_OK;
    case SOR_OPT_BATCH_PLAIN_STEP: *value = c->opt_plain_step.load(); return SOR_OK;
    case SOR_OPT_CUBE_DEPTH: *value = c->opt_cube_depth.load(); return SOR_OK;
    case SOR_OPT_BLOCK_CHAIN: *value = c->opt_block_chain.load(); return SOR_OK;
    default: return SOR_ERR_INVALID_ARG;
  }
}

sor_status sor_get_stats(sor_ctx* h, sor_stats* out) {
  if (!h || !out) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  {
    std::lock_guard<std::mutex> g(c->stats_mu);
    *out = c->stats;
  }
  {
    std::lock_guard<std::mutex> g(c->mem_mu);
    out->bytes_reserved = c->reserved;
    out->bytes_peak = c->peak;
  }
  return SOR_OK;
}

sor_status sor_reset_stats(sor_ctx* h) {
  if (!h) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  std::lock_guard<std::mutex> g(c->stats_mu);
  std::memset(&c->stats, 0, sizeof(c->stats));
  return SOR_OK;
}

sor_status sor_last_error(sor_ctx* h, char* buf, size_t len) {
  if (!h || !buf || len == 0) return SOR_ERR_INVALID_ARG;
  Ctx* c = &h->impl;
  std::lock_guard<std::mutex> g(c->err_mu);
  std::strncpy(buf, c->last_error.c_str(), len - 1);
  buf[len - 1] = '\0';
  return SOR_OK;
}

}  // extern "C"
