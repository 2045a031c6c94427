// Continuous-batching scheduler.
//
// One host thread per context owns the admitted requests ("slots").  Each
// scheduler step
//   1. admits queued requests in arrival order while their device memory fits
//      the context budget (and the slot cap), copying and packing their inputs;
//   2. launches one step over every active slot at once: the kernels walk a
//      device-side tile table that covers all slots of a kind, so grids of
//      different sizes share each launch (a defect-correction step is a
//      residual pass plus the inner sweeps; a plain step is a fixed number of
//      red-black iterations);
//   3. reads back the per-slot state (the only device->host sync of a step)
//      and retires finished slots: unpack, copy to the caller, free memory.
// Requests that arrive while others run are admitted at the next step, so
// their work overlaps on the device with the slots already running.  Slots
// never interact: every slot's arithmetic is the same as a lone solve.
#include <algorithm>
#include <cstring>
#include <sstream>
#include <unordered_set>

#include "sor_runtime.h"

namespace sorgb {

#define SOR_BCK(expr)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      std::ostringstream os_;                                                                      \
      os_ << #expr << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
      c->set_error(os_.str());                                                                     \
      return SOR_ERR_CUDA;                                                                         \
    }                                                                                              \
  } while (0)

// Iterations per scheduler step for plain slots: tried online in this order,
// kPlainTrialRounds rounds each, and the one with the highest update rate is
// kept (SOR_OPT_BATCH_PLAIN_STEP fixes it instead).
static constexpr int kPlainStepCand[] = {8, 16, 32, 64};
static constexpr int kPlainCands = 4;
static constexpr int kPlainTrialRounds = 2;
static constexpr int kBatchSegRows = 64;    // output rows per fused-sweep tile (many slots fill the GPU)

struct Batcher {
  Ctx* c = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;      // wakes the scheduler
  std::condition_variable done_cv; // wakes sor_wait callers
  std::deque<std::unique_ptr<Request>> queue;
  std::unordered_map<uint64_t, Completed> completed;
  std::unordered_set<uint64_t> pending;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool failed = false;
  sor_status fail_status = SOR_OK;

  // scheduler-thread state
  cudaStream_t stream = nullptr;
  std::vector<std::unique_ptr<Request>> slots;  // index = slot id (nullptr = free)
  int cap = 0;
  SlotDesc* d_desc = nullptr;
  SlotState* d_state = nullptr;
  SlotState* h_state = nullptr;  // pinned
  Tile* d_tiles = nullptr;       // [refine sweep | refine resid | plain64 | plain32 | retire]
  size_t tiles_cap = 0;
  int nt_refine = 0, nt_p64 = 0, nt_p32 = 0, nt_reftb = 0;
  size_t off_p64 = 0, off_p32 = 0, off_reftb = 0;
  int max_inner = 1;
  int tdepth = 0;             // fused iterations of the refine sweeps (1 = unfused; 0 = not chosen yet),
                              // fixed for the scheduler's lifetime so every slot's buffers stay consistent
  int fkind = 0;              // kernel family of the fused refine sweeps (FusedKind)
  size_t live_tiles = 0;      // tiles in the table at the last rebuild
  size_t dead_tiles = 0;      // of those, tiles of slots finished since
  bool any_resid_stop = false;
  uint64_t version = 0;       // bumps when the active set changes
  uint64_t graph_version = ~0ull;
  int graph_steps = 0;
  int graph_plain_step = 0;
  int plain_step = 0;                       // tuned iterations per step of plain slots (0: trial running)
  int plain_trial = 0;                      // trial rounds done
  double plain_rate[kPlainCands] = {};      // plain lattice updates per second, summed per candidate
  int plain_rounds[kPlainCands] = {};
  cudaGraphExec_t graph = nullptr;
  size_t reserved_tables = 0;

  // cube requests: solved whole, each by one of up to kCubeWorkers threads on
  // its own stream, concurrently with the plate steps and with each other
  std::deque<std::unique_ptr<Request>> cube_queue;
  std::vector<std::thread> cube_workers;
  int cube_busy = 0;
};

static constexpr int kCubeWorkers = 4;

static sor_status ensure_tables(Batcher* b, int cap, size_t ntiles) {
  Ctx* c = b->c;
  if (cap > b->cap) {
    int nc = std::max(cap, std::max(16, b->cap * 2));
    SlotDesc* nd = (SlotDesc*)ctx_dev_alloc(c, sizeof(SlotDesc) * nc);
    SlotState* ns = (SlotState*)ctx_dev_alloc(c, sizeof(SlotState) * nc);
    SlotState* nh = nullptr;
    if (!nd || !ns || cudaMallocHost(&nh, sizeof(SlotState) * nc) != cudaSuccess) {
      cudaGetLastError();
      ctx_dev_free(c, nd);
      ctx_dev_free(c, ns);
      c->set_error("batch table allocation failed");
      return SOR_ERR_OOM;
    }
    SOR_BCK(cudaMemsetAsync(ns, 0, sizeof(SlotState) * nc, b->stream));
    if (b->cap) {
      SOR_BCK(cudaMemcpyAsync(nd, b->d_desc, sizeof(SlotDesc) * b->cap, cudaMemcpyDeviceToDevice, b->stream));
      SOR_BCK(cudaMemcpyAsync(ns, b->d_state, sizeof(SlotState) * b->cap, cudaMemcpyDeviceToDevice, b->stream));
      SOR_BCK(cudaStreamSynchronize(b->stream));
    }
    ctx_dev_free(c, b->d_desc);
    ctx_dev_free(c, b->d_state);
    if (b->h_state) cudaFreeHost(b->h_state);
    b->d_desc = nd;
    b->d_state = ns;
    b->h_state = nh;
    b->cap = nc;
    b->slots.resize(nc);
  }
  if (ntiles > b->tiles_cap) {
    size_t nc = std::max(ntiles, b->tiles_cap * 2);
    Tile* nt = (Tile*)ctx_dev_alloc(c, sizeof(Tile) * nc);
    if (!nt) {
      c->set_error("batch tile table allocation failed");
      return SOR_ERR_OOM;
    }
    SOR_BCK(cudaStreamSynchronize(b->stream));
    ctx_dev_free(c, b->d_tiles);
    b->d_tiles = nt;
    b->tiles_cap = nc;
  }
  return SOR_OK;
}

// Rebuild the tile table after the active set changed.
static sor_status rebuild_tiles(Batcher* b) {
  std::vector<Tile> ref, p64, p32, reftb;
  b->max_inner = 1;
  b->any_resid_stop = false;
  const int T = b->tdepth;  // chosen when the first slot was activated
  for (size_t s = 0; s < b->slots.size(); ++s) {
    Request* r = b->slots[s].get();
    if (!r) continue;
    const Layout& L = r->buf.L;
    const size_t before = ref.size() + p64.size() + p32.size() + reftb.size();
    if (r->plan.kind == kRefine) {
      build_tiles(L, (int)s, &ref, nullptr);
      if (T > 1)
        build_tiles(L, (int)s, &reftb, nullptr, fused_out_rows(b->fkind, L.n, T, b->c->sm_count, kBatchSegRows),
                    fused_out_cols(b->fkind, T));
      b->max_inner = std::max(b->max_inner, r->plan.inner);
    } else if (r->plan.kind == kPlain64) {
      build_tiles(L, (int)s, &p64, nullptr);
      if (r->plan.stop == kStopResid) b->any_resid_stop = true;
    } else {
      build_tiles(L, (int)s, &p32, nullptr);
      if (r->plan.stop == kStopResid) b->any_resid_stop = true;
    }
    r->ntiles = ref.size() + p64.size() + p32.size() + reftb.size() - before;
  }
  const size_t total = ref.size() + p64.size() + p32.size() + reftb.size();
  b->live_tiles = total;
  b->dead_tiles = 0;
  sor_status rs = ensure_tables(b, (int)b->slots.size(), total + 1);
  if (rs != SOR_OK) return rs;
  std::vector<Tile> all;
  all.reserve(total);
  all.insert(all.end(), ref.begin(), ref.end());
  all.insert(all.end(), p64.begin(), p64.end());
  all.insert(all.end(), p32.begin(), p32.end());
  all.insert(all.end(), reftb.begin(), reftb.end());
  b->nt_refine = (int)ref.size();
  b->nt_p64 = (int)p64.size();
  b->nt_p32 = (int)p32.size();
  b->nt_reftb = (int)reftb.size();
  b->off_p64 = ref.size();
  b->off_p32 = ref.size() + p64.size();
  b->off_reftb = ref.size() + p64.size() + p32.size();
  Ctx* c = b->c;
  if (!all.empty())
    SOR_BCK(cudaMemcpyAsync(b->d_tiles, all.data(), sizeof(Tile) * all.size(), cudaMemcpyHostToDevice, b->stream));
  b->version++;
  return SOR_OK;
}

// The launches of one scheduler step over every active slot.
// Iterations per scheduler step of plain slots this round.
static int plain_step_len(const Batcher* b) {
  const int opt = b->c->opt_plain_step.load();
  if (opt > 0) return opt;
  if (b->plain_step > 0) return b->plain_step;
  return kPlainStepCand[std::min(kPlainCands - 1, b->plain_trial / kPlainTrialRounds)];
}

static sor_status enqueue_step(Batcher* b) {
  Ctx* c = b->c;
  cudaStream_t s = b->stream;
  if (b->nt_refine) {
    // residual pass: tests, writes r~; before it, the corrections of the
    // previous step (each slot's from the buffer its own inner sweep count
    // ends in), unless the fused sweeps already applied them (each slot's
    // last inner launch adds its d to u)
    const bool fix = b->tdepth > 1 && fused_corrects(b->fkind);
    SOR_BCK(launch_resid(fix ? kResidRefine64Fixed : kResidRefine64, b->d_desc, b->d_state, b->d_tiles,
                         b->nt_refine, 0, kDbufPerSlot, s));
    if (b->tdepth > 1) {
      const Tile* t = b->d_tiles + b->off_reftb;
      for (int j = 0, sw = 0; sw < b->max_inner; ++j, sw += b->tdepth) {
        const int nt = std::min(b->tdepth, b->max_inner - sw);
        SOR_BCK(launch_fused(b->fkind, true, b->tdepth, b->d_desc, b->d_state, t, b->nt_reftb, 0, nt,
                             (j % 2 == 0) ? 1 : 0, sw, s, fix));
      }
    } else {
      for (int sw = 0; sw < b->max_inner; ++sw) {
        SOR_BCK(launch_sweep(kSweepInner32, b->d_desc, b->d_state, b->d_tiles, b->nt_refine, 0, 0, sw, s));
        SOR_BCK(launch_sweep(kSweepInner32, b->d_desc, b->d_state, b->d_tiles, b->nt_refine, 0, 1, sw, s));
      }
    }
  }
  for (int kind = 0; kind < 2; ++kind) {
    const int nt = kind == 0 ? b->nt_p64 : b->nt_p32;
    if (!nt) continue;
    const Tile* t = b->d_tiles + (kind == 0 ? b->off_p64 : b->off_p32);
    const SweepKind sk = kind == 0 ? kSweepPlain64 : kSweepPlain32;
    const int iters = plain_step_len(b);
    for (int it = 0; it < iters; ++it) {
      SOR_BCK(launch_sweep(sk, b->d_desc, b->d_state, t, nt, 0, 0, 0, s));
      SOR_BCK(launch_sweep(sk, b->d_desc, b->d_state, t, nt, 0, 1, 0, s));
      if (b->any_resid_stop)
        SOR_BCK(launch_resid(kind == 0 ? kResidCheck64 : kResidCheck32, b->d_desc, b->d_state, t, nt, 0, 0, s));
    }
  }
  return SOR_OK;
}

// Steps replayed per host round trip: with little work active a step is a few
// short launches, so several of them go into one graph (slots that finish
// mid-way skip the rest on the device) and the host polls less often.
static int steps_per_round(const Batcher* b) {
  double cells = 0.0, sweeps = 0.0;
  for (const auto& r : b->slots)
    if (r) {
      cells += (double)r->plan.n * r->plan.n;
      sweeps = std::max(sweeps, (double)(r->plan.kind == kRefine ? r->plan.inner : plain_step_len(b)));
    }
  const double step_s = cells * sweeps / 4.0e11 + 40e-6;  // rough cost of one step
  return (int)std::max(1.0, std::min(16.0, std::floor(400e-6 / step_s)));
}

static sor_status run_step(Batcher* b, int* steps_out) {
  Ctx* c = b->c;
  const int m = steps_per_round(b);
  *steps_out = m;
  if (!c->opt_graphs.load()) {
    for (int k = 0; k < m; ++k) {
      sor_status rs = enqueue_step(b);
      if (rs != SOR_OK) return rs;
    }
    return SOR_OK;
  }
  if (b->graph_version != b->version || !b->graph || b->graph_steps != m || b->graph_plain_step != plain_step_len(b)) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    SOR_BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    sor_status rs = SOR_OK;
    for (int k = 0; k < m && rs == SOR_OK; ++k) rs = enqueue_step(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rs != SOR_OK) {
      if (g) cudaGraphDestroy(g);
      return rs;
    }
    SOR_BCK(e);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    SOR_BCK(e);
    b->graph_version = b->version;
    b->graph_steps = m;
    b->graph_plain_step = plain_step_len(b);
  }
  SOR_BCK(cudaGraphLaunch(b->graph, b->stream));
  return SOR_OK;
}


static size_t request_bytes(const Plan& p) {
  const size_t stage = (size_t)(p.n + 2) * (p.n + 2) * 8 + (p.has_f ? (size_t)p.n * p.n * 8 : 0);
  return slot_bytes(p, p.kind == kRefine) + stage;
}

// Allocate, copy and pack one request into slot `s` (scheduler thread).
static sor_status activate(Batcher* b, Request* r, int s) {
  Ctx* c = b->c;
  const Plan& p = r->plan;
  sor_status rs = alloc_slot(c, p, p.kind == kRefine, &r->buf);
  if (rs != SOR_OK) return rs;
  r->stage_bytes = (size_t)(p.n + 2) * (p.n + 2) * 8 + (p.has_f ? (size_t)p.n * p.n * 8 : 0);
  r->d_stage = (double*)ctx_dev_alloc(c, r->stage_bytes);
  if (!r->d_stage) {
    free_slot(c, &r->buf);
    return SOR_ERR_OOM;
  }
  r->slot = s;
  rs = zero_slot(c, p, &r->buf, b->stream);
  if (rs != SOR_OK) return rs;
  const size_t nu = (size_t)(p.n + 2) * (p.n + 2);
  SOR_BCK(cudaMemcpyAsync(r->d_stage, r->u0.data(), nu * 8, cudaMemcpyHostToDevice, b->stream));
  if (p.has_f)
    SOR_BCK(cudaMemcpyAsync(r->d_stage + nu, r->f.data(), (size_t)p.n * p.n * 8, cudaMemcpyHostToDevice, b->stream));
  if (b->tdepth == 0) {
    // the fused refine sweeps, chosen once (outside any capture) for the
    // whole scheduler: the size rule of sor_solve for this first request, or
    // the autotuner's choice for its size bucket if one was made
    Plan probe = p;
    resolve_fused(c, &probe);
    if (c->opt_autotune.load() && c->opt_tdepth.load() == 0 && c->opt_fused_kernel.load() == 0) {
      std::lock_guard<std::mutex> g(c->tune_mu);
      std::ostringstream key;
      int nb = 16;
      while (nb < p.n) nb <<= 1;
      key << nb << " " << 1;
      auto it = c->tuned.find(key.str());
      if (it != c->tuned.end()) {
        probe.fkind = it->second.fkind;
        probe.tdepth = it->second.tdepth;
      }
    }
    if (probe.tdepth > 1 && fused_prepare(probe.fkind, probe.tdepth) != cudaSuccess) {
      cudaGetLastError();
      c->set_error("fused FP32 sweep kernel does not fit");
      return SOR_ERR_CUDA;
    }
    b->fkind = probe.fkind;
    b->tdepth = std::max(1, probe.tdepth);
  }
  fill_desc(p, &r->buf);
  if (p.kind == kRefine) {
    Plan q = p;
    q.tdepth = b->tdepth;
    r->buf.desc.dbuf = refine_dbuf(q);
  }
  SlotState st0 = initial_state(p);
  SOR_BCK(cudaMemcpyAsync(b->d_desc + s, &r->buf.desc, sizeof(SlotDesc), cudaMemcpyHostToDevice, b->stream));
  SOR_BCK(cudaMemcpyAsync(b->d_state + s, &st0, sizeof(SlotState), cudaMemcpyHostToDevice, b->stream));
  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.u0 = r->d_stage;
  pa.f = p.has_f ? r->d_stage + nu : nullptr;
  pa.n = p.n;
  pa.pitch = r->buf.L.pitch;
  const double h = 1.0 / (double)(p.n + 1);
  pa.h2 = h * h;
  pa.fp32 = p.kind != kPlain64;
  const SlotDesc& d = r->buf.desc;
  if (p.kind == kRefine) {
    for (int k = 0; k < 2; ++k)
      for (int col = 0; col < 2; ++col) pa.u[k][col] = d.u[k][col];
    for (int col = 0; col < 2; ++col) pa.g64[col] = (double*)d.g64[col];
  } else {
    for (int col = 0; col < 2; ++col) {
      pa.x[0][col] = d.x[0][col];
      pa.g[col] = d.g[col];
      pa.g64[col] = p.kind == kPlain32 ? (double*)d.g64[col] : nullptr;
    }
  }
  pa.state = b->d_state + s;
  SOR_BCK(launch_pack(pa, b->stream));
  r->u0.clear();
  r->u0.shrink_to_fit();
  r->f.clear();
  r->f.shrink_to_fit();
  return SOR_OK;
}

static void complete(Batcher* b, uint64_t ticket, sor_status st, const sor_result& res) {
  {
    std::lock_guard<std::mutex> g(b->mu);
    b->pending.erase(ticket);
    Completed cp;
    cp.status = st;
    cp.res = res;
    b->completed[ticket] = cp;
  }
  b->done_cv.notify_all();
}

static void release_request(Batcher* b, Request* r) {
  Ctx* c = b->c;
  free_slot(c, &r->buf);
  ctx_dev_free(c, r->d_stage);
  r->d_stage = nullptr;
  ctx_release(c, request_bytes(r->plan));
}

// Retire finished slots: final residual for plain slots, unpack, copy out.
static sor_status retire(Batcher* b, const std::vector<int>& fin) {
  NvtxRange nvtx("sor_retire");
  Ctx* c = b->c;
  cudaStream_t s = b->stream;
  std::vector<Tile> p64, p32;
  for (int sidx : fin) {
    Request* r = b->slots[sidx].get();
    if (r->plan.kind == kPlain64) build_tiles(r->buf.L, sidx, &p64, nullptr);
    if (r->plan.kind == kPlain32) build_tiles(r->buf.L, sidx, &p32, nullptr);
  }
  if (!p64.empty() || !p32.empty()) {
    std::vector<Tile> all(p64);
    all.insert(all.end(), p32.begin(), p32.end());
    Tile* dt = (Tile*)ctx_dev_alloc(c, sizeof(Tile) * all.size());
    if (!dt) return SOR_ERR_OOM;
    SOR_BCK(cudaMemcpyAsync(dt, all.data(), sizeof(Tile) * all.size(), cudaMemcpyHostToDevice, s));
    if (!p64.empty()) SOR_BCK(launch_resid(kResidFinal64, b->d_desc, b->d_state, dt, (int)p64.size(), 0, 0, s));
    if (!p32.empty())
      SOR_BCK(launch_resid(kResidFinal32, b->d_desc, b->d_state, dt + p64.size(), (int)p32.size(), 0, 0, s));
    SOR_BCK(cudaStreamSynchronize(s));
    ctx_dev_free(c, dt);
    for (int sidx : fin)
      SOR_BCK(cudaMemcpyAsync(&b->h_state[sidx], b->d_state + sidx, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR_BCK(cudaStreamSynchronize(s));
  }
  for (int sidx : fin) {
    Request* r = b->slots[sidx].get();
    const SlotState& hs = b->h_state[sidx];
    const Plan& p = r->plan;
    const SlotDesc& d = r->buf.desc;
    double* dout = r->out_on_device ? r->u_out : r->d_stage;
    if (p.kind == kRefine)
      SOR_BCK(launch_unpack(d.u[hs.ubuf][0], d.u[hs.ubuf][1], false, p.n, r->buf.L.pitch, dout, s));
    else
      SOR_BCK(launch_unpack(d.x[hs.xbuf][0], d.x[hs.xbuf][1], p.kind == kPlain32, p.n, r->buf.L.pitch, dout, s));
    if (!r->out_on_device)
      SOR_BCK(cudaMemcpyAsync(r->u_out, dout, (size_t)(p.n + 2) * (p.n + 2) * 8, cudaMemcpyDeviceToHost, s));
  }
  SOR_BCK(cudaStreamSynchronize(s));
  const double t = now_s();
  for (int sidx : fin) {
    std::unique_ptr<Request> r = std::move(b->slots[sidx]);
    const SlotState& hs = b->h_state[sidx];
    sor_result res;
    std::memset(&res, 0, sizeof(res));
    res.iterations = hs.iters;
    res.converged = hs.converged;
    res.outer_steps = r->plan.kind == kRefine ? hs.outer : 0;
    res.final_maxdelta = hs.last_dmax;
    res.final_resid_rel = hs.last_rho;
    res.latency_s = t - r->t_submit;
    res.device_s = 0.0;
    {
      std::lock_guard<std::mutex> g(c->stats_mu);
      c->stats.batch_completed += 1;
      c->stats.sweep_launches += 2ull * (unsigned long long)hs.iters;
      c->stats.lattice_updates +=
          (unsigned long long)hs.iters * (unsigned long long)r->plan.n * (unsigned long long)r->plan.n;
    }
    release_request(b, r.get());
    complete(b, r->ticket, hs.error ? SOR_ERR_INTERNAL : SOR_OK, res);
  }
  return SOR_OK;
}

static int active_count(const Batcher* b) {
  int n = 0;
  for (const auto& r : b->slots)
    if (r) ++n;
  return n;
}

static void fail_all(Batcher* b, sor_status st) {
  sor_result res;
  std::memset(&res, 0, sizeof(res));
  std::vector<uint64_t> tickets;
  for (auto& r : b->slots)
    if (r) {
      tickets.push_back(r->ticket);
      release_request(b, r.get());
      r.reset();
    }
  {
    std::lock_guard<std::mutex> g(b->mu);
    for (auto& q : b->queue) tickets.push_back(q->ticket);
    b->queue.clear();
    b->failed = true;
    b->fail_status = st;
  }
  for (uint64_t t : tickets) complete(b, t, st, res);
}

static void scheduler_main(Batcher* b) {
  Ctx* c = b->c;
  cudaSetDevice(c->device);
  for (;;) {
    std::vector<std::unique_ptr<Request>> admitted;
    {
      std::unique_lock<std::mutex> g(b->mu);
      b->cv.wait(g, [&] { return b->stop || !b->queue.empty() || active_count(b) > 0; });
      if (b->stop) break;
      const int cap = c->opt_max_slots.load();
      int active = active_count(b);
      while (!b->queue.empty() && (cap <= 0 || active + (int)admitted.size() < cap)) {
        Request* r = b->queue.front().get();
        const size_t need = request_bytes(r->plan);
        if (ctx_reserve(c, need, false, 0.0) != SOR_OK) break;  // waits for retirements
        admitted.push_back(std::move(b->queue.front()));
        b->queue.pop_front();
      }
      if (admitted.empty() && active == 0) {
        // nothing running here will free memory: drop sor_solve's cached
        // workspace if no solve is using it, else wait for it to finish
        g.unlock();
        if (c->solve_mu.try_lock()) {
          release_solve_workspace(c);
          c->solve_mu.unlock();
        }
        std::unique_lock<std::mutex> mg(c->mem_mu);
        c->mem_cv.wait_for(mg, std::chrono::milliseconds(5));
        continue;
      }
    }
    sor_status rs = SOR_OK;
    std::vector<int> new_slots;  // slots activated this round (their host state copy is stale)
    for (auto& r : admitted) {
      int sidx = -1;
      for (size_t k = 0; k < b->slots.size(); ++k)
        if (!b->slots[k]) { sidx = (int)k; break; }
      if (sidx < 0) {
        sidx = (int)b->slots.size();
        rs = ensure_tables(b, sidx + 1, 1);
        if (rs != SOR_OK) break;
        if ((int)b->slots.size() <= sidx) b->slots.resize(sidx + 1);
      }
      rs = activate(b, r.get(), sidx);
      if (rs != SOR_OK) {
        sor_result res;
        std::memset(&res, 0, sizeof(res));
        ctx_release(c, request_bytes(r->plan));
        complete(b, r->ticket, rs, res);
        rs = SOR_OK;
        continue;
      }
      b->slots[sidx] = std::move(r);
      new_slots.push_back(sidx);
    }
    if (rs == SOR_OK && !admitted.empty()) {
      NvtxRange nvtx("sor_admit");
      rs = rebuild_tiles(b);
    }
    // online trial of the plain slots' step length: this round's update rate
    std::vector<std::pair<int, int>> plain_before;  // (slot, iterations before the round)
    int cand = -1;
    double t_round = 0.0;
    if (c->opt_plain_step.load() == 0 && b->plain_step == 0) {
      for (size_t k = 0; k < b->slots.size(); ++k) {
        const Request* r = b->slots[k].get();
        if (!r || r->plan.kind == kRefine) continue;
        const bool fresh = std::find(new_slots.begin(), new_slots.end(), (int)k) != new_slots.end();
        plain_before.emplace_back((int)k, fresh ? 0 : b->h_state[k].iters);
      }
      if (!plain_before.empty()) {
        cand = std::min(kPlainCands - 1, b->plain_trial / kPlainTrialRounds);
        t_round = now_s();
      }
    }
    if (rs == SOR_OK && active_count(b) > 0) {
      NvtxRange nvtx("sor_step");
      int steps = 1;
      rs = run_step(b, &steps);
    }
    if (rs == SOR_OK) {  // one copy of the whole state table
      cudaError_t e = cudaMemcpyAsync(b->h_state, b->d_state, sizeof(SlotState) * b->slots.size(),
                                      cudaMemcpyDeviceToHost, b->stream);
      if (e != cudaSuccess) {
        c->set_error(cudaGetErrorString(e));
        rs = SOR_ERR_CUDA;
      }
    }
    if (rs == SOR_OK) {
      cudaError_t e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) {
        c->set_error(cudaGetErrorString(e));
        rs = SOR_ERR_CUDA;
      }
    }
    if (rs == SOR_OK && cand >= 0) {
      double upd = 0.0;
      for (const auto& pb : plain_before) {
        const double nn = (double)b->slots[pb.first]->plan.n;
        upd += (double)(b->h_state[pb.first].iters - pb.second) * nn * nn;
      }
      const double dt = now_s() - t_round;
      if (dt > 0.0 && upd > 0.0) {
        b->plain_rate[cand] += upd / dt;
        b->plain_rounds[cand] += 1;
        if (++b->plain_trial >= kPlainCands * kPlainTrialRounds) {
          int best = 1;
          double best_rate = -1.0;
          for (int k = 0; k < kPlainCands; ++k)
            if (b->plain_rounds[k] > 0 && b->plain_rate[k] / b->plain_rounds[k] > best_rate) {
              best_rate = b->plain_rate[k] / b->plain_rounds[k];
              best = k;
            }
          b->plain_step = kPlainStepCand[best];
        }
      }
      std::lock_guard<std::mutex> g(c->stats_mu);
      c->stats.batch_plain_step = (unsigned long long)plain_step_len(b);
    } else if (rs == SOR_OK && c->opt_plain_step.load() > 0) {
      std::lock_guard<std::mutex> g(c->stats_mu);
      c->stats.batch_plain_step = (unsigned long long)c->opt_plain_step.load();
    } else if (rs == SOR_OK && b->plain_step > 0) {
      std::lock_guard<std::mutex> g(c->stats_mu);
      c->stats.batch_plain_step = (unsigned long long)b->plain_step;
    }
    if (rs == SOR_OK) {
      std::vector<int> fin;
      for (size_t k = 0; k < b->slots.size(); ++k)
        if (b->slots[k] && b->h_state[k].done) fin.push_back((int)k);
      if (!fin.empty()) {
        for (int k : fin) b->dead_tiles += b->slots[k]->ntiles;
        rs = retire(b, fin);
        // finished slots' tiles stay in the table (their state says done, so
        // every kernel skips them) until admissions rebuild it anyway or they
        // are a sizeable share of the launches
        if (rs == SOR_OK && b->dead_tiles * 10 > b->live_tiles * 3) rs = rebuild_tiles(b);
      }
    }
    if (rs != SOR_OK) {
      fail_all(b, rs);
      break;
    }
  }
  // shutdown: drop queued and active work
  for (auto& r : b->slots)
    if (r) {
      release_request(b, r.get());
      r.reset();
    }
}

void BatcherDeleter::operator()(Batcher* b) const { delete b; }

// A cube worker: takes cube requests in arrival order and solves each on its
// own stream (the cube kernels of sor_solve3d), waiting for device memory under
// the context's budget; results complete their tickets like plates do.
static void cube_worker(Batcher* b) {
  Ctx* c = b->c;
  cudaSetDevice(c->device);
  cudaStream_t s = nullptr;
  const bool have_stream = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    std::unique_ptr<Request> r;
    {
      std::unique_lock<std::mutex> g(b->mu);
      b->cv.wait(g, [&] { return b->stop || !b->cube_queue.empty(); });
      if (b->stop) break;
      r = std::move(b->cube_queue.front());
      b->cube_queue.pop_front();
      b->cube_busy += 1;
    }
    sor_result res;
    std::memset(&res, 0, sizeof(res));
    sor_status st = have_stream ? run_cube(c, &r->p3, r->u0.data(), r->f.empty() ? nullptr : r->f.data(), r->u_out,
                                           &res, s, true)
                                : SOR_ERR_CUDA;
    res.latency_s = now_s() - r->t_submit;
    {
      std::lock_guard<std::mutex> g(c->stats_mu);
      c->stats.batch_completed += 1;
    }
    {
      std::lock_guard<std::mutex> g(b->mu);
      b->cube_busy -= 1;
    }
    complete(b, r->ticket, st, res);
  }
  if (have_stream) cudaStreamDestroy(s);
}

static sor_status start_batcher(Ctx* c) {
  std::lock_guard<std::mutex> g(c->batcher_mu);
  if (c->batcher) return SOR_OK;
  std::unique_ptr<Batcher, BatcherDeleter> b(new Batcher());
  b->c = c;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    c->set_error(cudaGetErrorString(e));
    return SOR_ERR_CUDA;
  }
  sor_status rs = ensure_tables(b.get(), 16, 64);
  if (rs != SOR_OK) return rs;
  b->slots.clear();
  b->slots.resize(b->cap);
  Batcher* raw = b.get();
  c->batcher = std::move(b);
  raw->th = std::thread(scheduler_main, raw);
  return SOR_OK;
}

sor_status batch_submit(Ctx* c, const Plan& p, const double* u0, const double* f, double* u_out, uint64_t* ticket) {
  NvtxRange nvtx("sor_batch_submit");
  if (request_bytes(p) > c->budget) {
    c->set_error("request needs more device memory than the whole budget");
    return SOR_ERR_BUDGET;
  }
  sor_status rs = start_batcher(c);
  if (rs != SOR_OK) return rs;
  Batcher* b = c->batcher.get();
  auto r = std::make_unique<Request>();
  r->plan = p;
  // batched FP64 slots share launches with slots at other iteration counts, so
  // they use the exact-order phases (no per-chunk rescaling)
  if (r->plan.kind == kPlain64) r->plan.exact = true;
  r->t_submit = now_s();
  const size_t nu = (size_t)(p.n + 2) * (p.n + 2);
  r->u0.resize(nu);
  if (is_device_ptr(u0)) {
    if (cudaMemcpy(r->u0.data(), u0, nu * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
      c->set_error("copy of u0 failed");
      return SOR_ERR_CUDA;
    }
  } else {
    std::memcpy(r->u0.data(), u0, nu * 8);
  }
  if (p.has_f) {
    const size_t nf = (size_t)p.n * p.n;
    r->f.resize(nf);
    if (is_device_ptr(f)) {
      if (cudaMemcpy(r->f.data(), f, nf * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        c->set_error("copy of f failed");
        return SOR_ERR_CUDA;
      }
    } else {
      std::memcpy(r->f.data(), f, nf * 8);
    }
  }
  r->u_out = u_out;
  r->out_on_device = is_device_ptr(u_out);
  {
    std::lock_guard<std::mutex> g(b->mu);
    if (b->failed) return b->fail_status;
    r->ticket = b->next_ticket++;
    *ticket = r->ticket;
    b->pending.insert(r->ticket);
    b->queue.push_back(std::move(r));
  }
  b->cv.notify_all();
  return SOR_OK;
}

sor_status batch_submit3d(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                          uint64_t* ticket) {
  NvtxRange nvtx("sor_batch_submit3d");
  sor_status rs = check_params3d(c, p, u0, u_out);
  if (rs != SOR_OK) return rs;
  if (!ticket) {
    c->set_error("ticket must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  if (cube_bytes(p, f != nullptr) > c->budget) {
    c->set_error("request needs more device memory than the whole budget");
    return SOR_ERR_BUDGET;
  }
  rs = start_batcher(c);
  if (rs != SOR_OK) return rs;
  Batcher* b = c->batcher.get();
  auto r = std::make_unique<Request>();
  r->cube = true;
  r->p3 = *p;
  r->t_submit = now_s();
  const size_t m = (size_t)p->n + 2, nu = m * m * m, nf = (size_t)p->n * p->n * p->n;
  r->u0.resize(nu);
  if (is_device_ptr(u0)) {
    if (cudaMemcpy(r->u0.data(), u0, nu * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      c->set_error("copy of u0 failed");
      return SOR_ERR_CUDA;
    }
  } else {
    std::memcpy(r->u0.data(), u0, nu * 8);
  }
  if (f) {
    r->f.resize(nf);
    if (is_device_ptr(f)) {
      if (cudaMemcpy(r->f.data(), f, nf * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        c->set_error("copy of f failed");
        return SOR_ERR_CUDA;
      }
    } else {
      std::memcpy(r->f.data(), f, nf * 8);
    }
  }
  r->u_out = u_out;
  {
    std::lock_guard<std::mutex> g(b->mu);
    r->ticket = b->next_ticket++;
    *ticket = r->ticket;
    b->pending.insert(r->ticket);
    b->cube_queue.push_back(std::move(r));
    // one more worker while every running one is busy, up to kCubeWorkers
    if ((int)b->cube_workers.size() < kCubeWorkers &&
        (int)b->cube_queue.size() + b->cube_busy > (int)b->cube_workers.size())
      b->cube_workers.emplace_back(cube_worker, b);
  }
  b->cv.notify_all();
  return SOR_OK;
}

sor_status batch_poll(Ctx* c, uint64_t ticket, double timeout_s, sor_result* res) {
  Batcher* b = nullptr;
  {
    std::lock_guard<std::mutex> g(c->batcher_mu);
    b = c->batcher.get();
  }
  if (!b) return SOR_ERR_UNKNOWN_TICKET;
  std::unique_lock<std::mutex> g(b->mu);
  auto ready = [&] { return b->completed.count(ticket) > 0 || b->pending.count(ticket) == 0; };
  if (timeout_s != 0.0 && !ready()) {
    if (timeout_s < 0)
      b->done_cv.wait(g, ready);
    else
      b->done_cv.wait_for(g, std::chrono::duration<double>(timeout_s), ready);
  }
  auto it = b->completed.find(ticket);
  if (it != b->completed.end()) {
    const Completed cp = it->second;
    b->completed.erase(it);
    if (res) *res = cp.res;
    return cp.status;
  }
  if (b->pending.count(ticket)) return timeout_s != 0.0 ? SOR_ERR_TIMEOUT : SOR_NOT_READY;
  return SOR_ERR_UNKNOWN_TICKET;
}

void batch_shutdown(Ctx* c) {
  std::unique_ptr<Batcher, BatcherDeleter> b;
  {
    std::lock_guard<std::mutex> g(c->batcher_mu);
    b = std::move(c->batcher);
  }
  if (!b) return;
  c->closing = true;  // waits for memory and running cube solves give up
  {
    std::lock_guard<std::mutex> g(b->mu);
    b->stop = true;
  }
  b->cv.notify_all();
  c->mem_cv.notify_all();
  if (b->th.joinable()) b->th.join();
  for (auto& t : b->cube_workers)
    if (t.joinable()) t.join();
  {
    std::lock_guard<std::mutex> g(b->mu);
    b->cube_queue.clear();
  }
  {
    std::lock_guard<std::mutex> g(b->mu);
    b->queue.clear();  // queued requests hold no reservation yet
    b->pending.clear();
  }
  b->done_cv.notify_all();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaStreamSynchronize(b->stream);
  ctx_dev_free(c, b->d_desc);
  ctx_dev_free(c, b->d_state);
  ctx_dev_free(c, b->d_tiles);
  if (b->h_state) cudaFreeHost(b->h_state);
  cudaStreamDestroy(b->stream);
}

}  // namespace sorgb
