// Host runtime: context memory accounting, slot buffers, and the blocking
// solve driver.  Every arithmetic step runs in the kernels of sor_kernels.cu;
// this file only allocates, copies, launches and reads back state.
#include "sor_runtime.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include <sstream>

namespace sorgb {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define SOR_CK(ctx, expr)                                                                     \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      std::ostringstream os_;                                                                 \
      os_ << #expr << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
      (ctx)->set_error(os_.str());                                                            \
      return SOR_ERR_CUDA;                                                                    \
    }                                                                                         \
  } while (0)

// ------------------------------------------------------------------------------------------------
// plans and sizes
// ------------------------------------------------------------------------------------------------

sor_status make_plan(const sor_params* p, bool has_f, Plan* out, std::string* why) {
  if (!p) { *why = "params is NULL"; return SOR_ERR_INVALID_ARG; }
  if (p->n < 1 || p->n > 60000) { *why = "n must be in [1, 60000]"; return SOR_ERR_INVALID_ARG; }
  if (p->precision < SOR_FP64 || p->precision > SOR_FP32_REFINE) { *why = "unknown precision"; return SOR_ERR_INVALID_ARG; }
  if (p->stop != SOR_STOP_MAXDELTA && p->stop != SOR_STOP_RESID_REL) { *why = "unknown stop"; return SOR_ERR_INVALID_ARG; }
  if (p->max_iters < 0) { *why = "max_iters < 0"; return SOR_ERR_INVALID_ARG; }
  if (p->check_every < 1) { *why = "check_every < 1"; return SOR_ERR_INVALID_ARG; }
  if (p->inner_sweeps < 0) { *why = "inner_sweeps < 0"; return SOR_ERR_INVALID_ARG; }
  if (p->flags & ~SOR_FLAG_EXACT_ORDER) { *why = "unknown flag bits"; return SOR_ERR_INVALID_ARG; }
  if (p->stall_window < 0) { *why = "stall_window < 0"; return SOR_ERR_INVALID_ARG; }
  if (std::isnan(p->tol)) { *why = "tol is NaN"; return SOR_ERR_INVALID_ARG; }
  double w = p->omega;
  if (std::isnan(w)) { *why = "omega is NaN"; return SOR_ERR_INVALID_ARG; }
  if (w <= 0.0) w = sor_omega_opt(p->n);
  if (!(w > 0.0 && w < 2.0)) { *why = "omega must satisfy 0 < omega < 2"; return SOR_ERR_INVALID_ARG; }
  Plan P;
  P.n = p->n;
  P.omega = w;
  P.tol = p->tol;
  P.max_iters = p->max_iters;
  P.has_f = has_f;
  P.exact = (p->flags & SOR_FLAG_EXACT_ORDER) != 0;
  P.stall = p->stall_window;
  if (p->precision == SOR_FP32_REFINE) {
    P.kind = kRefine;
    P.stop = kStopResid;
    P.K = 1;
    P.inner = p->inner_sweeps > 0 ? p->inner_sweeps : 20;
  } else {
    P.kind = p->precision == SOR_FP64 ? kPlain64 : kPlain32;
    P.stop = p->stop == SOR_STOP_MAXDELTA ? kStopDelta : kStopResid;
    P.K = p->check_every;
    P.inner = 0;
  }
  *out = P;
  return SOR_OK;
}

size_t slot_bytes(const Plan& p, bool pingpong) {
  const Layout L = Layout::make(p.n);
  const size_t E = L.elems();
  const size_t nb = pingpong ? 2 : 1;
  switch (p.kind) {
    case kPlain64:
      return nb * 2 * E * 8 + (p.has_f ? 2 * E * 8 : 0);
    case kPlain32:
      return nb * 2 * E * 4 + (p.has_f ? 2 * E * (4 + 8) : 0);
    default:
      return 2 * 2 * E * 8 + (p.has_f ? 2 * E * 8 : 0) + nb * 2 * E * 4 + 2 * E * 4;
  }
}

// ------------------------------------------------------------------------------------------------
// device memory under the budget
// ------------------------------------------------------------------------------------------------

sor_status ctx_reserve(Ctx* c, size_t bytes, bool wait, double timeout_s) {
  std::unique_lock<std::mutex> g(c->mem_mu);
  if (bytes > c->budget) return SOR_ERR_BUDGET;
  if (c->reserved + bytes > c->budget) {
    if (!wait) return SOR_ERR_BUDGET;
    auto pred = [&] { return c->closing.load() || c->reserved + bytes <= c->budget; };
    if (timeout_s < 0) {
      c->mem_cv.wait(g, pred);
    } else if (!c->mem_cv.wait_for(g, std::chrono::duration<double>(timeout_s), pred)) {
      return SOR_ERR_BUDGET;
    }
    if (c->closing.load()) return SOR_ERR_CANCELLED;
  }
  c->reserved += bytes;
  c->peak = std::max(c->peak, c->reserved);
  return SOR_OK;
}

void ctx_release(Ctx* c, size_t bytes) {
  {
    std::lock_guard<std::mutex> g(c->mem_mu);
    c->reserved = bytes > c->reserved ? 0 : c->reserved - bytes;
  }
  c->mem_cv.notify_all();
}

void* ctx_dev_alloc(Ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (c->alloc) return c->alloc(bytes, c->alloc_user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void ctx_dev_free(Ctx* c, void* p) {
  if (!p) return;
  if (c->free_)
    c->free_(p, c->alloc_user);
  else
    cudaFree(p);
}

// ------------------------------------------------------------------------------------------------
// slot buffers
// ------------------------------------------------------------------------------------------------

static void* slot_take(Ctx* c, SlotBuffers* b, size_t bytes, bool* ok) {
  void* p = ctx_dev_alloc(c, bytes);
  if (!p) { *ok = false; return nullptr; }
  b->allocs.push_back(p);
  return p;
}

sor_status alloc_slot(Ctx* c, const Plan& p, bool pingpong, SlotBuffers* out) {
  SlotBuffers b;
  b.L = Layout::make(p.n);
  b.kind = p.kind;
  b.has_f = p.has_f;
  b.pingpong = pingpong;
  b.bytes = slot_bytes(p, pingpong);
  const size_t E = b.L.elems();
  bool ok = true;
  SlotDesc& d = b.desc;
  std::memset(&d, 0, sizeof(d));
  const int nb = pingpong ? 2 : 1;
  if (p.kind == kPlain64 || p.kind == kPlain32) {
    const size_t es = p.kind == kPlain64 ? 8 : 4;
    for (int k = 0; k < nb; ++k)
      for (int col = 0; col < 2; ++col) d.x[k][col] = slot_take(c, &b, E * es, &ok);
    if (p.has_f) {
      for (int col = 0; col < 2; ++col) d.g[col] = slot_take(c, &b, E * es, &ok);
      for (int col = 0; col < 2; ++col)
        d.g64[col] = p.kind == kPlain64 ? (const double*)d.g[col] : (const double*)slot_take(c, &b, E * 8, &ok);
    }
  } else {
    for (int k = 0; k < 2; ++k)
      for (int col = 0; col < 2; ++col) d.u[k][col] = (double*)slot_take(c, &b, E * 8, &ok);
    if (p.has_f)
      for (int col = 0; col < 2; ++col) d.g64[col] = (const double*)slot_take(c, &b, E * 8, &ok);
    for (int k = 0; k < nb; ++k)
      for (int col = 0; col < 2; ++col) d.x[k][col] = slot_take(c, &b, E * 4, &ok);
    for (int col = 0; col < 2; ++col) d.g[col] = slot_take(c, &b, E * 4, &ok);
  }
  if (!ok) {
    free_slot(c, &b);
    return SOR_ERR_OOM;
  }
  *out = std::move(b);
  return SOR_OK;
}

void free_slot(Ctx* c, SlotBuffers* b) {
  for (void* p : b->allocs) ctx_dev_free(c, p);
  b->allocs.clear();
}

void fill_desc(const Plan& p, SlotBuffers* b) {
  SlotDesc& d = b->desc;
  d.n = p.n;
  d.pitch = b->L.pitch;
  d.qmax = b->L.qmax;
  d.kind = p.kind;
  d.K = p.K;
  d.max_iters = p.max_iters;
  d.stop = p.stop;
  d.inner = p.inner;
  d.stall = p.stall;
  d.a64 = 1.0 - p.omega;
  d.b64 = p.omega / 4.0;
  d.a32 = (float)(1.0 - p.omega);
  d.b32 = (float)(p.omega / 4.0);
  d.tol = p.tol;
  d.sweep_tiles = b->L.row_tiles() * b->L.col_tiles();
  d.resid_tiles = d.sweep_tiles;
}

void build_tiles(const Layout& L, int slot, std::vector<Tile>* sweep, std::vector<Tile>* resid, int tile_rows,
                 int tile_cols) {
  const int row_tiles = (L.n + tile_rows - 1) / tile_rows;
  const int col_tiles = (L.qmax + tile_cols - 1) / tile_cols;
  for (int r = 0; r < row_tiles; ++r) {
    const int row0 = 1 + r * tile_rows;
    const int nrows = std::min(tile_rows, L.n - r * tile_rows);
    for (int t = 0; t < col_tiles; ++t) {
      Tile tl{slot, row0, 1 + t * tile_cols, nrows};
      if (sweep) sweep->push_back(tl);
      if (resid) resid->push_back(tl);
    }
  }
}

// Warp strips for the FP64 phase kernel: each 128-column tile is cut into m
// row ranges of (nearly) equal length so that the warps of a persistent grid
// of `warps` warps each get one strip of the same size.
void build_strips(const Layout& L, int slot, int warps, std::vector<Tile>* out) {
  const int ct = L.col_tiles();
  int m = std::max(1, warps / std::max(1, ct));
  m = std::min(m, std::max(1, L.n / 8));  // at least 8 rows per strip
  // column tiles vary fastest: consecutive warps (hence every block and SM)
  // get strips of different column tiles, spreading the first and last
  // column tiles -- whose strips also read Dirichlet ring values -- evenly
  for (int r = 0; r < m; ++r)
    for (int t = 0; t < ct; ++t) {
      const int a = 1 + (int)((long long)r * L.n / m);
      const int b = 1 + (int)((long long)(r + 1) * L.n / m);
      if (b > a) out->push_back(Tile{slot, a, 1 + t * kWarpCols, b - a});
    }
}

SlotState initial_state(const Plan& p) {
  SlotState s;
  std::memset(&s, 0, sizeof(s));
  s.checked_iter = -1;
  s.last_dmax = -1.0;
  s.last_rho = -1.0;
  s.best_rho = HUGE_VAL;
  if (p.kind != kRefine && p.max_iters == 0) s.done = 1;
  return s;
}

// ------------------------------------------------------------------------------------------------
// blocking solve
// ------------------------------------------------------------------------------------------------

static void free_workspace(Ctx* c, SolveWorkspace* w) {
  if (!w) return;
  for (auto& kv : w->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  w->graphs.clear();
  free_slot(c, &w->slot);
  ctx_dev_free(c, w->d_desc);
  ctx_dev_free(c, w->d_state);
  ctx_dev_free(c, w->d_sweep_tiles);
  ctx_dev_free(c, w->d_resid_tiles);
  ctx_dev_free(c, w->d_fast_tiles);
  ctx_dev_free(c, w->d_tb_tiles);
  ctx_dev_free(c, w->d_nat_u);
  ctx_dev_free(c, w->d_nat_f);
  ctx_dev_free(c, w->d_ring);
  ctx_dev_free(c, w->d_progress);
  ctx_dev_free(c, w->d_gridsync);
  for (auto& kv : w->chain_phases) ctx_dev_free(c, kv.second);
  w->chain_phases.clear();
  if (w->h_state) cudaFreeHost(w->h_state);
  for (auto e : w->poll_events) cudaEventDestroy(e);
  for (auto& pr : w->chunk_events) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  ctx_release(c, w->bytes);
}

void release_solve_workspace(Ctx* c) {
  if (c->ws) {
    free_workspace(c, c->ws.get());
    c->ws.reset();
  }
}

sor_status zero_slot(Ctx* c, const Plan& p, SlotBuffers* b, cudaStream_t s) {
  const size_t E = b->L.elems();
  const SlotDesc& d = b->desc;
  const size_t xs = p.kind == kPlain64 ? 8 : 4;
  for (int k = 0; k < 2; ++k)
    for (int col = 0; col < 2; ++col) {
      if (d.x[k][col]) SOR_CK(c, cudaMemsetAsync(d.x[k][col], 0, E * xs, s));
      if (d.u[k][col]) SOR_CK(c, cudaMemsetAsync(d.u[k][col], 0, E * 8, s));
    }
  for (int col = 0; col < 2; ++col) {
    if (d.g[col]) SOR_CK(c, cudaMemsetAsync(d.g[col], 0, E * (p.kind == kPlain64 ? 8 : 4), s));
    if (d.g64[col] && (void*)d.g64[col] != d.g[col]) SOR_CK(c, cudaMemsetAsync((void*)d.g64[col], 0, E * 8, s));
  }
  return SOR_OK;
}

static constexpr int kInflight = 3;

// Fused FP32 sweep kernel of an FP32 or defect-correction plan: the family
// from SOR_OPT_FUSED_KERNEL, by default the tile family up to a size and
// the wavefront family above it, as measured on GB300: plain FP32 sweeps up
// to n = 6144 (the FP32 state near the L2 size), the inner sweeps of defect
// correction up to n = 12288 (they also read the right-hand side, and the
// tile family folds the correction into its last launch: faster at 8192^2
// by 10 %, slower at 16384^2 by 4 %); the depth from
// SOR_OPT_TEMPORAL_DEPTH, by default 6 (tile) or 4 (wavefront), rounded down
// to a depth the family is built for; rows per tile the family's default.
static constexpr int kTileFamilyMaxN = 6144;
static constexpr int kTileFamilyMaxNRefine = 12288;

void resolve_fused(Ctx* c, Plan* p) {
  if (p->kind == kPlain64) {
    p->tdepth = 1;
    return;
  }
  const int opt = c->opt_fused_kernel.load();
  const int tile_max = p->kind == kRefine ? kTileFamilyMaxNRefine : kTileFamilyMaxN;
  const int fk = opt == 1 ? kFusedTile : opt == 2 ? kFusedWave : (p->n <= tile_max ? kFusedTile : kFusedWave);
  int t = c->opt_tdepth.load();
  if (t == 0) t = fk == kFusedWave ? 4 : 6;
  while (t > 1 && !fused_depth_supported(fk, t)) --t;
  p->fkind = fk;
  p->tdepth = std::max(1, t);
  p->tseg = 0;
}

// Most tiles a fused-sweep table of an n x n plate can have (wavefront
// segments of 16 rows, the narrowest output columns).
static size_t fused_tile_cap(int n) {
  const Layout L = Layout::make(n);
  const size_t cols = (L.qmax + 111) / 112 + 1;
  return cols * ((size_t)(n + 15) / 16 + 1);
}

// The fused-sweep tile table of the workspace for the plan's kernel family,
// depth and rows per tile, rebuilt when one of them changes (the graphs
// cached for the old table are dropped with it).  The stream is idle between
// solves, so the table is never rewritten under a running launch.
static sor_status ensure_fused_tiles(Ctx* c, SolveWorkspace* w, const Plan& p) {
  if (p.kind == kPlain64 || p.tdepth <= 1) return SOR_OK;
  const int rows = fused_out_rows(p.fkind, p.n, p.tdepth, c->sm_count, p.tseg);
  if (w->fkind == p.fkind && w->tdepth == p.tdepth && w->tseg_rows == rows) return SOR_OK;
  if (fused_prepare(p.fkind, p.tdepth) != cudaSuccess) {
    cudaGetLastError();
    c->set_error("fused FP32 sweep kernel does not fit");
    return SOR_ERR_CUDA;
  }
  std::vector<Tile> tt;
  build_tiles(w->slot.L, 0, &tt, nullptr, rows, fused_out_cols(p.fkind, p.tdepth));
  if (tt.size() > w->tb_cap) {
    c->set_error("fused-sweep tile table larger than its reservation");
    return SOR_ERR_INTERNAL;
  }
  SOR_CK(c, cudaMemcpyAsync(w->d_tb_tiles, tt.data(), tt.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  for (auto& kv : w->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  w->graphs.clear();
  w->fkind = p.fkind;
  w->tdepth = p.tdepth;
  w->tseg_rows = rows;
  w->n_tb_tiles = (int)tt.size();
  return SOR_OK;
}

static sor_status get_workspace(Ctx* c, const Plan& p, SolveWorkspace** out) {
  const bool pingpong = p.tdepth > 1;
  if (c->ws && c->ws->n == p.n && c->ws->kind == p.kind && c->ws->has_f == p.has_f && c->ws->pingpong == pingpong) {
    *out = c->ws.get();
    return ensure_fused_tiles(c, c->ws.get(), p);
  }
  release_solve_workspace(c);
  auto w = std::make_unique<SolveWorkspace>();
  w->n = p.n;
  w->kind = p.kind;
  w->has_f = p.has_f;
  w->pingpong = pingpong;
  const Layout L = Layout::make(p.n);
  std::vector<Tile> st, rt, ft;
  build_tiles(L, 0, &st, &rt, kTileRows);
  build_strips(L, 0, c->sm_count * fast_blocks_per_sm() * kWarpsY, &ft);
  w->tb_cap = pingpong ? fused_tile_cap(p.n) : 1;
  const size_t nat_u = (size_t)(p.n + 2) * (p.n + 2) * 8;
  const size_t nat_f = p.has_f ? (size_t)p.n * p.n * 8 : 0;
  // barrier state of the grid solver, or the exchange and decision words of
  // its barrier-free form for the plain plates small enough for it
  size_t gsync = grid_sync_bytes();
  if ((p.kind == kPlain64 && p.n <= kGridMaxN64) || (p.kind == kPlain32 && p.n <= kGridMaxN32))
    gsync = std::max(gsync, grid_flow_sync_bytes(p.kind == kPlain32, p.n, L.pitch, c->sm_count));
  const size_t small = gsync + sizeof(SlotDesc) + sizeof(SlotState) +
                       (st.size() + rt.size() + ft.size() + w->tb_cap) * sizeof(Tile) +
                       2 * (2 * (size_t)L.pitch + 2 * (size_t)(p.n + 2)) * sizeof(double);  // saved ring
  const size_t total = slot_bytes(p, pingpong) + nat_u + nat_f + small + 4096;
  sor_status rs = ctx_reserve(c, total, false, 0.0);
  if (rs != SOR_OK) {
    c->set_error("solve needs more device memory than the budget has free");
    return rs;
  }
  w->bytes = total;
  rs = alloc_slot(c, p, pingpong, &w->slot);
  if (rs != SOR_OK) {
    ctx_release(c, total);
    c->set_error("device allocation failed");
    return rs;
  }
  bool ok = true;
  w->d_desc = (SlotDesc*)ctx_dev_alloc(c, sizeof(SlotDesc));
  w->d_state = (SlotState*)ctx_dev_alloc(c, sizeof(SlotState));
  w->d_sweep_tiles = (Tile*)ctx_dev_alloc(c, st.size() * sizeof(Tile));
  w->d_resid_tiles = (Tile*)ctx_dev_alloc(c, rt.size() * sizeof(Tile));
  w->d_fast_tiles = (Tile*)ctx_dev_alloc(c, ft.size() * sizeof(Tile));
  w->d_tb_tiles = (Tile*)ctx_dev_alloc(c, w->tb_cap * sizeof(Tile));
  w->d_nat_u = (double*)ctx_dev_alloc(c, nat_u);
  w->d_gridsync = ctx_dev_alloc(c, gsync);
  w->gridsync_bytes = gsync;
  if (p.has_f) w->d_nat_f = (double*)ctx_dev_alloc(c, nat_f);
  const size_t ring_elems = 2 * (size_t)L.pitch + 2 * (size_t)(p.n + 2);  // per colour
  if (p.kind == kPlain64) w->d_ring = (double*)ctx_dev_alloc(c, 2 * ring_elems * sizeof(double));
  if (p.kind == kPlain64) {
    // chunk launches: cooperative, so the strip table's warps must all be
    // resident at once in the chain kernel's own occupancy (allocated for
    // exact-order solves too: a later default solve reuses the workspace)
    w->d_progress = (unsigned*)ctx_dev_alloc(c, std::max<size_t>(1, ft.size()) * sizeof(unsigned));
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    const int bps = fast_blocks_per_sm();
    w->fast_ct = L.col_tiles();
    if (coop && fast_chain_blocks_per_sm() >= bps && (int)ft.size() % w->fast_ct == 0 &&
        (int)ft.size() <= c->sm_count * bps * kWarpsY)
      w->chain_grid = c->sm_count * bps;
  }
  ok = w->d_desc && w->d_state && w->d_sweep_tiles && w->d_resid_tiles && w->d_fast_tiles && w->d_tb_tiles &&
       w->d_nat_u && w->d_gridsync &&
       (!p.has_f || w->d_nat_f) && (p.kind != kPlain64 || w->d_ring) &&
       (p.kind != kPlain64 || w->d_progress);
  if (!ok || cudaMallocHost(&w->h_state, sizeof(SlotState) * kInflight) != cudaSuccess) {
    cudaGetLastError();
    free_workspace(c, w.get());
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  w->h_state_count = kInflight;
  w->poll_events.resize(kInflight);
  w->chunk_events.resize(kInflight);
  for (int k = 0; k < kInflight; ++k) {
    cudaEventCreateWithFlags(&w->poll_events[k], cudaEventDisableTiming);
    cudaEventCreate(&w->chunk_events[k].first);
    cudaEventCreate(&w->chunk_events[k].second);
  }
  cudaEventCreate(&w->ev0);
  cudaEventCreate(&w->ev1);
  w->n_sweep_tiles = (int)st.size();
  w->n_resid_tiles = (int)rt.size();
  w->n_fast_tiles = (int)ft.size();
  w->n_tb_tiles = 0;
  SOR_CK(c, cudaMemcpyAsync(w->d_sweep_tiles, st.data(), st.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  SOR_CK(c, cudaMemcpyAsync(w->d_resid_tiles, rt.data(), rt.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  SOR_CK(c, cudaMemcpyAsync(w->d_fast_tiles, ft.data(), ft.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  // zero every array once: kernels write interior cells only, so padding and
  // the correction's ring stay zero for the workspace's lifetime
  rs = zero_slot(c, p, &w->slot, c->stream);
  if (rs != SOR_OK) {
    free_workspace(c, w.get());
    return rs;
  }
  c->ws = std::move(w);
  *out = c->ws.get();
  return ensure_fused_tiles(c, c->ws.get(), p);
}

// Chunk length (iterations for plain kinds, corrections for refine) between
// convergence polls: a few milliseconds of work, at most 256 iterations.
static int chunk_length(Ctx* c, const Plan& p) {
  const int opt = c->opt_chunk.load();
  const double cells = (double)p.n * (double)p.n;
  if (p.kind == kRefine) {
    if (opt > 0) return opt;
    if (p.rchunk > 0) return p.rchunk;
    const double per_step = cells * p.inner;
    int k = (int)std::ceil(4.0e8 / std::max(per_step, 1.0));
    return std::max(1, std::min(k, 16));
  }
  int L = opt > 0 ? opt : (int)std::ceil(2.0e8 / std::max(cells, 1.0));
  L = std::max(4, std::min(L, 256));
  if (p.stop == kStopResid) {
    // align residual tests with chunk positions: multiples of K inside a chunk
    if (p.K <= L) {
      L = p.K * std::max(1, L / p.K);
    } else {
      int best = 1;
      for (int d = L; d >= 1; --d)
        if (p.K % d == 0) { best = d; break; }
      if (best >= 4) L = best;
    }
  }
  return L;
}

// Launch sequence of one chunk of a plain solve: L iterations, each a red
// and a black phase, with residual tests where the iteration may be a
// multiple of K (the kernel itself skips the others).
static sor_status enqueue_plain_chunk(Ctx* c, SolveWorkspace* w, const Plan& p, int L, cudaStream_t s) {
  if (p.kind == kPlain32 && p.tdepth > 1) {
    // launches of tdepth fused iterations; the chunk ends where |change| or
    // the residual is tested, so no launch spans a tested iteration
    for (int done = 0; done < L;) {
      const int nt = std::min(p.tdepth, L - done);
      SOR_CK(c, launch_fused(p.fkind, false, p.tdepth, w->d_desc, w->d_state, w->d_tb_tiles, w->n_tb_tiles, 0, nt, 0, 0,
                                s));
      done += nt;
    }
    if (p.stop == kStopResid)
      SOR_CK(c, launch_resid(kResidCheck32, w->d_desc, w->d_state, w->d_resid_tiles, w->n_resid_tiles, 0, 0, s));
    return SOR_OK;
  }
  const SweepKind sk = p.kind == kPlain64 ? kSweepPlain64 : kSweepPlain32;
  const bool resid_every = p.stop == kStopResid && !(p.K <= L && L % p.K == 0) && !(p.K > L && p.K % L == 0);
  for (int it = 0; it < L; ++it) {
    SOR_CK(c, launch_sweep(sk, w->d_desc, w->d_state, w->d_sweep_tiles, w->n_sweep_tiles, 0, 0, 0, s));
    SOR_CK(c, launch_sweep(sk, w->d_desc, w->d_state, w->d_sweep_tiles, w->n_sweep_tiles, 0, 1, 0, s));
    if (p.stop == kStopResid) {
      const bool at = resid_every || (p.K <= L ? ((it + 1) % p.K == 0) : (it == L - 1));
      if (at)
        SOR_CK(c, launch_resid(p.kind == kPlain64 ? kResidCheck64 : kResidCheck32, w->d_desc, w->d_state,
                               w->d_resid_tiles, w->n_resid_tiles, 0, 0, s));
    }
  }
  return SOR_OK;
}

// One chunk of defect correction: C steps of [residual pass (applies the
// pending correction, tests rho, writes r~), inner sweeps].
// Buffer holding the correction after a correction's launches: launch j of
// the temporally blocked sweeps reads buffer (j even ? 1 : 0) -- the first
// one reads nothing, d starting from 0 -- and writes the other one.
int refine_dbuf(const Plan& p) {
  if (p.tdepth <= 1) return 0;
  const int launches = (p.inner + p.tdepth - 1) / p.tdepth;
  return ((launches - 1) % 2 == 0) ? 0 : 1;
}

static sor_status enqueue_refine_chunk(Ctx* c, SolveWorkspace* w, const Plan& p, int C, cudaStream_t s) {
  if (p.tdepth > 1) {
    // the tile family's last launch of each correction adds d to u itself,
    // so the residual pass needs no correction pass before it
    const int dbuf = refine_dbuf(p);
    const bool fix = fused_corrects(p.fkind);
    for (int step = 0; step < C; ++step) {
      SOR_CK(c, launch_resid(fix ? kResidRefine64Fixed : kResidRefine64, w->d_desc, w->d_state, w->d_resid_tiles,
                             w->n_resid_tiles, 0, dbuf, s));
      for (int j = 0, sw = 0; sw < p.inner; ++j, sw += p.tdepth) {
        const int nt = std::min(p.tdepth, p.inner - sw);
        SOR_CK(c, launch_fused(p.fkind, true, p.tdepth, w->d_desc, w->d_state, w->d_tb_tiles, w->n_tb_tiles, 0, nt,
                               (j % 2 == 0) ? 1 : 0, sw, s, fix));
      }
    }
    return SOR_OK;
  }
  for (int step = 0; step < C; ++step) {
    SOR_CK(c, launch_resid(kResidRefine64, w->d_desc, w->d_state, w->d_resid_tiles, w->n_resid_tiles, 0, 0, s));
    for (int sw = 0; sw < p.inner; ++sw) {
      SOR_CK(c, launch_sweep(kSweepInner32, w->d_desc, w->d_state, w->d_sweep_tiles, w->n_sweep_tiles, 0, 0, sw, s));
      SOR_CK(c, launch_sweep(kSweepInner32, w->d_desc, w->d_state, w->d_sweep_tiles, w->n_sweep_tiles, 0, 1, sw, s));
    }
  }
  return SOR_OK;
}

// Longest chunk for the rescaled FP64 phases: the carried scale grows by
// (4/w)^2 per iteration; keep it below 2^400 so values stay far from overflow.
static int fast_lmax(double omega) {
  const double bits = 2.0 * std::log2(4.0 / omega);
  const int L = bits > 0.0 ? (int)std::floor(400.0 / bits) : 256;
  return std::max(1, std::min(L, 256));
}

// Inside a chunk of L iterations the rescaled phases store each colour at a
// scale of at most (c / omega)^(2L - 2), c = 4 (plate) or 6 (cube); the last
// iteration of a chunk runs unscaled, so L = 1 carries no scale at all.  The
// stored values are the iterates times that scale.  Bound on the iterates:
//  * the discrete solution satisfies |u*| <= max|ring| + max|f| / 8 (maximum
//    principle with the comparison function sum_d (x_d - 1/2)^2 / (2 dims),
//    which the 5- and 7-point stencils differentiate exactly), and max|f| =
//    max|h^2 f| (n + 1)^2, so M = umax + gmax max(1, (n + 1)^2 / 8) bounds
//    both |u*| and |u0|;
//  * every single-cell SOR update with 0 < omega < 2 lowers the energy
//    norm of the error (the Ostrowski-Reich argument), so at any point of
//    the iteration |e|_inf <= |e|_2 <= sqrt(kappa) n^(dims/2) |e0|_inf with
//    sqrt(kappa) < n + 1: |u| <= M + 2M (n + 1)^(1 + dims/2);
//  * neighbour sums and coefficient products add at most a few more bits.
// The cap keeps log2 of the largest stored value below 1020.
int rescaled_lcap(double umax, double gmax, int n, int dims, double omega) {
  const double c = dims == 3 ? 6.0 : 4.0;
  const double M = umax + gmax * std::max(1.0, (double)(n + 1) * (n + 1) / 8.0);
  if (!std::isfinite(M) || !(M > 0.0)) return 0;
  const double mbits = std::log2(M);
  if (mbits < -960.0) return 0;
  const double growth = std::log2(3.0) + (1.0 + 0.5 * dims) * std::log2((double)n + 1.0);
  const double room = 1020.0 - (mbits + growth + 6.0);  // 6: sums of up to 7 terms, (1 - w) (c / w)^2 products
  if (room < 0.0) return 0;
  const double per_iter = 2.0 * std::log2(c / omega);  // scale bits per iteration
  const double L = per_iter > 0.0 ? 1.0 + std::floor(room / per_iter) : 256.0;
  return (int)std::max(1.0, std::min(L, 256.0));
}

// Iterations in the next chunk of a plain solve that has planned k0 so far.
// The rescaled FP64 phases must end a chunk wherever |change| is measured
// (multiples of K and the cap), since only chunk ends hold unscaled values.
static int next_chunk(Ctx* c, const Plan& p, long long k0, int L) {
  if (p.kind == kPlain32 && p.tdepth > 1) {
    const long long to_check = p.K - (k0 % p.K);
    const long long to_cap = (long long)p.max_iters - k0;
    return (int)std::max<long long>(1, std::min<long long>(std::max(L, p.tdepth), std::min(to_check, to_cap)));
  }
  if (p.kind == kPlain64 && !p.exact) {
    const long long to_check = p.K - (k0 % p.K);
    const long long to_cap = (long long)p.max_iters - k0;
    const int lmax = p.lcap > 0 ? std::min(p.lcap, fast_lmax(p.omega)) : fast_lmax(p.omega);
    long long Lc = std::min<long long>(lmax, std::min(to_check, to_cap));
    (void)c;
    (void)L;
    return (int)std::max<long long>(1, Lc);
  }
  return L;
}

static FastPhaseArgs fast_phase(const Plan& p, int t, int L, int colour) {
  const double w4 = p.omega / 4.0, omc = 1.0 - p.omega;
  FastPhaseArgs a;
  // scale at which the next phase reads this phase's colour (its ring cells
  // are rewritten so): black at t reads red at a_t (1 at t = L); red at t + 1
  // reads black at b_t (1 at t = L: the next chunk starts unscaled)
  if (colour == 0)
    a.nscale = t == L ? 1.0 : std::pow(w4, -(2 * t - 1));
  else
    a.nscale = t == L ? 1.0 : std::pow(w4, -(2 * t));
  if (colour == 0) {
    if (t == L) {  // back to unscaled values
      const double inv_a = t == 1 ? 1.0 : std::pow(w4, 2 * t - 3);  // 1 / a_{t-1}
      const double inv_b = t == 1 ? 1.0 : std::pow(w4, 2 * t - 2);  // 1 / b_{t-1}
      a.alpha = omc * inv_a;
      a.beta = w4 * inv_b;
      a.gamma = w4;
      a.dscale = inv_a;
      a.last = 1;
    } else {
      a.alpha = t == 1 ? omc / w4 : omc / (w4 * w4);
      a.beta = 1.0;
      a.gamma = std::pow(w4, -(2 * t - 2));
      a.dscale = 0.0;
      a.last = 0;
    }
  } else {
    if (t == L) {
      const double inv_b = t == 1 ? 1.0 : std::pow(w4, 2 * t - 2);
      a.alpha = omc * inv_b;
      a.beta = w4;
      a.gamma = w4;
      a.dscale = inv_b;
      a.last = 1;
    } else {
      a.alpha = omc / (w4 * w4);
      a.beta = 1.0;
      a.gamma = std::pow(w4, -(2 * t - 1));
      a.dscale = 0.0;
      a.last = 0;
    }
  }
  return a;
}

// L iterations of the rescaled FP64 phases (one chunk).
static bool use_chain(Ctx* c, const SolveWorkspace* w) { return w->chain_grid > 0 && c->opt_fast_chain.load(); }

static std::string chain_key(const Plan& p, int L) {
  std::ostringstream k;
  k.precision(17);
  k << L << ":" << p.omega;
  return k.str();
}

// Packed phase records of a chunk of L iterations (uploaded once per length
// and omega, before any capture).
static sor_status ensure_chain_phases(Ctx* c, SolveWorkspace* w, const Plan& p, int L) {
  const std::string key = chain_key(p, L);
  if (w->chain_phases.count(key)) return SOR_OK;
  const size_t rec = fast_phase_bytes();
  std::vector<unsigned char> host(rec * 2 * (size_t)L);
  for (int t = 1; t <= L; ++t)
    for (int colour = 0; colour < 2; ++colour)
      fast_phase_pack(fast_phase(p, t, L, colour), host.data() + rec * (size_t)(2 * (t - 1) + colour));
  void* d = ctx_dev_alloc(c, host.size());
  if (!d) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  if (cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    ctx_dev_free(c, d);
    c->set_error("copy of the phase records failed");
    return SOR_ERR_CUDA;
  }
  w->chain_phases[key] = d;
  return SOR_OK;
}

static sor_status enqueue_fast_chunk(Ctx* c, SolveWorkspace* w, const Plan& p, int L, cudaStream_t s) {
  if (use_chain(c, w)) {
    auto it = w->chain_phases.find(chain_key(p, L));
    if (it == w->chain_phases.end()) {
      c->set_error("phase records of the chunk were not prepared");
      return SOR_ERR_INTERNAL;
    }
    SOR_CK(c, cudaMemsetAsync(w->d_progress, 0, (size_t)w->n_fast_tiles * sizeof(unsigned), s));
    SOR_CK(c, launch_fast_chain(w->d_desc, w->d_state, w->d_fast_tiles, w->n_fast_tiles, w->fast_ct, it->second,
                                2 * L, w->d_progress, p.has_f, w->chain_grid, s));
    if (p.stop == kStopResid)
      SOR_CK(c, launch_resid(kResidCheck64, w->d_desc, w->d_state, w->d_resid_tiles, w->n_resid_tiles, 0, 0, s));
    return SOR_OK;
  }
  for (int t = 1; t <= L; ++t) {
    for (int colour = 0; colour < 2; ++colour) {
      const FastPhaseArgs a = fast_phase(p, t, L, colour);
      SOR_CK(c, launch_sweep_fast64(w->d_desc, w->d_state, w->d_fast_tiles, w->n_fast_tiles, 0, colour, a, p.has_f,
                                    s));
    }
  }
  if (p.stop == kStopResid)
    SOR_CK(c, launch_resid(kResidCheck64, w->d_desc, w->d_state, w->d_resid_tiles, w->n_resid_tiles, 0, 0, s));
  return SOR_OK;
}

static sor_status enqueue_chunk(Ctx* c, SolveWorkspace* w, const Plan& p, int L, cudaStream_t s) {
  if (p.kind == kRefine) return enqueue_refine_chunk(c, w, p, L, s);
  if (p.kind == kPlain64 && !p.exact) return enqueue_fast_chunk(c, w, p, L, s);
  return enqueue_plain_chunk(c, w, p, L, s);
}

static sor_status launch_chunk(Ctx* c, SolveWorkspace* w, const Plan& p, int L, cudaStream_t s) {
  const bool chain = p.kind == kPlain64 && !p.exact && use_chain(c, w);
  if (chain) {
    sor_status rs = ensure_chain_phases(c, w, p, L);
    if (rs != SOR_OK) return rs;
  }
  if (!c->opt_graphs.load()) return enqueue_chunk(c, w, p, L, s);
  std::ostringstream key;
  key.precision(17);
  key << p.kind << ":" << p.exact << ":" << p.stop << ":" << p.K << ":" << p.inner << ":" << L << ":" << p.has_f
      << ":" << p.omega << ":" << p.tdepth << ":" << p.fkind << ":" << w->tseg_rows << ":" << chain;
  auto it = w->graphs.find(key.str());
  if (it == w->graphs.end()) {
    cudaGraph_t g = nullptr;
    SOR_CK(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const unsigned long long l0 = kernel_launch_count();
    sor_status rs = enqueue_chunk(c, w, p, L, s);
    const unsigned long long captured = kernel_launch_count() - l0;
    w->captured += captured;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rs != SOR_OK) {
      if (g) cudaGraphDestroy(g);
      return rs;
    }
    SOR_CK(c, e);
    GraphEntry ge;
    ge.launches = captured;
    e = cudaGraphInstantiate(&ge.exec, g, 0);
    cudaGraphDestroy(g);
    SOR_CK(c, e);
    it = w->graphs.emplace(key.str(), ge).first;
  }
  SOR_CK(c, cudaGraphLaunch(it->second.exec, s));
  w->replayed += it->second.launches;
  return SOR_OK;
}

static sor_status solve_locked(Ctx* c, const Plan& p, const double* u0, const double* f, double* u_out,
                               sor_result* res, double t0);

// ------------------------------------------------------------------------------------------------
// autotuner: the fused FP32 sweep kernel and the corrections per graph
// ------------------------------------------------------------------------------------------------
//
// On the first FP32 or defect-correction solve of a size bucket (and source
// presence) with SOR_OPT_AUTOTUNE, short solves on the call's own inputs time
//  * the FP32 sweeps: unfused (one launch per colour phase), the tile family
//    at depths 2, 3, 4, 6, 8, and the wavefront family at depths 2 .. 5 with
//    rows per tile {its default, 32, 64, 128} -- a plain FP32 solve of 120
//    iterations each, its sweep chunks timed with CUDA events;
//  * for defect correction, with that kernel, the corrections replayed per
//    graph between host polls (the residual test runs in every correction
//    regardless; this sets how often the host looks): 1, 2, 4, 8, timed on a
//    chain of 16 corrections.
// Every candidate gives bit-identical results, so the choice affects time
// only.  SOR_AUTOTUNE_CACHE names an optional file holding the choices across
// processes ("<n_bucket> <has_f> <family> <depth> <rows> <chunk>" per line;
// lines of three numbers, "<n_bucket> <has_f> <depth>", name a tile-family
// depth).

static const int kTuneTileDepths[] = {2, 3, 4, 6, 8};
static const int kTuneWaveDepths[] = {2, 3, 4, 5};
static const int kTuneWaveRows[] = {0, 32, 64, 128};
static const int kTuneChunks[] = {1, 2, 4, 8};
static constexpr int kTuneIters = 120;   // a multiple of every candidate depth
static constexpr int kTuneCorrections = 16;

static int n_bucket(int n) {
  int b = 16;
  while (b < n) b <<= 1;
  return b;
}

static std::string tune_key(int n, bool has_f) {
  std::ostringstream os;
  os << n_bucket(n) << " " << (has_f ? 1 : 0);
  return os.str();
}

static bool tune_valid(const TuneChoice& t) {
  return (t.fkind == kFusedTile || t.fkind == kFusedWave) && (t.tdepth == 1 || fused_depth_supported(t.fkind, t.tdepth)) &&
         t.tseg >= 0 && t.rchunk >= 0 && t.rchunk <= 64;
}

void load_tune_cache(Ctx* c) {
  const char* path = std::getenv("SOR_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return;
  char line[256];
  std::lock_guard<std::mutex> g(c->tune_mu);
  while (std::fgets(line, sizeof(line), fp)) {
    int v[6];
    const int k = std::sscanf(line, "%d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]);
    TuneChoice t;
    if (k == 3) {
      t.fkind = kFusedTile;
      t.tdepth = v[2];
    } else if (k == 6) {
      t.fkind = v[2];
      t.tdepth = v[3];
      t.tseg = v[4];
      t.rchunk = v[5];
    } else {
      continue;
    }
    if (tune_valid(t)) c->tuned[tune_key(v[0], v[1] != 0)] = t;
  }
  std::fclose(fp);
}

static void save_tune_cache(Ctx* c) {
  const char* path = std::getenv("SOR_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* fp = std::fopen(path, "w");
  if (!fp) return;
  for (const auto& kv : c->tuned)
    std::fprintf(fp, "%s %d %d %d %d\n", kv.first.c_str(), kv.second.fkind, kv.second.tdepth, kv.second.tseg,
                 kv.second.rchunk);
  std::fclose(fp);
}

// Sweep time of the plain FP32 tuning solve q (the second of two runs: the
// first builds the tile table and the graphs); result into the workspace.
static sor_status tune_sweeps(Ctx* c, const Plan& q, const double* u0, const double* f, double* ms) {
  sor_status rs = SOR_OK;
  for (int rep = 0; rep < 2 && rs == SOR_OK; ++rep) {
    {
      std::lock_guard<std::mutex> g(c->stats_mu);
      c->stats.sweep_ms = 0.0;
    }
    SolveWorkspace* w = nullptr;
    rs = get_workspace(c, q, &w);
    if (rs != SOR_OK) break;
    rs = solve_locked(c, q, u0, f, w->d_nat_u, nullptr, now_s());
    std::lock_guard<std::mutex> g(c->stats_mu);
    *ms = c->stats.sweep_ms;
  }
  return rs;
}

static sor_status autotune(Ctx* c, const Plan& p, const double* u0, const double* f, TuneChoice* out) {
  Plan q = p;
  q.kind = kPlain32;
  q.stop = kStopDelta;
  q.K = kTuneIters;
  q.max_iters = kTuneIters;
  q.tol = -1.0;
  q.exact = false;
  q.stall = 0;
  q.rchunk = 0;
  const int saved_timing = c->opt_timing.exchange(1);
  sor_stats keep;
  {
    std::lock_guard<std::mutex> g(c->stats_mu);
    keep = c->stats;
  }
  std::vector<TuneChoice> cand;
  cand.push_back(TuneChoice{kFusedTile, 1, 0, 0});
  for (int d : kTuneTileDepths) cand.push_back(TuneChoice{kFusedTile, d, 0, 0});
  for (int d : kTuneWaveDepths) {
    std::vector<int> seen;
    for (int rows : kTuneWaveRows) {
      const int eff = fused_out_rows(kFusedWave, p.n, d, c->sm_count, rows);
      if (std::find(seen.begin(), seen.end(), eff) != seen.end()) continue;
      seen.push_back(eff);
      cand.push_back(TuneChoice{kFusedWave, d, rows, 0});
    }
  }
  double best_ms = 1e300;
  TuneChoice best = cand[0];
  sor_status rs = SOR_OK;
  for (const TuneChoice& t : cand) {
    q.fkind = t.fkind;
    q.tdepth = t.tdepth;
    q.tseg = t.tseg;
    double ms = 0.0;
    rs = tune_sweeps(c, q, u0, f, &ms);
    if (rs != SOR_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  if (rs == SOR_OK && p.kind == kRefine) {
    Plan r = p;
    r.fkind = best.fkind;
    r.tdepth = best.tdepth;
    r.tseg = best.tseg;
    r.tol = -1.0;  // never converges: a fixed chain of corrections
    r.stall = 0;
    r.max_iters = r.inner * kTuneCorrections;
    double best_s = 1e300;
    for (int chunk : kTuneChunks) {
      r.rchunk = chunk;
      sor_result res;
      std::memset(&res, 0, sizeof(res));
      for (int rep = 0; rep < 2 && rs == SOR_OK; ++rep) {  // the first run builds the graphs
        SolveWorkspace* w = nullptr;
        rs = get_workspace(c, r, &w);
        if (rs == SOR_OK) rs = solve_locked(c, r, u0, f, w->d_nat_u, &res, now_s());
      }
      if (rs != SOR_OK) break;
      if (res.device_s < best_s) {
        best_s = res.device_s;
        best.rchunk = chunk;
      }
    }
  }
  c->opt_timing = saved_timing;
  {
    std::lock_guard<std::mutex> g(c->stats_mu);
    c->stats = keep;
  }
  *out = best;
  return rs;
}

sor_status solve_blocking(Ctx* c, const Plan& plan_in, const double* u0, const double* f, double* u_out,
                          sor_result* res) {
  NvtxRange nvtx("sor_solve");
  const double t0 = now_s();
  std::lock_guard<std::mutex> lock(c->solve_mu);
  Plan p = plan_in;
  resolve_fused(c, &p);
  if (p.kind != kPlain64 && c->opt_tdepth.load() == 0 && c->opt_fused_kernel.load() == 0 &&
      c->opt_autotune.load()) {
    const std::string key = tune_key(p.n, p.has_f || p.kind == kRefine);
    TuneChoice ch;
    bool found = false;
    {
      std::lock_guard<std::mutex> g(c->tune_mu);
      auto it = c->tuned.find(key);
      if (it != c->tuned.end()) {
        ch = it->second;
        found = true;
      }
    }
    if (!found) {
      sor_status rs = autotune(c, p, u0, f, &ch);
      if (rs != SOR_OK) return rs;
      std::lock_guard<std::mutex> g(c->tune_mu);
      c->tuned[key] = ch;
      save_tune_cache(c);
    }
    p.fkind = ch.fkind;
    p.tdepth = ch.tdepth;
    p.tseg = ch.tseg;
    p.rchunk = ch.rchunk;
  }
  return solve_locked(c, p, u0, f, u_out, res, t0);
}

static sor_status solve_locked(Ctx* c, const Plan& plan, const double* u0, const double* f, double* u_out,
                               sor_result* res, double t0) {
  cudaStream_t s = c->stream;
  Plan p = plan;  // the FP64 default path may turn exact-order once the input magnitudes are known
  SolveWorkspace* w = nullptr;
  sor_status rs = get_workspace(c, p, &w);
  if (rs != SOR_OK) return rs;
  const unsigned long long launches0 = kernel_launch_count();
  w->captured = 0;
  w->replayed = 0;

  const bool timing = c->opt_timing.load() != 0;
  SOR_CK(c, cudaEventRecord(w->ev0, s));
  const size_t nat_u = (size_t)(p.n + 2) * (p.n + 2);
  const double* du0 = u0;
  if (!is_device_ptr(u0)) {
    SOR_CK(c, cudaMemcpyAsync(w->d_nat_u, u0, nat_u * 8, cudaMemcpyHostToDevice, s));
    du0 = w->d_nat_u;
  }
  const double* df = nullptr;
  if (p.has_f) {
    df = f;
    if (!is_device_ptr(f)) {
      SOR_CK(c, cudaMemcpyAsync(w->d_nat_f, f, (size_t)p.n * p.n * 8, cudaMemcpyHostToDevice, s));
      df = w->d_nat_f;
    }
  }
  fill_desc(p, &w->slot);
  if (p.kind == kPlain64 && !p.exact) w->slot.desc.sweep_tiles = w->n_fast_tiles;  // warp strips
  if (p.kind == kPlain64) {
    const size_t ring_elems = 2 * (size_t)w->slot.L.pitch + 2 * (size_t)(p.n + 2);
    w->slot.desc.ring[0] = w->d_ring;
    w->slot.desc.ring[1] = w->d_ring + ring_elems;
  }
  if (p.kind == kPlain32 && p.tdepth > 1) w->slot.desc.sweep_tiles = w->n_tb_tiles;  // fused-iteration tiles
  SlotState st0 = initial_state(p);
  SOR_CK(c, cudaMemcpyAsync(w->d_desc, &w->slot.desc, sizeof(SlotDesc), cudaMemcpyHostToDevice, s));
  SOR_CK(c, cudaMemcpyAsync(w->d_state, &st0, sizeof(SlotState), cudaMemcpyHostToDevice, s));

  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.u0 = du0;
  pa.f = df;
  pa.n = p.n;
  pa.pitch = w->slot.L.pitch;
  const double h = 1.0 / (double)(p.n + 1);
  pa.h2 = h * h;
  pa.fp32 = p.kind != kPlain64;
  const SlotDesc& d = w->slot.desc;
  if (p.kind == kRefine) {
    for (int k = 0; k < 2; ++k)
      for (int col = 0; col < 2; ++col) pa.u[k][col] = d.u[k][col];
    for (int col = 0; col < 2; ++col) pa.g64[col] = (double*)d.g64[col];
  } else {
    for (int k = 0; k < 2; ++k)
      for (int col = 0; col < 2; ++col) pa.x[k][col] = d.x[k][col];
    for (int col = 0; col < 2; ++col) {
      pa.g[col] = d.g[col];
      pa.g64[col] = p.kind == kPlain32 ? (double*)d.g64[col] : nullptr;
    }
  }
  pa.state = w->d_state;
  SOR_CK(c, launch_pack(pa, s));
  // small plain plates: the whole solve in one launch, on a cooperative grid
  // (max|change| stop) or in one thread-block cluster (exact order either way)
  const bool small = p.kind == kPlain64 ? p.n <= kGridMaxN64 : p.n <= kGridMaxN32;
  const int small_opt = c->opt_cluster.load();
  const bool one_launch = !(p.kind != kRefine && p.max_iters == 0) && p.kind != kRefine && small && small_opt != 0;
  const bool fp32 = p.kind == kPlain32;
  const bool flow = one_launch && small_opt == 1 && p.stop == kStopDelta &&
                    grid_flow_fits(fp32, p.n, w->slot.L.pitch, c->sm_count) &&
                    grid_flow_sync_bytes(fp32, p.n, w->slot.L.pitch, c->sm_count) <= w->gridsync_bytes;
  const bool grid = one_launch && !flow && (small_opt == 1 || small_opt == 3) && p.stop == kStopDelta &&
                    grid_solve_fits(fp32, p.n, w->slot.L.pitch, c->sm_count);
  const bool cluster = one_launch && !flow && !grid && cluster_solve_fits(fp32, p.n, w->slot.L.pitch);
  if (p.kind == kPlain64 && !p.exact && !cluster && !grid && !flow) {
    // the rescaled phases need the input magnitudes to bound their chunk
    // length; inputs they cannot carry take the exact-order phases
    SOR_CK(c, cudaMemcpyAsync(&w->h_state[0], w->d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR_CK(c, cudaStreamSynchronize(s));
    double umax = 0.0, gmax = 0.0;
    std::memcpy(&umax, &w->h_state[0].umax_bits, sizeof(double));
    std::memcpy(&gmax, &w->h_state[0].gmax_bits, sizeof(double));
    p.lcap = rescaled_lcap(umax, gmax, p.n, 2, p.omega);
    if (p.lcap == 0) {
      p.exact = true;
      w->slot.desc.sweep_tiles = w->n_sweep_tiles;
      SOR_CK(c, cudaMemcpyAsync(w->d_desc, &w->slot.desc, sizeof(SlotDesc), cudaMemcpyHostToDevice, s));
    }
  }
  if (p.kind == kPlain64 && !p.exact) SOR_CK(c, launch_ring_save(w->d_desc, s));  // ring kept for the rescaled phases

  // chunks, polled with a lag of kInflight - 1 so the device never idles
  const int L = chunk_length(c, p);
  const long long total_units =
      p.kind == kRefine ? (long long)(p.max_iters / p.inner) + 1 : (long long)p.max_iters;
  long long planned = 0;
  std::deque<int> inflight;
  int slot_i = 0;
  bool finished = (p.kind != kRefine && p.max_iters == 0);
  int last_iters = 0;  // device iteration count after the last harvested chunk (chunks harvest in order)
  long long updates_timed = 0;
  double ms_timed = 0.0;
  long long launches_timed = 0;
  auto harvest = [&](int k) -> sor_status {
    SOR_CK(c, cudaEventSynchronize(w->poll_events[k]));
    const SlotState& hs = w->h_state[k];
    if (hs.done) finished = true;
    if (timing) {
      float ms = 0.f;
      SOR_CK(c, cudaEventElapsedTime(&ms, w->chunk_events[k].first, w->chunk_events[k].second));
      const int di = hs.iters - last_iters;
      ms_timed += ms;
      updates_timed += (long long)di * p.n * p.n;
      launches_timed += p.kind == kRefine ? 2LL * di : 2LL * di;
    }
    last_iters = hs.iters;
    return SOR_OK;
  };
  if (cluster || grid || flow) {
    const int k = slot_i;
    if (timing) SOR_CK(c, cudaEventRecord(w->chunk_events[k].first, s));
    if (flow)
      SOR_CK(c, launch_grid_flow(fp32, p.n, w->slot.L.pitch, c->sm_count, w->d_desc, w->d_state, 0, w->d_gridsync,
                                 w->gridsync_bytes, s));
    else if (grid)
      SOR_CK(c, launch_grid_solve(p.kind == kPlain32, p.n, w->slot.L.pitch, c->sm_count, w->d_desc, w->d_state, 0,
                                  w->d_gridsync, s));
    else
      SOR_CK(c, launch_cluster_solve(p.kind == kPlain32, p.n, w->slot.L.pitch, w->d_desc, w->d_state, 0, s));
    if (timing) SOR_CK(c, cudaEventRecord(w->chunk_events[k].second, s));
    SOR_CK(c, cudaMemcpyAsync(&w->h_state[k], w->d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR_CK(c, cudaEventRecord(w->poll_events[k], s));
    rs = harvest(k);
    if (rs != SOR_OK) return rs;
    finished = true;
  }
  while (!finished && planned < total_units) {
    if ((int)inflight.size() == kInflight - 1) {
      rs = harvest(inflight.front());
      inflight.pop_front();
      if (rs != SOR_OK) return rs;
      if (finished) break;
    }
    const int k = slot_i;
    slot_i = (slot_i + 1) % kInflight;
    if (timing) SOR_CK(c, cudaEventRecord(w->chunk_events[k].first, s));
    const long long left = total_units - planned;
    const int Lc = (int)std::min<long long>(next_chunk(c, p, planned, L), left);
    rs = launch_chunk(c, w, p, Lc, s);
    if (rs != SOR_OK) return rs;
    planned += Lc;
    if (timing) SOR_CK(c, cudaEventRecord(w->chunk_events[k].second, s));
    SOR_CK(c, cudaMemcpyAsync(&w->h_state[k], w->d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR_CK(c, cudaEventRecord(w->poll_events[k], s));
    inflight.push_back(k);
  }
  while (!inflight.empty()) {
    rs = harvest(inflight.front());
    inflight.pop_front();
    if (rs != SOR_OK) return rs;
  }

  // residual of the returned iterate (plain kinds; refine measured it last)
  if (p.kind == kPlain64)
    SOR_CK(c, launch_resid(kResidFinal64, w->d_desc, w->d_state, w->d_resid_tiles, w->n_resid_tiles, 0, 0, s));
  else if (p.kind == kPlain32)
    SOR_CK(c, launch_resid(kResidFinal32, w->d_desc, w->d_state, w->d_resid_tiles, w->n_resid_tiles, 0, 0, s));

  // read the final state, then unpack the buffer it names
  SlotState fin;
  SOR_CK(c, cudaMemcpyAsync(&w->h_state[0], w->d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
  SOR_CK(c, cudaStreamSynchronize(s));
  fin = w->h_state[0];
  const bool out_dev = is_device_ptr(u_out);
  double* dout = out_dev ? u_out : w->d_nat_u;
  if (p.kind == kRefine) {
    SOR_CK(c, launch_unpack(d.u[fin.ubuf][0], d.u[fin.ubuf][1], false, p.n, w->slot.L.pitch, dout, s));
  } else {
    SOR_CK(c, launch_unpack(d.x[fin.xbuf][0], d.x[fin.xbuf][1], p.kind == kPlain32, p.n, w->slot.L.pitch, dout, s));
  }
  if (!out_dev) SOR_CK(c, cudaMemcpyAsync(u_out, dout, nat_u * 8, cudaMemcpyDeviceToHost, s));
  SOR_CK(c, cudaEventRecord(w->ev1, s));
  SOR_CK(c, cudaStreamSynchronize(s));
  float dev_ms = 0.f;
  SOR_CK(c, cudaEventElapsedTime(&dev_ms, w->ev0, w->ev1));
  if (fin.error) {
    c->set_error(fin.error == kErrBounds ? "device-side index check failed" : "device-side consistency check failed");
    return SOR_ERR_INTERNAL;
  }
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->iterations = fin.iters;
    res->converged = fin.converged;
    res->outer_steps = p.kind == kRefine ? fin.outer : 0;
    res->final_maxdelta = fin.last_dmax;
    res->final_resid_rel = fin.last_rho;
    res->latency_s = now_s() - t0;
    res->device_s = dev_ms * 1e-3;
  }
  {
    std::lock_guard<std::mutex> g(c->stats_mu);
    c->stats.solves += 1;
    c->stats.sweep_launches += 2ull * (unsigned long long)fin.iters;
    c->stats.lattice_updates += (unsigned long long)fin.iters * (unsigned long long)p.n * (unsigned long long)p.n;
    c->stats.sweep_ms += ms_timed;
    c->stats.timed_launches += (unsigned long long)launches_timed;
    c->stats.timed_updates += (unsigned long long)updates_timed;
    c->stats.kernel_launches += (kernel_launch_count() - launches0 - w->captured) + w->replayed;
  }
  return SOR_OK;
}

}  // namespace sorgb
