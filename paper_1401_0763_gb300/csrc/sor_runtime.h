// Host runtime of the SOR library: context, device memory under a budget,
// per-solve device state, launch plans replayed as CUDA graphs, and the
// continuous-batching scheduler.  Exposed to C callers only through sor.h.
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sor.h"
#include "sor_device.cuh"
#include "sor_kernels.h"

namespace sorgb {

// A named NVTX range for the lifetime of the object: solves, batch steps,
// admissions and retirements show up on Nsight timelines (no cost unless a
// tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Ctx;

// Device memory of one slot (one problem) in the colour-split layout.
struct SlotBuffers {
  Layout L{};
  int kind = kPlain64;
  bool has_f = false;
  bool pingpong = false;  // second iterate buffer (temporally blocked sweeps)
  size_t bytes = 0;
  std::vector<void*> allocs;
  SlotDesc desc{};  // device pointers filled in; solver parameters set per solve
};

// Resolved parameters of one solve.
struct Plan {
  int n = 0;
  int kind = kPlain64;
  int stop = kStopDelta;
  int K = 1;
  int max_iters = 0;
  int inner = 20;
  bool exact = false;
  bool has_f = false;
  int tdepth = 1;  // FP32 sweeps: iterations fused per tile pass (1 = one launch per colour phase)
  int fkind = 0;   // FP32 sweeps: kernel family of the fused sweeps (FusedKind)
  int tseg = 0;    // FP32 sweeps, wavefront family: output rows per tile (0 = its default)
  int rchunk = 0;  // defect correction: corrections per graph between polls (0 = by grid size)
  int stall = 0;   // residual tests without a new minimum that end the solve (0 = never)
  int lcap = 0;    // FP64 default path: longest chunk the input magnitudes allow (0 = not yet known)
  double omega = 0.0;
  double tol = 0.0;
};

sor_status make_plan(const sor_params* p, bool has_f, Plan* out, std::string* why);
size_t slot_bytes(const Plan& p, bool pingpong);

// A cached CUDA graph keyed by the launch sequence it replays.
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  unsigned long long launches = 0;  // kernel launches one replay runs
};

// Workspace of sor_solve: slot buffers plus the small device tables, kept
// between solves of the same shape so buffers and graphs are reused.
struct SolveWorkspace {
  int n = -1, kind = -1;
  bool has_f = false;
  bool pingpong = false;
  int fkind = -1, tdepth = 0, tseg_rows = 0;  // shape of the fused-sweep tile table (ensure_fused_tiles)
  size_t tb_cap = 0;                          // tiles the table can hold
  SlotBuffers slot;
  SlotDesc* d_desc = nullptr;
  SlotState* d_state = nullptr;
  Tile* d_sweep_tiles = nullptr;
  Tile* d_resid_tiles = nullptr;
  Tile* d_fast_tiles = nullptr;  // warp strips of the rescaled FP64 phases
  Tile* d_tb_tiles = nullptr;    // tiles of the temporally blocked FP32 phases
  int n_sweep_tiles = 0, n_resid_tiles = 0, n_fast_tiles = 0, n_tb_tiles = 0;
  double* d_nat_u = nullptr;  // (n+2)^2 staging (host inputs / outputs)
  double* d_nat_f = nullptr;  // n^2 staging
  double* d_ring = nullptr;   // FP64: unscaled Dirichlet ring cells of both colours (SlotDesc::ring)
  unsigned* d_progress = nullptr;  // FP64 chunk launches: phases completed per strip
  void* d_gridsync = nullptr;      // small plates solved on a cooperative grid: barrier state
  size_t gridsync_bytes = 0;       // its size (the barrier-free form needs the larger one)
  int fast_ct = 0;                 // column tiles of the strip table (strips are rows x fast_ct)
  int chain_grid = 0;              // blocks of a chunk launch (0: chunk launches unavailable)
  std::map<std::string, void*> chain_phases;  // packed phase records per chunk length and omega
  unsigned long long captured = 0, replayed = 0;  // launch counting of the current solve
  SlotState* h_state = nullptr;  // pinned mirror, one per in-flight poll
  int h_state_count = 0;
  std::vector<cudaEvent_t> poll_events;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> chunk_events;
  std::map<std::string, GraphEntry> graphs;
  size_t bytes = 0;
};

// One queued or active batch request.
struct Request {
  uint64_t ticket = 0;
  Plan plan;
  std::vector<double> u0, f;  // host copies of the inputs
  bool cube = false;          // a cube (sor_batch_submit3d): solved whole by a cube worker
  sor_params p3{};            // its parameters
  double* u_out = nullptr;
  bool out_on_device = false;
  double t_submit = 0.0;
  // filled while active
  int slot = -1;
  size_t ntiles = 0;  // tiles of this request in the batch tile table
  SlotBuffers buf;
  double* d_stage = nullptr;  // natural staging for inputs / output
  size_t stage_bytes = 0;
  cudaEvent_t ev_start = nullptr;
};

struct Completed {
  sor_status status = SOR_OK;
  sor_result res{};
};

// What the autotuner chose for a size bucket: the fused FP32 sweep kernel
// (family, depth, rows per tile) and the corrections per defect-correction
// graph.
struct TuneChoice {
  int fkind = 0, tdepth = 1, tseg = 0, rchunk = 0;
};

struct Batcher;
struct BatcherDeleter {
  void operator()(Batcher* b) const;  // defined in sor_batch.cu
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  sor_alloc_fn alloc = nullptr;
  sor_free_fn free_ = nullptr;
  void* alloc_user = nullptr;
  size_t budget = 0;
  int sm_count = 0;

  std::mutex mem_mu;
  std::condition_variable mem_cv;
  std::atomic<bool> closing{false};  // sor_destroy has begun: waits for memory give up
  size_t reserved = 0, peak = 0;

  std::mutex solve_mu;  // serialises sor_solve callers
  std::unique_ptr<SolveWorkspace> ws;

  std::mutex err_mu;
  std::string last_error;

  std::mutex stats_mu;
  sor_stats stats{};

  // options
  std::atomic<int> opt_timing{0};
  std::atomic<int> opt_graphs{1};
  std::atomic<int> opt_chunk{0};
  std::atomic<int> opt_tdepth{0};
  std::atomic<int> opt_autotune{0};
  std::atomic<int> opt_max_slots{0};
  std::atomic<int> opt_cluster{1};
  std::atomic<int> opt_fast_chain{1};
  std::atomic<int> opt_fused_kernel{0};  // 0: by grid size, 1: tile family, 2: wavefront family
  std::atomic<int> opt_plain_step{0};    // batch plain slots: iterations per step (0: tuned online)
  std::atomic<int> opt_cube_depth{0};    // FP32 cube sweeps: iterations per blocked launch (0: per-phase flow)
  std::atomic<int> opt_block_chain{0};   // block SOR: blocks per warp-segment run (0: about 128 columns)

  std::mutex tune_mu;
  std::map<std::string, TuneChoice> tuned;  // autotuned choices per "<n bucket> <has source>"

  std::unique_ptr<Batcher, BatcherDeleter> batcher;
  std::mutex batcher_mu;

  void set_error(const std::string& s) {
    std::lock_guard<std::mutex> g(err_mu);
    last_error = s;
  }
};

// device memory accounting
sor_status ctx_reserve(Ctx* c, size_t bytes, bool wait, double timeout_s);
void ctx_release(Ctx* c, size_t bytes);
void* ctx_dev_alloc(Ctx* c, size_t bytes);
void ctx_dev_free(Ctx* c, void* p);

sor_status alloc_slot(Ctx* c, const Plan& p, bool pingpong, SlotBuffers* out);
void free_slot(Ctx* c, SlotBuffers* b);
void fill_desc(const Plan& p, SlotBuffers* b);
void build_tiles(const Layout& L, int slot, std::vector<Tile>* sweep, std::vector<Tile>* resid,
                 int tile_rows = kTileRows, int tile_cols = kWarpCols);

void build_strips(const Layout& L, int slot, int warps, std::vector<Tile>* out);
sor_status zero_slot(Ctx* c, const Plan& p, SlotBuffers* b, cudaStream_t s);
SlotState initial_state(const Plan& p);
void release_solve_workspace(Ctx* c);
void resolve_fused(Ctx* c, Plan* p);
void load_tune_cache(Ctx* c);
int refine_dbuf(const Plan& p);
sor_status solve_blocking(Ctx* c, const Plan& p, const double* u0, const double* f, double* u_out,
                          sor_result* res);

// Four-colour 9-point solve (sor_solve9); the caller holds solve_mu.
sor_status solve9_blocking(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                           sor_result* res);

// Block two-colour SOR (sor_solve_block, sor_block.cu); the caller holds
// solve_mu.  Blocks of by x bx cells, by <= kBlockMaxRows (a block's rows are
// the lanes of one warp).
constexpr int kBlockMaxN = 60000;
constexpr int kBlockMaxRows = 32;
constexpr size_t kBlockMaxTileBytes = 200 * 1024;  // FP32: shared-memory tiles of one warp's blocks
sor_status solve_block_blocking(Ctx* c, const sor_params* p, int by, int bx, const double* u0, const double* f,
                                double* u_out, sor_result* res);

// 3D cube solve (sor_solve3d); the caller holds solve_mu.
// Runs the flow kernels' bounded device-side wait on a counter preset to 0
// (nothing advances it: the wait gives up after `polls` polls) or 1.
sor_status diag_flow_wait(Ctx* c, int polls, int preset, int* timed_out);
// FP64 lane operations per second of the whole GPU on independent chains of
// FMAs (kind 0) or additions (kind 1) (sor_probe.cu).
sor_status diag_fp64_rate(Ctx* c, int kind, double* ops_per_s);
// Whether the device-side index checks are compiled in and fire (sor_probe.cu).
sor_status diag_bounds(Ctx* c, int* fired);
sor_status solve3d_blocking(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                            sor_result* res);
// The parts of a cube solve the batch scheduler uses (sor3d.cu): argument
// checks, the solve on a given stream (optionally waiting for budget), and an
// upper bound of the device bytes it reserves.
sor_status check_params3d(Ctx* c, const sor_params* p, const double* u0, const double* u_out);
sor_status run_cube(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out, sor_result* res,
                    cudaStream_t s, bool wait_budget);
size_t cube_bytes(const sor_params* p, bool has_f);
sor_status batch_submit3d(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                          uint64_t* ticket);

sor_status batch_submit(Ctx* c, const Plan& p, const double* u0, const double* f, double* u_out, uint64_t* ticket);
sor_status batch_poll(Ctx* c, uint64_t ticket, double timeout_s, sor_result* res);
void batch_shutdown(Ctx* c);

double now_s();
bool is_device_ptr(const void* p);

// Longest chunk of the rescaled FP64 phases that the inputs allow: umax =
// max |u0| (whole array), gmax = max |h^2 f|, n the interior side, dims 2
// (plate, scale factor 4 / omega per half iteration) or 3 (cube, 6 / omega).
// 0: the magnitudes leave no room even unscaled (or are not finite, zero or
// below 2^-960): the solve must take the exact-order phases.
int rescaled_lcap(double umax, double gmax, int n, int dims, double omega);

}  // namespace sorgb
