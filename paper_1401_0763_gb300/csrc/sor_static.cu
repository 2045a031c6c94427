// sor_solve_static: a blocking FP64 solve that allocates no memory.
//
// Who needs it: callers that must not allocate device memory while solving --
// code running under a fixed memory plan (real-time or embedded hosts that
// reserve every buffer up front), plug-ins whose host framework owns the
// device allocator, and code paths that may not call cudaMalloc at all.
// sor_solve creates its buffers with cudaMalloc (or the context's allocator);
// this entry point instead keeps all of its working memory -- the colour
// arrays, the source arrays, the solve state and the tile table -- in one
// file-scope __device__ array of fixed size, and the caller passes inputs
// and outputs already in device memory.
//
// The paper has no counterpart: it concerns library integration only.  The
// arithmetic is the exact-order FP64 path of sor_solve (SOR_FLAG_EXACT_ORDER),
// so results equal that path's bit for bit.
#include <cmath>
#include <cstring>
#include <mutex>

#include "sor_runtime.h"

namespace sorgb {
namespace {

constexpr int kStaticMaxN = 512;  // largest interior side the static scratch holds

constexpr int static_pitch(int n) {  // same pitch rule as Layout::make
  return (kOff + ((n + 1) / 2 + kWarpCols - 1) / kWarpCols * kWarpCols + 2 * kVec + 31) / 32 * 32;
}
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr int kStaticMaxTiles =
    ((kStaticMaxN + kTileRows - 1) / kTileRows) * (((kStaticMaxN + 1) / 2 + kWarpCols - 1) / kWarpCols);
constexpr size_t kArrayBytes = align256((size_t)(kStaticMaxN + 2) * static_pitch(kStaticMaxN) * sizeof(double));
constexpr size_t kDescOff = 0;
constexpr size_t kStateOff = kDescOff + align256(sizeof(SlotDesc));
constexpr size_t kTilesOff = kStateOff + align256(sizeof(SlotState));
constexpr size_t kArraysOff = kTilesOff + align256(sizeof(Tile) * kStaticMaxTiles);
constexpr size_t kScratchBytes = kArraysOff + 4 * kArrayBytes;  // about 4.8 MB

}  // namespace

// The scratch.  Every device that loads this library holds it until the
// process exits.  In host code the name is only a stand-in for the device
// address, so host code never passes it to a kernel directly: the device
// address comes from cudaGetSymbolAddress (static_scratch below).
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;                   // serialises host callers: every call shares the scratch
void* g_static_ptr[kMaxDevices] = {};     // device address of the scratch, per device

// Device address of the scratch on the current device (set up on the first
// call per device, with that device current).
cudaError_t static_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = (unsigned char*)g_static_ptr[dev];
  return cudaSuccess;
}

// Argument checks of the static path; the rules are those of sor_solve
// restricted to FP64 and N <= kStaticMaxN.
sor_status static_plan(const sor_params* p, bool has_f, Plan* out) {
  if (!p) return SOR_ERR_INVALID_ARG;
  if (p->n < 1 || p->n > kStaticMaxN) return SOR_ERR_INVALID_ARG;
  if (p->precision != SOR_FP64) return SOR_ERR_INVALID_ARG;
  if (p->stop != SOR_STOP_MAXDELTA && p->stop != SOR_STOP_RESID_REL) return SOR_ERR_INVALID_ARG;
  if (p->max_iters < 0 || p->check_every < 1 || p->inner_sweeps < 0) return SOR_ERR_INVALID_ARG;
  if ((p->flags & ~SOR_FLAG_EXACT_ORDER) || p->stall_window < 0) return SOR_ERR_INVALID_ARG;
  if (std::isnan(p->tol) || std::isnan(p->omega)) return SOR_ERR_INVALID_ARG;
  double w = p->omega <= 0.0 ? sor_omega_opt(p->n) : p->omega;
  if (!(w > 0.0 && w < 2.0)) return SOR_ERR_INVALID_ARG;
  Plan P;
  P.n = p->n;
  P.kind = kPlain64;
  P.exact = true;
  P.stop = p->stop == SOR_STOP_MAXDELTA ? kStopDelta : kStopResid;
  P.K = p->check_every;
  P.max_iters = p->max_iters;
  P.inner = 0;
  P.has_f = has_f;
  P.omega = w;
  P.tol = p->tol;
  P.stall = p->stall_window;
  *out = P;
  return SOR_OK;
}

#define SOR_SCK(expr)                  \
  do {                                 \
    if ((expr) != cudaSuccess) {       \
      cudaGetLastError();              \
      return SOR_ERR_CUDA;             \
    }                                  \
  } while (0)

// Failure after work was queued on the stream: wait for that work before the
// caller's lock on the scratch is dropped, so the next call cannot overwrite
// the scratch while it is still being read.
#define SOR_SCK_Q(expr, s)             \
  do {                                 \
    if ((expr) != cudaSuccess) {       \
      cudaGetLastError();              \
      cudaStreamSynchronize(s);        \
      cudaGetLastError();              \
      return SOR_ERR_CUDA;             \
    }                                  \
  } while (0)

// Device memory of the current device (the header requires inputs and
// outputs there): a pointer on another GPU, or host memory, is refused.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

constexpr int kStaticChunk = 32;  // iterations between polls of the solve state

}  // namespace
}  // namespace sorgb

using namespace sorgb;

extern "C" sor_status sor_solve_static(const sor_params* params, const double* u0, const double* f, double* u_out,
                                       sor_result* res, void* cuda_stream) {
  const double t0 = now_s();
  if (!u0 || !u_out) return SOR_ERR_INVALID_ARG;
  Plan plan;
  sor_status rs = static_plan(params, f != nullptr, &plan);
  if (rs != SOR_OK) return rs;
  int dev = -1;
  SOR_SCK(cudaGetDevice(&dev));
  if (!on_device(u0, dev) || !on_device(u_out, dev) || (f && !on_device(f, dev))) return SOR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_static_mu);
  unsigned char* base = nullptr;
  SOR_SCK(static_scratch(dev, &base));
  cudaStream_t s = (cudaStream_t)cuda_stream;

  const Layout L = Layout::make(plan.n);
  const size_t E = L.elems();
  SlotDesc* d_desc = (SlotDesc*)(base + kDescOff);
  SlotState* d_state = (SlotState*)(base + kStateOff);
  Tile* d_tiles = (Tile*)(base + kTilesOff);
  double* arr[4];
  for (int k = 0; k < 4; ++k) arr[k] = (double*)(base + kArraysOff + k * kArrayBytes);

  SlotDesc d;
  std::memset(&d, 0, sizeof(d));
  d.x[0][0] = arr[0];
  d.x[0][1] = arr[1];
  if (plan.has_f) {
    d.g[0] = arr[2];
    d.g[1] = arr[3];
    d.g64[0] = arr[2];
    d.g64[1] = arr[3];
  }
  d.n = plan.n;
  d.pitch = L.pitch;
  d.qmax = L.qmax;
  d.kind = kPlain64;
  d.K = plan.K;
  d.max_iters = plan.max_iters;
  d.stop = plan.stop;
  d.inner = 0;
  d.stall = plan.stall;
  d.a64 = 1.0 - plan.omega;
  d.b64 = plan.omega / 4.0;
  d.a32 = (float)d.a64;
  d.b32 = (float)d.b64;
  d.tol = plan.tol;
  // the scratch was sized with a copy of Layout::make's pitch rule: refuse
  // to run if the two ever disagree
  if (E * sizeof(double) > kArrayBytes || L.row_tiles() * L.col_tiles() > kStaticMaxTiles) return SOR_ERR_INTERNAL;
  Tile tiles[kStaticMaxTiles];
  int nt = 0;
  for (int r = 0; r < L.row_tiles(); ++r)
    for (int t = 0; t < L.col_tiles(); ++t)
      tiles[nt++] = Tile{0, 1 + r * kTileRows, 1 + t * kWarpCols, std::min(kTileRows, plan.n - r * kTileRows)};
  d.sweep_tiles = nt;
  d.resid_tiles = nt;
  SlotState st;
  std::memset(&st, 0, sizeof(st));
  st.checked_iter = -1;
  st.last_dmax = -1.0;
  st.last_rho = -1.0;
  st.best_rho = HUGE_VAL;
  st.done = plan.max_iters == 0;

  // The scratch keeps whatever the previous call left: clear the arrays this
  // call reads before it writes them (padding included), then upload the
  // descriptor, the zeroed state and the tile table.
  SOR_SCK_Q(cudaMemsetAsync(arr[0], 0, E * sizeof(double), s), s);
  SOR_SCK_Q(cudaMemsetAsync(arr[1], 0, E * sizeof(double), s), s);
  if (plan.has_f) {
    SOR_SCK_Q(cudaMemsetAsync(arr[2], 0, E * sizeof(double), s), s);
    SOR_SCK_Q(cudaMemsetAsync(arr[3], 0, E * sizeof(double), s), s);
  }
  SOR_SCK_Q(cudaMemcpyAsync(d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, s), s);
  SOR_SCK_Q(cudaMemcpyAsync(d_state, &st, sizeof(st), cudaMemcpyHostToDevice, s), s);
  SOR_SCK_Q(cudaMemcpyAsync(d_tiles, tiles, sizeof(Tile) * nt, cudaMemcpyHostToDevice, s), s);

  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.u0 = u0;
  pa.f = f;
  pa.n = plan.n;
  pa.pitch = L.pitch;
  const double h = 1.0 / (double)(plan.n + 1);
  pa.h2 = h * h;
  pa.fp32 = false;
  pa.x[0][0] = arr[0];
  pa.x[0][1] = arr[1];
  if (plan.has_f) {
    pa.g[0] = arr[2];
    pa.g[1] = arr[3];
  }
  pa.state = d_state;
  SOR_SCK_Q(launch_pack(pa, s), s);

  SlotState hs;
  long long planned = 0;
  bool finished = st.done != 0;
  while (!finished && planned < plan.max_iters) {
    const int Lc = (int)std::min<long long>(kStaticChunk, plan.max_iters - planned);
    for (int it = 0; it < Lc; ++it) {
      SOR_SCK_Q(launch_sweep(kSweepPlain64, d_desc, d_state, d_tiles, nt, 0, 0, 0, s), s);
      SOR_SCK_Q(launch_sweep(kSweepPlain64, d_desc, d_state, d_tiles, nt, 0, 1, 0, s), s);
      // residual tests fall on multiples of K only (as in sor_solve)
      if (plan.stop == kStopResid && (planned + it + 1) % plan.K == 0)
        SOR_SCK_Q(launch_resid(kResidCheck64, d_desc, d_state, d_tiles, nt, 0, 0, s), s);
    }
    planned += Lc;
    SOR_SCK_Q(cudaMemcpyAsync(&hs, d_state, sizeof(hs), cudaMemcpyDeviceToHost, s), s);
    SOR_SCK_Q(cudaStreamSynchronize(s), s);
    finished = hs.done != 0;
  }
  SOR_SCK_Q(launch_resid(kResidFinal64, d_desc, d_state, d_tiles, nt, 0, 0, s), s);
  SOR_SCK_Q(launch_unpack(arr[0], arr[1], false, plan.n, L.pitch, u_out, s), s);
  SOR_SCK_Q(cudaMemcpyAsync(&hs, d_state, sizeof(hs), cudaMemcpyDeviceToHost, s), s);
  SOR_SCK_Q(cudaStreamSynchronize(s), s);
  if (hs.error) return SOR_ERR_INTERNAL;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->iterations = hs.iters;
    res->converged = hs.converged;
    res->final_maxdelta = hs.last_dmax;
    res->final_resid_rel = hs.last_rho;
    res->latency_s = now_s() - t0;
    res->device_s = 0.0;
  }
  return SOR_OK;
}
