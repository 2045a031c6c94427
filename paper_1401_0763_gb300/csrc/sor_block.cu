// Block two-colour SOR (block-parallel SOR) on the 2D plate.
//
// Section 3.1 names block-parallel SOR beside red-black and multi-colour SOR
// as a parallel form of SOR without defining it; the reading built here:
// the interior is tiled into blocks of by rows x bx columns (block (I, J):
// rows 1 + I*by .., columns 1 + J*bx .., the last ones clipped at N), block
// (I, J) has colour (I + J) mod 2, an iteration updates every colour-0 block
// and then every colour-1 block, and inside a block the cells are updated in
// row-major order with the update of Eq. 1, each reading the newest value of
// every neighbour.  Blocks of one colour touch only at corners, so the
// 5-point stencil couples a block only to itself and to blocks of the other
// colour: all blocks of a colour run at once, one warp (or a segment of one,
// for blocks of 16 rows or fewer) each.
//
// Inside a block the row-major order is a chain (every cell reads its west
// and north neighbours' new values), but it is the same chain as a wavefront:
// lane r holds block row r and updates column c at step r + c.  At that step
// the cell's north neighbour was updated one step earlier by lane r - 1 and
// its west neighbour one step earlier by lane r itself, while its south and
// east neighbours are still old, exactly as in row-major order.  So every
// update reads the same values as the sequential order and the results equal
// it bit for bit (the operations are rounded one at a time in the order of
// the CPU reference: ((N + S) + (W + E)) [+ h^2 f], then (1-w) u + (w/4) s).
//
// Data flow of a step: a lane loads the east neighbour of its current cell
// (which becomes its own old value at the next step); the north value comes
// from lane r - 1 by a shuffle of its last result, the south value from lane
// r + 1 by a shuffle of the value that lane loaded this step (its east
// neighbour, one column behind, i.e. the old value of the cell below this
// one), the west value is the lane's own last result.  Only the block's
// first row, last row and first column read neighbours outside the block
// (cells of other-colour blocks or the Dirichlet ring, unchanged during the
// phase).  No cell is read from memory after a lane of the warp wrote it in
// the phase, so the lanes need no barrier beyond the shuffles.
//
// Storage is the natural (N+2)^2 row-major array: the method reads all four
// neighbours of a cell from one array, and a block's rows are contiguous.
// The arithmetic is FP64 in the exact order (6 FP64 operations per update,
// 7 with a source), so the phases are bound by GB300's FP64 rate.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <sstream>
#include <vector>

#include "sor_devfn.cuh"
#include "sor_runtime.h"

namespace sorgb {
namespace {

constexpr int kBlkWarps = 4;  // method blocks (one per warp) per CTA
constexpr int kBlkThreads = 32 * kBlkWarps;

#define SORB_CK(ctx, expr)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      std::ostringstream os_;                                                                 \
      os_ << #expr << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
      (ctx)->set_error(os_.str());                                                            \
      return SOR_ERR_CUDA;                                                                    \
    }                                                                                         \
  } while (0)

// g = h^2 f on the (N+2)^2 array (the ring stays 0, set by a memset).
__global__ void k_blk_source(const double* __restrict__ f, double* __restrict__ g, int n, int pitch, double h2) {
  const long long cells = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cells; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n) + 1, j = (int)(t % n) + 1;
    g[(size_t)i * pitch + j] = __dmul_rn(h2, f[t]);
  }
}

constexpr int kBlkAhead = 4;  // steps between a load and its use

// The values a lane needs at its column c (when 0 <= c < cols): its east
// neighbour, the north / south neighbour when it holds the block's first /
// last row, and the source.  Zero when the lane is idle at that column.
template <bool HAS_G>
__device__ __forceinline__ void blk_fetch(double& e, double& nn, double& ss, double& g, int c, bool live, bool top,
                                          bool bottom, int cols, int j0, const double* __restrict__ Ur,
                                          const double* __restrict__ Un, const double* __restrict__ Us,
                                          const double* __restrict__ Gr) {
  const bool on = live && c >= 0 && c < cols;
  const int j = j0 + c;
  e = on ? Ur[j + 1] : 0.0;
  nn = (on && top) ? Un[j] : 0.0;
  ss = (on && bottom) ? Us[j] : 0.0;
  g = (HAS_G && on) ? __ldg(Gr + j) : 0.0;
}

// One colour phase: every block of colour `colour`.  Blocks of the colour
// are numbered w = I * slots + k with J = 2k + ((I + colour) & 1), slots =
// ceil(nbc / 2); a number whose J lies past the last block column is
// skipped.  A warp is cut into 32 / SEG segments of SEG lanes (SEG the
// smallest power of two >= by, passed as seg_log2), one block per segment,
// so blocks of few rows still fill the warp and their wavefronts ramp up and
// down in by - 1 steps, not 31; the shuffles stay inside a segment.
// MEASURE: fold |change| into st->dmax_bits.
template <bool HAS_G, bool MEASURE>
__global__ void __launch_bounds__(kBlkThreads) k_blk_phase(double* __restrict__ U, const double* __restrict__ G,
                                                           int n, int pitch, int by, int bx, int nbr, int slots,
                                                           int seg_log2, int colour, double a, double b,
                                                           SlotState* st) {
  if (*((volatile int*)&st->done)) return;
  const int lane = threadIdx.x & 31;
  const int segw = 1 << seg_log2, per_warp = 32 >> seg_log2;
  const int r = lane & (segw - 1);  // the lane's row in its block
  const long long nblk = (long long)nbr * slots;
  const long long tasks = (nblk + per_warp - 1) / per_warp;
  unsigned long long dm = 0;
  for (long long task = blockIdx.x * (long long)kBlkWarps + (threadIdx.x >> 5); task < tasks;
       task += (long long)gridDim.x * kBlkWarps) {
    const long long w = task * per_warp + (lane >> seg_log2);
    int i0 = 1, j0 = 1, rows = 0, cols = 0;
    if (w < nblk) {
      const int I = (int)(w / slots);
      const int J = 2 * (int)(w - (long long)I * slots) + ((I + colour) & 1);
      if ((long long)J * bx < n) {
        i0 = 1 + I * by;
        j0 = 1 + J * bx;
        rows = min(by, n + 1 - i0);
        cols = min(bx, n + 1 - j0);
        // the block and the neighbours it reads: rows i0-1 .. i0+rows, columns j0-1 .. j0+cols
        if (!dbg_range(i0 - 1, i0 + rows + 1, (long long)n + 2, st) ||
            !dbg_range(j0 - 1, j0 + cols + 1, pitch, st))
          rows = cols = 0;
      }
    }
    const bool live = r < rows;
    const int i = i0 + (live ? r : 0);
    double* __restrict__ Ur = U + (size_t)i * pitch;
    const double* __restrict__ Gr = HAS_G ? G + (size_t)i * pitch : nullptr;
    const double* __restrict__ Un = U + (size_t)(i - 1) * pitch;  // north row (another block or the ring)
    const double* __restrict__ Us = U + (size_t)(i + 1) * pitch;  // south row
    const bool top = r == 0, bottom = r == rows - 1;
    double cur = live ? Ur[j0] : 0.0;          // old value of the cell the lane updates next
    const double west0 = live ? Ur[j0 - 1] : 0.0;  // west neighbour of its first cell (old)
    double last = 0.0;                         // the lane's most recent result
    const int steps = __reduce_max_sync(0xffffffffu, (unsigned)max(cols + rows - 1, 0));
    // Loads run kBlkAhead steps ahead of their use (all of them read old
    // values: a lane's east cells are updated only by the lane itself, after
    // their use; north / south rows of the first / last lane and the source
    // are not written in the phase), so the per-step chain holds only the
    // shuffles and the arithmetic.
    double qe[kBlkAhead], qn[kBlkAhead], qs[kBlkAhead], qg[kBlkAhead];
#pragma unroll
    for (int d = 0; d < kBlkAhead; ++d)
      blk_fetch<HAS_G>(qe[d], qn[d], qs[d], qg[d], d - r, live, top, bottom, cols, j0, Ur, Un, Us, Gr);
    for (int t0 = 0; t0 < steps; t0 += kBlkAhead) {
#pragma unroll
      for (int d = 0; d < kBlkAhead; ++d) {
        const int c = t0 + d - r;
        const bool act = live && c >= 0 && c < cols;
        const double east = qe[d], north_m = qn[d], south_m = qs[d], gv = qg[d];
        blk_fetch<HAS_G>(qe[d], qn[d], qs[d], qg[d], c + kBlkAhead, live, top, bottom, cols, j0, Ur, Un, Us, Gr);
        // to the lane above: the old value of the cell below its current one
        const double offer = (c == -1) ? cur : east;
        const double below = __shfl_down_sync(0xffffffffu, offer, 1, segw);
        const double above = __shfl_up_sync(0xffffffffu, last, 1, segw);
        if (act) {
          const double north = top ? north_m : above;
          const double south = bottom ? south_m : below;
          const double west = c == 0 ? west0 : last;
          double sum = __dadd_rn(__dadd_rn(north, south), __dadd_rn(west, east));
          if (HAS_G) sum = __dadd_rn(sum, gv);
          const double nu = __dadd_rn(__dmul_rn(a, cur), __dmul_rn(b, sum));
          Ur[j0 + c] = nu;
          if (MEASURE) dm = umax64(dm, abs_bits(__dadd_rn(nu, -cur)));
          last = nu;
          cur = east;
        }
      }
    }
  }
  if (MEASURE) {
    dm = warp_max64(dm);
    if (lane == 0 && dm) atomicMax(&st->dmax_bits, dm);
  }
}

// Scaled residual r~ = (g + ((N + S) + (W + E))) - 4u and b~ = g + (ring
// neighbours), in the order of the CPU reference; max|r~| and max|b~| into
// the state (a NaN in r~ is kept, as the reference keeps it; one in b~ is
// skipped, as the reference's comparison skips it).
template <bool HAS_G>
__global__ void __launch_bounds__(kBlkThreads) k_blk_resid(const double* __restrict__ U,
                                                           const double* __restrict__ G, int n, int pitch,
                                                           SlotState* st) {
  const long long cells = (long long)n * n;
  unsigned long long rm = 0, bm = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cells;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n) + 1, j = (int)(t % n) + 1;
    const double* __restrict__ Ur = U + (size_t)i * pitch;
    const double gij = HAS_G ? G[(size_t)i * pitch + j] : 0.0;
    const double nb = __dadd_rn(__dadd_rn(Ur[j - pitch], Ur[j + pitch]), __dadd_rn(Ur[j - 1], Ur[j + 1]));
    const double res = __dadd_rn(__dadd_rn(gij, nb), -__dmul_rn(4.0, Ur[j]));
    double bnd = 0.0;
    if (i == 1) bnd = __dadd_rn(bnd, Ur[j - pitch]);
    if (i == n) bnd = __dadd_rn(bnd, Ur[j + pitch]);
    if (j == 1) bnd = __dadd_rn(bnd, Ur[j - 1]);
    if (j == n) bnd = __dadd_rn(bnd, Ur[j + 1]);
    const double bt = __dadd_rn(gij, bnd);
    rm = umax64(rm, abs_bits(res));
    if (bt == bt) bm = umax64(bm, abs_bits(bt));
  }
  rm = warp_max64(rm);
  bm = warp_max64(bm);
  if ((threadIdx.x & 31) == 0) {
    if (rm) atomicMax(&st->rmax_bits, rm);
    if (bm) atomicMax(&st->bmax_bits, bm);
  }
}

// End of an iteration (one thread): count it, keep max|change| of a measured
// iteration, and at a multiple of K test it (or the residual) against tol.
__global__ void k_blk_end(SlotState* st, int K, int max_iters, int stop, double tol) {
  if (st->done) return;
  const int k = ++st->iters;
  const bool tested = (k % K) == 0;
  if (tested || k >= max_iters) {
    st->last_dmax = bits_to_double(st->dmax_bits);
    st->dmax_bits = 0ull;
  }
  if (tested) {
    double q = st->last_dmax;
    if (stop != kStopDelta) {
      const double rm = bits_to_double(st->rmax_bits), bm = bits_to_double(st->bmax_bits);
      q = bm > 0.0 ? __ddiv_rn(rm, bm) : rm;
      st->last_rho = q;
      st->rmax_bits = 0ull;
      st->bmax_bits = 0ull;
    }
    if (q < tol) {
      st->converged = 1;
      st->done = 1;
    }
  }
  if (k >= max_iters) st->done = 1;
}

template <bool HAS_G>
void launch_blk_phase(bool measure, int grid, cudaStream_t s, double* U, const double* G, int n, int pitch, int by,
                      int bx, int nbr, int slots, int seg_log2, int colour, double a, double b, SlotState* st) {
  if (measure)
    k_blk_phase<HAS_G, true><<<grid, kBlkThreads, 0, s>>>(U, G, n, pitch, by, bx, nbr, slots, seg_log2, colour, a, b,
                                                           st);
  else
    k_blk_phase<HAS_G, false><<<grid, kBlkThreads, 0, s>>>(U, G, n, pitch, by, bx, nbr, slots, seg_log2, colour, a,
                                                            b, st);
}

struct BlkBuffers {
  Ctx* c = nullptr;
  std::vector<void*> ptrs;
  size_t reserved = 0;
  void* get(size_t bytes) {
    void* p = ctx_dev_alloc(c, bytes);
    if (p) ptrs.push_back(p);
    return p;
  }
  ~BlkBuffers() {
    for (void* p : ptrs) ctx_dev_free(c, p);
    if (reserved) ctx_release(c, reserved);
  }
};

}  // namespace

sor_status solve_block_blocking(Ctx* c, const sor_params* p, int by, int bx, const double* u0, const double* f,
                                double* u_out, sor_result* res) {
  NvtxRange nvtx("sor_solve_block");
  const double t0 = now_s();
  if (!p || !u0 || !u_out) {
    c->set_error("params, u0 and u_out must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  std::ostringstream why;
  if (p->n < 1 || p->n > kBlockMaxN) why << "n must be in [1, " << kBlockMaxN << "]";
  else if (by < 1 || by > kBlockMaxRows) why << "block_rows must be in [1, " << kBlockMaxRows << "]";
  else if (bx < 1) why << "block_cols must be >= 1";
  else if (p->precision != SOR_FP64) why << "block SOR runs in FP64";
  else if (p->stop != SOR_STOP_MAXDELTA && p->stop != SOR_STOP_RESID_REL) why << "unknown stop rule";
  else if (p->max_iters < 0 || p->check_every < 1) why << "max_iters >= 0 and check_every >= 1 required";
  else if (p->flags & ~SOR_FLAG_EXACT_ORDER) why << "unknown flags";
  else if (p->stall_window != 0) why << "block SOR has no stall rule: stall_window must be 0";
  else if (std::isnan(p->tol) || std::isnan(p->omega)) why << "tol and omega must not be NaN";
  else if (p->omega > 0.0 && !(p->omega < 2.0)) why << "omega must be in (0, 2)";
  if (!why.str().empty()) {
    c->set_error(why.str());
    return SOR_ERR_INVALID_ARG;
  }
  const int n = p->n, m = n + 2, pitch = m;
  const size_t nnat = (size_t)m * m, nf = (size_t)n * n;
  const bool has_f = f != nullptr;
  const bool in_dev = is_device_ptr(u0), f_dev = has_f && is_device_ptr(f), out_dev = is_device_ptr(u_out);
  const double w = p->omega <= 0.0 ? sor_omega_opt(n) : p->omega;
  const int stop = p->stop == SOR_STOP_MAXDELTA ? kStopDelta : kStopResid;
  const int nbr = (n + by - 1) / by, nbc = (n + bx - 1) / bx, slots = (nbc + 1) / 2;

  // the iterate lives in u_out when that is device memory, else in a buffer
  size_t bytes = sizeof(SlotState) + 256;
  if (!out_dev) bytes += nnat * sizeof(double);
  if (has_f) bytes += nnat * sizeof(double) + (f_dev ? 0 : nf * sizeof(double));
  BlkBuffers B;
  B.c = c;
  sor_status rs = ctx_reserve(c, bytes, false, 0.0);
  if (rs != SOR_OK) {
    c->set_error("block SOR solve does not fit the device-memory budget");
    return rs;
  }
  B.reserved = bytes;
  double* d_u = out_dev ? u_out : (double*)B.get(nnat * sizeof(double));
  double* d_g = has_f ? (double*)B.get(nnat * sizeof(double)) : nullptr;
  double* d_f = (has_f && !f_dev) ? (double*)B.get(nf * sizeof(double)) : nullptr;
  SlotState* d_state = (SlotState*)B.get(sizeof(SlotState));
  if (!d_u || (has_f && !d_g) || (has_f && !f_dev && !d_f) || !d_state) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  cudaStream_t s = c->stream;
  SlotState st;
  std::memset(&st, 0, sizeof(st));
  st.checked_iter = -1;
  st.last_dmax = 0.0;
  st.last_rho = -1.0;
  st.done = p->max_iters == 0;
  SORB_CK(c, cudaMemcpyAsync(d_state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  if (d_u != u0)
    SORB_CK(c, cudaMemcpyAsync(d_u, u0, nnat * sizeof(double), in_dev ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyHostToDevice, s));
  const int fill_grid = c->sm_count * 8;
  if (has_f) {
    const double* f_src = f;
    if (!f_dev) {
      SORB_CK(c, cudaMemcpyAsync(d_f, f, nf * sizeof(double), cudaMemcpyHostToDevice, s));
      f_src = d_f;
    }
    SORB_CK(c, cudaMemsetAsync(d_g, 0, nnat * sizeof(double), s));
    const double h = 1.0 / (double)(n + 1);
    k_blk_source<<<fill_grid, 256, 0, s>>>(f_src, d_g, n, pitch, h * h);
    SORB_CK(c, cudaGetLastError());
  }

  const double a = 1.0 - w, b = w / 4.0;
  int seg_log2 = 0;  // segments of 2^seg_log2 >= by lanes, one block each
  while ((1 << seg_log2) < by) ++seg_log2;
  const long long nblk = (long long)nbr * slots;
  const long long tasks = (nblk + (32 >> seg_log2) - 1) / (32 >> seg_log2);
  const int grid = (int)std::max<long long>(1, std::min<long long>((tasks + kBlkWarps - 1) / kBlkWarps,
                                                                   (long long)c->sm_count * 16));
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SORB_CK(c, cudaEventCreate(&ev0));
  if (cudaEventCreate(&ev1) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(ev0);
    c->set_error("event creation failed");
    return SOR_ERR_CUDA;
  }
  SlotState* h_state = nullptr;
  if (cudaMallocHost(&h_state, sizeof(SlotState)) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    c->set_error("pinned allocation failed");
    return SOR_ERR_OOM;
  }
  struct Cleanup {
    cudaEvent_t a, b;
    SlotState* hs;
    ~Cleanup() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaFreeHost(hs);
    }
  } cl{ev0, ev1, h_state};

  // iterations between host polls of the state; the device skips the rest of
  // a batch once the test has passed
  const int chunk = c->opt_chunk.load() > 0 ? c->opt_chunk.load() : 64;
  SORB_CK(c, cudaEventRecord(ev0, s));
  long long planned = 0;
  bool finished = st.done != 0;
  while (!finished && planned < p->max_iters) {
    const int Lc = (int)std::min<long long>(chunk, p->max_iters - planned);
    for (int it = 1; it <= Lc; ++it) {
      const long long k = planned + it;
      const bool tested = k % p->check_every == 0;
      const bool measure = tested || k == p->max_iters;
      for (int colour = 0; colour < 2; ++colour) {
        if (has_f)
          launch_blk_phase<true>(measure, grid, s, d_u, d_g, n, pitch, by, bx, nbr, slots, seg_log2, colour, a, b,
                                 d_state);
        else
          launch_blk_phase<false>(measure, grid, s, d_u, nullptr, n, pitch, by, bx, nbr, slots, seg_log2, colour, a,
                                  b, d_state);
      }
      if (stop == kStopResid && tested) {
        if (has_f)
          k_blk_resid<true><<<fill_grid, kBlkThreads, 0, s>>>(d_u, d_g, n, pitch, d_state);
        else
          k_blk_resid<false><<<fill_grid, kBlkThreads, 0, s>>>(d_u, nullptr, n, pitch, d_state);
      }
      k_blk_end<<<1, 1, 0, s>>>(d_state, p->check_every, p->max_iters, stop, p->tol);
    }
    SORB_CK(c, cudaGetLastError());
    planned += Lc;
    SORB_CK(c, cudaMemcpyAsync(h_state, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SORB_CK(c, cudaStreamSynchronize(s));
    finished = h_state->done != 0 || h_state->error != 0;
  }
  SORB_CK(c, cudaEventRecord(ev1, s));
  // residual of the final iterate
  SORB_CK(c, cudaMemsetAsync(&d_state->rmax_bits, 0, 2 * sizeof(unsigned long long), s));
  if (has_f)
    k_blk_resid<true><<<fill_grid, kBlkThreads, 0, s>>>(d_u, d_g, n, pitch, d_state);
  else
    k_blk_resid<false><<<fill_grid, kBlkThreads, 0, s>>>(d_u, nullptr, n, pitch, d_state);
  SORB_CK(c, cudaGetLastError());
  if (!out_dev) SORB_CK(c, cudaMemcpyAsync(u_out, d_u, nnat * sizeof(double), cudaMemcpyDeviceToHost, s));
  SORB_CK(c, cudaMemcpyAsync(h_state, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
  SORB_CK(c, cudaStreamSynchronize(s));
  float ms = 0.0f;
  SORB_CK(c, cudaEventElapsedTime(&ms, ev0, ev1));
  if (h_state->error) {
    c->set_error("device-side consistency check failed");
    return SOR_ERR_INTERNAL;
  }
  if (res) {
    double rm, bm;
    std::memcpy(&rm, &h_state->rmax_bits, sizeof(double));
    std::memcpy(&bm, &h_state->bmax_bits, sizeof(double));
    std::memset(res, 0, sizeof(*res));
    res->iterations = h_state->iters;
    res->converged = h_state->converged;
    res->final_maxdelta = h_state->last_dmax;
    res->final_resid_rel = bm > 0.0 ? rm / bm : rm;
    res->latency_s = now_s() - t0;
    res->device_s = ms * 1e-3;
  }
  return SOR_OK;
}

}  // namespace sorgb
