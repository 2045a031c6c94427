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
// colour: all blocks of a colour can run at once.  Each goes to a warp (or a
// segment of one, for blocks of 16 rows or fewer); a segment may take a run
// of several blocks of its block row one after another (narrow blocks).
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
// Data flow of a step: a lane has loaded (a few steps earlier) the east
// neighbour of its current cell and the old value of its next cell (the
// same cell inside a block; the next block's first cell at the end of a
// block in a run); the north value comes from lane r - 1 by a shuffle of its
// last result, the south value from lane r + 1 by a shuffle of that lane's
// next-cell value (one column behind, i.e. the old value of the cell below
// this one), the west value is the lane's own last result.  Only the
// block's first row, last row and first column read neighbours outside the
// block (cells of other-colour blocks or the Dirichlet ring, unchanged
// during the phase).  No cell is read from memory after a lane of the warp
// wrote it in the phase, so the lanes need no barrier beyond the shuffles.
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

#include "sor_bits.cuh"
#include "sor_devfn.cuh"
#include "sor_runtime.h"

namespace sorgb {
namespace {

constexpr int kBlkThreads = 128;  // residual pass
// A phase runs one warp per CTA: the warps share nothing, and a CTA per
// warp lets the block scheduler even out the warps per SM (with 4-warp CTAs,
// 512 CTAs on 152 SMs left some SMs a fourth CTA while the rest idled, 18 %
// of the cycles in ncu).
constexpr int kBlkPhaseWarps = 1;
constexpr int kBlkPhaseThreads = 32 * kBlkPhaseWarps;

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

// A warp segment's run: up to `chain` blocks of one block row of the phase's
// colour (block columns J, J + 2, ...), done back to back.  Position v =
// 0 .. total-1 walks the run's columns (block q covers v in [q*bx, q*bx +
// cols_q); only the last block of a run can be narrower, and a run never
// ends in an empty block).  Lane r updates position v at step r + v.
struct BlkRun {
  int i0, rows;  // the block row's first grid row and its rows
  int jb;        // grid column of the run's first cell
  int stride;    // grid columns from one block's first column to the next one's (2 bx)
  int total;     // positions in the run (0: no run)
};

// What a lane needs at position v of its run: the column jv of the cell (0
// when the lane is idle there, negated at a block's first column), its east
// neighbour, the old value of the lane's next cell (the east neighbour inside
// a block, the next block's first cell at a block's end), the north / south
// neighbour when the lane holds the block's first / last row, the west
// neighbour at a block's first column, and the source.  Every value read is
// old: the lane's own later cells are updated only by the lane, after their
// use, and the rows above and below the block row, the column left of a
// block and the source are not written in the phase.
// RUNS false (runs of one block): the next cell is always the east one and
// the west neighbour of the first column is read once, before the walk.
template <bool HAS_G, bool RUNS>
__device__ __forceinline__ void blk_fetch(int& jv, double& e, double& nf, double& nn, double& ss, double& w0,
                                          double& g, int v, int q, int c, const BlkRun& R, int bx, bool live,
                                          bool top, bool bottom, const double* __restrict__ Ur,
                                          const double* __restrict__ Un, const double* __restrict__ Us,
                                          const double* __restrict__ Gr) {
  const bool on = live && v >= 0 && v < R.total;
  const int j = R.jb + q * R.stride + c;
  jv = on ? (c == 0 ? -j : j) : 0;
  e = on ? Ur[j + 1] : 0.0;
  if (RUNS) {
    const bool block_end = c + 1 == bx || v + 1 == R.total;
    nf = (on && block_end && v + 1 < R.total) ? Ur[j + R.stride - bx + 1] : e;
    w0 = (on && c == 0) ? Ur[j - 1] : 0.0;
  } else {
    nf = e;
    w0 = 0.0;
  }
  nn = (on && top) ? Un[j] : 0.0;
  ss = (on && bottom) ? Us[j] : 0.0;
  g = (HAS_G && on) ? __ldg(Gr + j) : 0.0;
}

// One colour phase: every block of colour `colour`.  A warp is cut into
// 32 / SEG segments of SEG lanes (SEG the smallest power of two >= by,
// passed as seg_log2); each segment takes runs of up to `chain` blocks of one
// block row (numbered run = I * runs_per_row + h), so blocks of few rows
// still fill the warp and a wavefront ramps up and down once per run rather
// than once per block; the shuffles stay inside a segment.
// RUNS false: runs of one block (chain == 1), with fewer values in flight
// per lane (fewer registers: more warps per SM, measured faster for blocks
// of 128 columns or more).  MEASURE: fold |change| into st->dmax_bits.
template <bool HAS_G, bool MEASURE, bool RUNS>
__global__ void __launch_bounds__(kBlkPhaseThreads) k_blk_phase(double* __restrict__ U, const double* __restrict__ G,
                                                           int n, int pitch, int by, int bx, int nbr, int nbc,
                                                           int chain, int seg_log2, int colour, double a, double b,
                                                           SlotState* st) {
  if (*((volatile int*)&st->done)) return;
  const int lane = threadIdx.x & 31;
  const int segw = 1 << seg_log2, per_warp = 32 >> seg_log2;
  const int r = lane & (segw - 1);  // the lane's row in its block row
  const int slots = (nbc + 1) >> 1;
  const int runs_per_row = (slots + chain - 1) / chain;
  const long long nruns = (long long)nbr * runs_per_row;
  const long long tasks = (nruns + per_warp - 1) / per_warp;
  unsigned long long dm = 0;
  for (long long task = blockIdx.x * (long long)kBlkPhaseWarps + (threadIdx.x >> 5); task < tasks;
       task += (long long)gridDim.x * kBlkPhaseWarps) {
    const long long run = task * per_warp + (lane >> seg_log2);
    BlkRun R{1, 0, 1, 2 * bx, 0};
    if (run < nruns) {
      const int I = (int)(run / runs_per_row), h = (int)(run - (long long)I * runs_per_row);
      const int J = ((I + colour) & 1) + 2 * h * chain;  // first block column of the run
      if ((long long)J * bx < n) {
        // blocks J, J + 2, ... below nbc, at most `chain` of them
        const int nq = min(chain, (nbc - J + 1) >> 1);
        const int jlast0 = 1 + (J + 2 * (nq - 1)) * bx;  // first column of the run's last block
        const int cols_last = min(bx, n + 1 - jlast0);
        R.i0 = 1 + I * by;
        R.rows = min(by, n + 1 - R.i0);
        R.jb = 1 + J * bx;
        R.total = (nq - 1) * bx + cols_last;
        // the run's rows and columns with the neighbours it reads
        if (!dbg_range(R.i0 - 1, R.i0 + R.rows + 1, (long long)n + 2, st) ||
            !dbg_range(R.jb - 1, (long long)jlast0 + cols_last + 1, pitch, st))
          R.rows = R.total = 0;
      }
    }
    const bool live = r < R.rows;
    const int i = R.i0 + (live ? r : 0);
    double* __restrict__ Ur = U + (size_t)i * pitch;
    const double* __restrict__ Gr = HAS_G ? G + (size_t)i * pitch : nullptr;
    const double* __restrict__ Un = U + (size_t)(i - 1) * pitch;  // north row (another block row or the ring)
    const double* __restrict__ Us = U + (size_t)(i + 1) * pitch;  // south row
    const bool top = r == 0, bottom = r == R.rows - 1;
    double cur = (live && R.total > 0) ? Ur[R.jb] : 0.0;  // old value of the cell the lane updates next
    double last = 0.0;                                   // the lane's most recent result
    const double west_first = (!RUNS && live && R.total > 0) ? Ur[R.jb - 1] : 0.0;
    const int steps = __reduce_max_sync(0xffffffffu, (unsigned)max(R.total + R.rows - 1, 0));
    // fetch position fv, block fq and column fc in it (a run of one block:
    // fc = fv): loads run kBlkAhead steps ahead of their use
    int fv = -r, fq = 0, fc = 0;
    int jq[kBlkAhead];
    double qe[kBlkAhead], qf[kBlkAhead], qn[kBlkAhead], qs[kBlkAhead], qw[kBlkAhead], qg[kBlkAhead];
#pragma unroll
    for (int d = 0; d < kBlkAhead; ++d) {
      blk_fetch<HAS_G, RUNS>(jq[d], qe[d], qf[d], qn[d], qs[d], qw[d], qg[d], fv, RUNS ? fq : 0, RUNS ? fc : fv, R,
                             bx, live, top, bottom, Ur, Un, Us, Gr);
      if (++fv > 0 && RUNS && ++fc == bx) {
        fc = 0;
        ++fq;
      }
    }
    for (int t0 = 0; t0 < steps; t0 += kBlkAhead) {
#pragma unroll
      for (int d = 0; d < kBlkAhead; ++d) {
        const int v = t0 + d - r;
        const int j = abs(jq[d]);
        const bool first_col = jq[d] < 0;
        const double east = qe[d], next = qf[d], north_m = qn[d], south_m = qs[d], west0 = qw[d], gv = qg[d];
        blk_fetch<HAS_G, RUNS>(jq[d], qe[d], qf[d], qn[d], qs[d], qw[d], qg[d], fv, RUNS ? fq : 0,
                               RUNS ? fc : fv, R, bx, live, top, bottom, Ur, Un, Us, Gr);
        if (++fv > 0 && RUNS && ++fc == bx) {
          fc = 0;
          ++fq;
        }
        // to the lane above: the old value of the cell below its next one
        const double offer = (v == -1) ? cur : next;
        const double below = __shfl_down_sync(0xffffffffu, offer, 1, segw);
        const double above = __shfl_up_sync(0xffffffffu, last, 1, segw);
        if (j != 0) {
          const double north = top ? north_m : above;
          const double south = bottom ? south_m : below;
          const double west = first_col ? (RUNS ? west0 : west_first) : last;
          double sum = __dadd_rn(__dadd_rn(north, south), __dadd_rn(west, east));
          if (HAS_G) sum = __dadd_rn(sum, gv);
          const double nu = __dadd_rn(__dmul_rn(a, cur), __dmul_rn(b, sum));
          Ur[j] = nu;
          if (MEASURE) dm = umax64(dm, abs_bits(__dadd_rn(nu, -cur)));
          last = nu;
          cur = next;
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

template <bool HAS_G, bool MEASURE>
void launch_blk_phase2(int grid, cudaStream_t s, double* U, const double* G, int n, int pitch, int by, int bx,
                       int nbr, int nbc, int chain, int seg_log2, int colour, double a, double b, SlotState* st) {
  if (chain > 1)
    k_blk_phase<HAS_G, MEASURE, true><<<grid, kBlkPhaseThreads, 0, s>>>(U, G, n, pitch, by, bx, nbr, nbc, chain,
                                                                    seg_log2, colour, a, b, st);
  else
    k_blk_phase<HAS_G, MEASURE, false><<<grid, kBlkPhaseThreads, 0, s>>>(U, G, n, pitch, by, bx, nbr, nbc, 1, seg_log2,
                                                                     colour, a, b, st);
}

template <bool HAS_G>
void launch_blk_phase(bool measure, int grid, cudaStream_t s, double* U, const double* G, int n, int pitch, int by,
                      int bx, int nbr, int nbc, int chain, int seg_log2, int colour, double a, double b,
                      SlotState* st) {
  if (measure)
    launch_blk_phase2<HAS_G, true>(grid, s, U, G, n, pitch, by, bx, nbr, nbc, chain, seg_log2, colour, a, b, st);
  else
    launch_blk_phase2<HAS_G, false>(grid, s, U, G, n, pitch, by, bx, nbr, nbc, chain, seg_log2, colour, a, b, st);
}

// FP32 phases (precision SOR_FP32) stage each block in shared memory.  An
// FP32 step is short, so the FP64 kernel's loads from global memory (each
// lane walking its own row; L1 hit rate near 30 % in FP32) stall every step;
// here a warp segment copies its block with the surrounding halo, (rows + 2)
// x (cols + 2) cells, into its tile, runs the wavefront there and writes the
// block's cells back.  In the tile, lane r's cell of column c is (r + 1, c +
// 1): its north neighbour (tile row r) was written by lane r - 1 one step
// earlier, its south neighbour (tile row r + 2) is still old, its west one is
// the lane's last result and its east one is still old, as in row-major
// order; a __syncwarp after every step orders those writes and reads.  Tile
// rows are ws floats, ws even, so the lanes of a step (addresses r (ws - 1)
// apart) fall in different banks.  One-block runs only.
constexpr int kBlkGAhead = 8;  // steps between a source load and its use

// 4-byte asynchronous copy from global to shared memory.
__device__ __forceinline__ void blk_cp_async4(float* smem_dst, const float* gsrc) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(gsrc) : "memory");
}

template <bool HAS_G, bool MEASURE>
__global__ void __launch_bounds__(kBlkPhaseThreads) k_blk_phase_s(float* __restrict__ U, const float* __restrict__ G,
                                                                 int n, int pitch, int by, int bx, int nbr, int nbc,
                                                                 int seg_log2, int ws, int colour, float a, float b,
                                                                 SlotState* st) {
  extern __shared__ float blk_tile[];
  if (*((volatile int*)&st->done)) return;
  const int lane = threadIdx.x & 31;
  const int segw = 1 << seg_log2, per_warp = 32 >> seg_log2;
  const int r = lane & (segw - 1), seg = lane >> seg_log2;
  float* const tile = blk_tile + (size_t)seg * (by + 2) * ws;
  const int slots = (nbc + 1) >> 1;
  const long long nblk = (long long)nbr * slots;
  const long long tasks = (nblk + per_warp - 1) / per_warp;
  unsigned long long dm = 0;
  for (long long task = blockIdx.x; task < tasks; task += gridDim.x) {
    const long long w = task * per_warp + seg;
    int i0 = 1, j0 = 1, rows = 0, cols = 0;
    if (w < nblk) {
      const int I = (int)(w / slots);
      const int J = 2 * (int)(w - (long long)I * slots) + ((I + colour) & 1);
      if ((long long)J * bx < n) {
        i0 = 1 + I * by;
        j0 = 1 + J * bx;
        rows = min(by, n + 1 - i0);
        cols = min(bx, n + 1 - j0);
        if (!dbg_range(i0 - 1, i0 + rows + 1, (long long)n + 2, st) || !dbg_range(j0 - 1, j0 + cols + 1, pitch, st))
          rows = cols = 0;
      }
    }
    // stage rows i0-1 .. i0+rows and columns j0-1 .. j0+cols: asynchronous
    // copies, all in flight together, then one wait
    if (rows > 0)
      for (int rr = 0; rr < rows + 2; ++rr) {
        const float* __restrict__ src = U + (size_t)(i0 - 1 + rr) * pitch + (j0 - 1);
        for (int cc = r; cc < cols + 2; cc += segw) blk_cp_async4(tile + rr * ws + cc, src + cc);
      }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();
    const bool live = r < rows;
    float* const trow = tile + (r + 1) * ws;
    const float* __restrict__ Gr = HAS_G ? G + (size_t)(i0 + (live ? r : 0)) * pitch + j0 : nullptr;
    float cur = live ? trow[1] : 0.0f;  // old value of the cell the lane updates next
    float last = 0.0f;                  // the lane's most recent result
    const int steps = __reduce_max_sync(0xffffffffu, (unsigned)max(rows + cols - 1, 0));
    float qg[kBlkGAhead];
#pragma unroll
    for (int d = 0; d < kBlkGAhead; ++d) {
      const int c = d - r;
      qg[d] = (HAS_G && live && c >= 0 && c < cols) ? __ldg(Gr + c) : 0.0f;
    }
    for (int t0 = 0; t0 < steps; t0 += kBlkGAhead) {
#pragma unroll
      for (int d = 0; d < kBlkGAhead; ++d) {
        const int c = t0 + d - r;
        const float gv = qg[d];
        if (HAS_G) {
          const int cf = c + kBlkGAhead;
          qg[d] = (live && cf >= 0 && cf < cols) ? __ldg(Gr + cf) : 0.0f;
        }
        if (live && c >= 0 && c < cols) {
          const float north = tile[r * ws + c + 1];
          const float south = tile[(r + 2) * ws + c + 1];
          const float west = c == 0 ? trow[0] : last;
          const float east = trow[c + 2];
          float sum = radd(radd(north, south), radd(west, east));
          if (HAS_G) sum = radd(sum, gv);
          const float nu = radd(rmul(a, cur), rmul(b, sum));
          trow[c + 1] = nu;
          if (MEASURE) dm = umax64(dm, abs_bits(widen_f32(radd(nu, -cur))));
          last = nu;
          cur = east;
        }
        __syncwarp();
      }
    }
    // write the block's cells back
    for (int rr = 0; rr < rows; ++rr) {
      float* __restrict__ dst = U + (size_t)(i0 + rr) * pitch + j0;
      for (int cc = r; cc < cols; cc += segw) dst[cc] = tile[(rr + 1) * ws + cc + 1];
    }
    __syncwarp();  // the next task stages over the tile
  }
  if (MEASURE) {
    dm = warp_max64(dm);
    if (lane == 0 && dm) atomicMax(&st->dmax_bits, dm);
  }
}

void launch_blk_phase_s(bool measure, bool has_g, int grid, size_t smem, cudaStream_t s, float* U, const float* G,
                        int n, int pitch, int by, int bx, int nbr, int nbc, int seg_log2, int ws, int colour, float a,
                        float b, SlotState* st) {
  if (has_g) {
    if (measure)
      k_blk_phase_s<true, true><<<grid, kBlkPhaseThreads, smem, s>>>(U, G, n, pitch, by, bx, nbr, nbc, seg_log2, ws,
                                                                     colour, a, b, st);
    else
      k_blk_phase_s<true, false><<<grid, kBlkPhaseThreads, smem, s>>>(U, G, n, pitch, by, bx, nbr, nbc, seg_log2, ws,
                                                                      colour, a, b, st);
  } else {
    if (measure)
      k_blk_phase_s<false, true><<<grid, kBlkPhaseThreads, smem, s>>>(U, G, n, pitch, by, bx, nbr, nbc, seg_log2, ws,
                                                                      colour, a, b, st);
    else
      k_blk_phase_s<false, false><<<grid, kBlkPhaseThreads, smem, s>>>(U, G, n, pitch, by, bx, nbr, nbc, seg_log2,
                                                                       ws, colour, a, b, st);
  }
}

cudaError_t blk_phase_s_allow(size_t smem) {
  cudaError_t e = cudaSuccess;
  const int v = (int)smem;
  for (cudaError_t x : {cudaFuncSetAttribute(k_blk_phase_s<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, v),
                        cudaFuncSetAttribute(k_blk_phase_s<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, v),
                        cudaFuncSetAttribute(k_blk_phase_s<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, v),
                        cudaFuncSetAttribute(k_blk_phase_s<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             v)})
    if (x != cudaSuccess) e = x;
  return e;
}

// FP32 storage: the FP64 array rounded to nearest (every cell, the ring
// included), and back (exact).
__global__ void k_blk_narrow(const double* __restrict__ src, float* __restrict__ dst, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x)
    dst[t] = __double2float_rn(src[t]);
}
__global__ void k_blk_widen(const float* __restrict__ src, double* __restrict__ dst, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x)
    dst[t] = (double)src[t];
}

// The solve's device buffers; released when the solve returns, after the
// work queued on its stream has finished (an early error return must not
// free memory that queued kernels still use).
struct BlkBuffers {
  Ctx* c = nullptr;
  cudaStream_t s = nullptr;
  std::vector<void*> ptrs;
  size_t reserved = 0;
  void* get(size_t bytes) {
    void* p = ctx_dev_alloc(c, bytes);
    if (p) ptrs.push_back(p);
    return p;
  }
  ~BlkBuffers() {
    if (!ptrs.empty() && cudaStreamSynchronize(s) != cudaSuccess) cudaGetLastError();
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
  else if (p->precision != SOR_FP64 && p->precision != SOR_FP32) why << "block SOR runs in FP64 or FP32";
  else if (p->stop != SOR_STOP_MAXDELTA && p->stop != SOR_STOP_RESID_REL) why << "unknown stop rule";
  else if (p->precision == SOR_FP32 && p->stop != SOR_STOP_MAXDELTA) why << "FP32 block SOR stops on max|change|";
  else if (p->max_iters < 0 || p->check_every < 1) why << "max_iters >= 0 and check_every >= 1 required";
  else if (p->flags & ~SOR_FLAG_EXACT_ORDER) why << "unknown flags";
  else if (p->stall_window != 0) why << "block SOR has no stall rule: stall_window must be 0";
  else if (std::isnan(p->tol) || std::isnan(p->omega)) why << "tol and omega must not be NaN";
  else if (p->omega > 0.0 && !(p->omega < 2.0)) why << "omega must be in (0, 2)";
  // FP32: a shared-memory tile of (by + 2) x ws floats per warp segment
  int seg_log2 = 0;  // segments of 2^seg_log2 >= by lanes, one run of blocks each
  while ((1 << seg_log2) < by) ++seg_log2;
  const int ws = (bx + 2) % 2 == 0 ? bx + 2 : bx + 3;
  const size_t tile_bytes = (size_t)(32 >> seg_log2) * (by + 2) * ws * sizeof(float);
  if (why.str().empty() && p->precision == SOR_FP32 && tile_bytes > kBlockMaxTileBytes)
    why << "FP32 block SOR stages each block in shared memory: (32 / s) x (block_rows + 2) x (block_cols + 2) floats, "
           "s the smallest power of two >= block_rows, must stay within " << kBlockMaxTileBytes << " bytes";
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
  const bool f32 = p->precision == SOR_FP32;  // FP32 storage and arithmetic in the phases
  if (f32) bytes += (has_f ? 2 : 1) * nnat * sizeof(float);
  BlkBuffers B;
  B.c = c;
  B.s = c->stream;
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
  float* d_u32 = f32 ? (float*)B.get(nnat * sizeof(float)) : nullptr;
  float* d_g32 = (f32 && has_f) ? (float*)B.get(nnat * sizeof(float)) : nullptr;
  if (!d_u || (has_f && !d_g) || (has_f && !f_dev && !d_f) || !d_state || (f32 && !d_u32) ||
      (f32 && has_f && !d_g32)) {
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
  if (f32) {  // the FP32 iterate and source: each FP64 value rounded once
    k_blk_narrow<<<fill_grid, 256, 0, s>>>(d_u, d_u32, (long long)nnat);
    if (has_f) k_blk_narrow<<<fill_grid, 256, 0, s>>>(d_g, d_g32, (long long)nnat);
    SORB_CK(c, cudaGetLastError());
    SORB_CK(c, blk_phase_s_allow(tile_bytes));
  }

  const double a = 1.0 - w, b = w / 4.0;
  const float a32 = (float)a, b32 = (float)b;
  // blocks per run: set by the option, else enough for about 128 columns
  // when that raises the wavefront's busy lanes, L / (L + by - 1) for a run
  // of L columns, by more than 15 % (measured on the 4098^2 plate: runs of
  // several blocks cost about 8 % in bookkeeping, so 32 x 32 and 16 x 32
  // blocks gain from them, 16 x 64 and 8 x 64 lose)
  int chain = c->opt_block_chain.load();
  if (chain <= 0) {
    chain = std::max(1, 128 / bx);
    const double one = (double)bx / (bx + by - 1), run = (double)(chain * bx) / (chain * bx + by - 1);
    if (run < 1.15 * one) chain = 1;
  }
  chain = std::max(1, std::min(slots, f32 ? 1 : chain));  // the FP32 kernel runs one block per segment
  const long long nruns = (long long)nbr * ((slots + chain - 1) / chain);
  const long long tasks = (nruns + (32 >> seg_log2) - 1) / (32 >> seg_log2);
  const int grid = (int)std::max<long long>(1, std::min<long long>((tasks + kBlkPhaseWarps - 1) / kBlkPhaseWarps,
                                                                   (long long)c->sm_count * 64));
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
        if (f32)
          launch_blk_phase_s(measure, has_f, grid, tile_bytes, s, d_u32, d_g32, n, pitch, by, bx, nbr, nbc, seg_log2,
                             ws, colour, a32, b32, d_state);
        else if (has_f)
          launch_blk_phase<true>(measure, grid, s, d_u, d_g, n, pitch, by, bx, nbr, nbc, chain, seg_log2, colour,
                                 a, b, d_state);
        else
          launch_blk_phase<false>(measure, grid, s, d_u, nullptr, n, pitch, by, bx, nbr, nbc, chain, seg_log2,
                                  colour, a, b, d_state);
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
  if (f32) {
    k_blk_widen<<<fill_grid, 256, 0, s>>>(d_u32, d_u, (long long)nnat);
    SORB_CK(c, cudaGetLastError());
  }
  // residual of the final iterate (in FP64, of the returned values)
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
