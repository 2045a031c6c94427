// Four-colour SOR on the compact 9-point stencil.  Section 3.1 names
// multi-colour SOR beside red-black SOR as a parallel ordering; the 9-point
// stencil also couples diagonal neighbours, so four colours are needed for
// the cells of one colour to be independent:
//   colour c = 2 (i & 1) + (j & 1), phases in the order 0, 1, 2, 3.
// Cell equation 20 u = 4 (N + S + W + E) + (NW + NE + SW + SE) + 6 h^2 f, and
// the update (Eq. 1 with this Gauss-Seidel value), summed in this order:
//   s4 = (N + S) + (W + E),  sd = (NW + NE) + (SW + SE),
//   s = (4 s4 + sd) [+ g],   u <- (1-w) u + (w/20) s,   g = 6 h^2 f.
// Every product and sum is rounded on its own, so FP64 and FP32 results equal
// the CPU oracle's bit for bit.
//
// Storage: four quarter arrays.  Cell (i, j) lives in quarter c at row
// a = (i + 1) >> 1 and column b = (j + 1) >> 1, element a * pitch + b + kOff,
// so with pi = c >> 1, pj = c & 1 the interior of quarter c is
// 1 <= a <= (N + pi) / 2, 1 <= b <= (N + pj) / 2 (aligned vectors from b = 1)
// and the eight neighbours of (a, b) are, in quarters c^2, c^1 and c^3:
//   N = [a - pi][b],  S = [a + 1 - pi][b]                       (quarter c ^ 2)
//   W = [a][b - pj],  E = [a][b + 1 - pj]                       (quarter c ^ 1)
//   NW, NE, SW, SE = [a - pi or a + 1 - pi][b - pj or b + 1 - pj] (quarter c ^ 3)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <sstream>
#include <vector>

#include "sor_devfn.cuh"
#include "sor_strips.cuh"
#include "sor_bits.cuh"
#include "sor_runtime.h"

namespace sorgb {
namespace {

__device__ __forceinline__ size_t e9(int a, int b, int pitch) {
  return (size_t)a * (size_t)pitch + (size_t)(b + kOff);
}

// Debug check (SOR_DEBUG_BOUNDS) of a work item that touches quarter rows
// [a0, a1) and columns [b0, b1) of the quarter arrays ((N+1)/2 + 2 rows): on
// failure the state records kErrBounds and stops; release builds compile it
// to true.
__device__ __forceinline__ bool dbg_tile9(SlotState* st, int a0, int a1, int b0, int b1, int n, int pitch) {
  if (dbg_range(a0, a1, ((n + 1) >> 1) + 2, st) && dbg_range((long long)b0 + kOff, (long long)b1 + kOff, pitch, st))
    return true;
  st->done = 1;
  return false;
}

struct Desc9 {
  void* x[4];            // quarter arrays (FP64 or FP32)
  const void* g[4];      // 6 h^2 f per quarter in the sweep type, or null
  const double* g64[4];  // 6 h^2 f in FP64 for the residual, or null
  int n, pitch, K, max_iters, stop, tiles;
  float a32, b32;        // (float)(1 - w), (float)(w / 20)
  double a64, b64;       // 1 - w, w / 20
  double tol;
  int stall;             // residual stop: stall window (0 = off), the 2D rule
  float* rhs32[4];       // defect correction, residual pass: r~ rounded to FP32, per quarter (else null)
  SlotState* inner;      // defect correction, residual pass: the inner solve's state (skipped once converged)
  double* ucorr[4];      // defect correction, inner sweeps: u, corrected by the final d (else null)
  SlotState* outer;      // defect correction, inner sweeps: the outer state (counts corrections)
};

// Natural (N+2)^2 <-> quarters; interior cells also get 6 h^2 f and
// contribute |b~| = |g + (4 (edge ring neighbours) + (diagonal ring
// neighbours))| to ||b~||_inf.
template <typename T>
__global__ void k_pack9(const double* __restrict__ u0, const double* __restrict__ f, int n, int pitch, double s6,
                        T* x0, T* x1, T* x2, T* x3, T* g0, T* g1, T* g2, T* g3, double* h0, double* h1, double* h2,
                        double* h3, SlotState* st) {
  __shared__ unsigned long long red[kWarpsY];
  const int m = n + 2;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  unsigned long long bb = 0;
  if (j < m) {
    const int c = 2 * (i & 1) + (j & 1);
    const size_t e = e9((i + 1) >> 1, (j + 1) >> 1, pitch);
    T* X[4] = {x0, x1, x2, x3};
    T* G[4] = {g0, g1, g2, g3};
    double* H[4] = {h0, h1, h2, h3};
    const double v = u0[(size_t)i * m + j];
    X[c][e] = (T)v;
    const bool interior = i >= 1 && i <= n && j >= 1 && j <= n;
    double gc = 0.0;
    if (interior && f) gc = __dmul_rn(s6, f[(size_t)(i - 1) * n + (j - 1)]);
    if (G[c]) G[c][e] = (T)gc;
    if (H[c]) H[c][e] = gc;
    if (interior) {
      auto U = [&](int ii, int jj) { return u0[(size_t)ii * m + jj]; };
      double b4 = 0.0, bd = 0.0;
      if (i == 1) b4 = __dadd_rn(b4, U(0, j));
      if (i == n) b4 = __dadd_rn(b4, U(n + 1, j));
      if (j == 1) b4 = __dadd_rn(b4, U(i, 0));
      if (j == n) b4 = __dadd_rn(b4, U(i, n + 1));
      if (i == 1 || j == 1) bd = __dadd_rn(bd, U(i - 1, j - 1));
      if (i == 1 || j == n) bd = __dadd_rn(bd, U(i - 1, j + 1));
      if (i == n || j == 1) bd = __dadd_rn(bd, U(i + 1, j - 1));
      if (i == n || j == n) bd = __dadd_rn(bd, U(i + 1, j + 1));
      bb = abs_bits(__dadd_rn(gc, __dadd_rn(__dmul_rn(4.0, b4), bd)));
    }
  }
  block_max_to(bb, &st->bmax_bits, red);
}

template <typename T>
__global__ void k_unpack9(const T* __restrict__ x0, const T* __restrict__ x1, const T* __restrict__ x2,
                          const T* __restrict__ x3, int n, int pitch, double* u) {
  const int m = n + 2;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= m) return;
  const T* X[4] = {x0, x1, x2, x3};
  u[(size_t)i * m + j] = (double)X[2 * (i & 1) + (j & 1)][e9((i + 1) >> 1, (j + 1) >> 1, pitch)];
}

// The W and E vectors of a quarter row v (this lane's columns q0..q0+3) for
// column parity PJ: PJ = 0 -> W = v, E = v shifted left by one; PJ = 1 ->
// W = v shifted right by one, E = v.  The value crossing into the next or
// previous lane comes by a shuffle, at the warp's edges from memory.
template <typename T, int PJ>
__device__ __forceinline__ void we_of(const T (&v)[4], const T* __restrict__ rowp, int q0, int lane, T (&W)[4],
                                      T (&E)[4]) {
  if (PJ == 0) {
    T r = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lane == 31) r = rowp[q0 + kVec + kOff];
    W[0] = v[0]; W[1] = v[1]; W[2] = v[2]; W[3] = v[3];
    E[0] = v[1]; E[1] = v[2]; E[2] = v[3]; E[3] = r;
  } else {
    T l = __shfl_up_sync(0xffffffffu, v[3], 1);
    if (lane == 0) l = rowp[q0 - 1 + kOff];
    W[0] = l; W[1] = v[0]; W[2] = v[1]; W[3] = v[2];
    E[0] = v[0]; E[1] = v[1]; E[2] = v[2]; E[3] = v[3];
  }
}

// Rows [a0, a1) of quarter C for one warp, exact order.
template <typename T, int C, bool MEASURE, bool HAS_G>
__device__ __forceinline__ unsigned long long sweep9_rows(const Desc9& d, int q0, int a0, int a1, int lane) {
  constexpr int PI = C >> 1, PJ = C & 1;
  unsigned long long dm = 0;
  unsigned dm32 = 0;
  if (a0 >= a1) return 0;
  T* X = (T*)d.x[C];
  const T* Q1 = (const T*)d.x[C ^ 1];
  const T* Q2 = (const T*)d.x[C ^ 2];
  const T* Q3 = (const T*)d.x[C ^ 3];
  const T* G = (const T*)d.g[C];
  const int pitch = d.pitch;
  const int blim = (d.n + PJ) >> 1;
  const T a = sizeof(T) == 4 ? (T)d.a32 : (T)d.a64;
  const T b = sizeof(T) == 4 ? (T)d.b32 : (T)d.b64;
  const T four = T(4);
  T n2[4], n3[4];
  load4(Q2 + e9(a0 - PI, q0, pitch), n2);
  load4(Q3 + e9(a0 - PI, q0, pitch), n3);
  for (int r = a0; r < a1; ++r) {
    T s2[4], s3[4], w1[4], own[4], gv[4];
    load4(Q2 + e9(r + 1 - PI, q0, pitch), s2);
    load4(Q3 + e9(r + 1 - PI, q0, pitch), s3);
    load4(Q1 + e9(r, q0, pitch), w1);
    load4(X + e9(r, q0, pitch), own);
    if (HAS_G) load4(G + e9(r, q0, pitch), gv);
    T W[4], E[4], NW[4], NE[4], SW[4], SE[4];
    we_of<T, PJ>(w1, Q1 + (size_t)r * pitch, q0, lane, W, E);
    we_of<T, PJ>(n3, Q3 + (size_t)(r - PI) * pitch, q0, lane, NW, NE);
    we_of<T, PJ>(s3, Q3 + (size_t)(r + 1 - PI) * pitch, q0, lane, SW, SE);
    T nv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const T s4 = radd(radd(n2[v], s2[v]), radd(W[v], E[v]));
      const T sd = radd(radd(NW[v], NE[v]), radd(SW[v], SE[v]));
      T s = radd(rmul(four, s4), sd);
      if (HAS_G) s = radd(s, gv[v]);
      const T nu = radd(rmul(a, own[v]), rmul(b, s));
      const bool in = (q0 + v) <= blim;
      nv[v] = in ? nu : own[v];  // cells past the interior keep their value
      if (MEASURE && in) {
        if (sizeof(T) == 4)
          dm32 = max(dm32, abs_bits32((float)radd(nu, -own[v])));
        else
          dm = umax64(dm, abs_bits((double)radd(nu, -own[v])));
      }
    }
    store4(X + e9(r, q0, pitch), nv);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      n2[v] = s2[v];
      n3[v] = s3[v];
    }
  }
  if (sizeof(T) == 4 && MEASURE) dm = abs_bits_of(__uint_as_float(dm32));
  return dm;
}

// Rows [a0, a1) of quarter C for one warp, FP64 default.  The north triple
// T_N = NW + 4 N + NE of a cell and the south triple T_S = SW + 4 S + SE hold
// the same three cells when T_S belongs to the cell one quarter row up (two
// natural rows), so each row forms only its T_S and inherits T_N:
//   s = fma(4, W + E, T_N + T_S) [+ g],   u <- fma(1 - w, u, (w/20) s),
// 7 FP64 operations per update (11 in the exact order, which this equals
// within rounding: 1e-12 of it over the solves tested).
template <int C, bool MEASURE, bool HAS_G>
__device__ __forceinline__ unsigned long long sweep9_fast_rows(const Desc9& d, int q0, int a0, int a1, int lane) {
  constexpr int PI = C >> 1, PJ = C & 1;
  unsigned long long dm = 0;
  if (a0 >= a1) return 0;
  double* X = (double*)d.x[C];
  const double* Q1 = (const double*)d.x[C ^ 1];
  const double* Q2 = (const double*)d.x[C ^ 2];
  const double* Q3 = (const double*)d.x[C ^ 3];
  const double* G = (const double*)d.g[C];
  const int pitch = d.pitch;
  const int blim = (d.n + PJ) >> 1;
  const double a = d.a64, b = d.b64;
  double tn[4];
  {
    double n2[4], n3[4], NW[4], NE[4];
    load4(Q2 + e9(a0 - PI, q0, pitch), n2);
    load4(Q3 + e9(a0 - PI, q0, pitch), n3);
    we_of<double, PJ>(n3, Q3 + (size_t)(a0 - PI) * pitch, q0, lane, NW, NE);
#pragma unroll
    for (int v = 0; v < 4; ++v) tn[v] = __fma_rn(4.0, n2[v], __dadd_rn(NW[v], NE[v]));
  }
  for (int r = a0; r < a1; ++r) {
    double s2[4], s3[4], w1[4], own[4], gv[4];
    load4(Q2 + e9(r + 1 - PI, q0, pitch), s2);
    load4(Q3 + e9(r + 1 - PI, q0, pitch), s3);
    load4(Q1 + e9(r, q0, pitch), w1);
    load4(X + e9(r, q0, pitch), own);
    if (HAS_G) load4(G + e9(r, q0, pitch), gv);
    double W[4], E[4], SW[4], SE[4];
    we_of<double, PJ>(w1, Q1 + (size_t)r * pitch, q0, lane, W, E);
    we_of<double, PJ>(s3, Q3 + (size_t)(r + 1 - PI) * pitch, q0, lane, SW, SE);
    double nv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double ts = __fma_rn(4.0, s2[v], __dadd_rn(SW[v], SE[v]));
      double sum = __fma_rn(4.0, __dadd_rn(W[v], E[v]), __dadd_rn(tn[v], ts));
      if (HAS_G) sum = __dadd_rn(sum, gv[v]);
      const double nu = __fma_rn(a, own[v], __dmul_rn(b, sum));
      const bool in = (q0 + v) <= blim;
      nv[v] = in ? nu : own[v];  // cells past the interior keep their value
      if (MEASURE && in) dm = umax64(dm, abs_bits(__dadd_rn(nu, -own[v])));
      tn[v] = ts;
    }
    store4(X + e9(r, q0, pitch), nv);
  }
  return dm;
}

__device__ __forceinline__ void finalize9(const Desc9& d, SlotState* st, int k, int measure) {
  st->arrive = 0;
  st->iters = k;
  if (measure) {
    const double mk = bits_to_double(atomicExch(&st->dmax_bits, 0ull));
    st->last_dmax = mk;
    if (d.stop == kStopDelta && (k % d.K) == 0 && mk < d.tol) {
      st->done = 1;
      st->converged = 1;
    }
  }
  if (k >= d.max_iters) st->done = 1;
}

// One colour phase over tiles (quarter rows, 128 columns), the FP32 phases:
// their phases are short (about 9 us on a 4098^2 plate), so a launch per
// phase beats the data-flow schedule, whose per-item claims, waits and
// fences sit on the critical path of every phase.  The last tile of the
// phase of colour 3 closes the iteration.
// u += (double)d over the interior cells of quarter C in rows [a0, a1) (this
// lane's columns), d just written by this lane.
template <int C>
__device__ __forceinline__ void correct9_rows(const Desc9& d, const float* __restrict__ D, int q0, int a0, int a1) {
  double* U = d.ucorr[C];
  const int pitch = d.pitch, blim = (d.n + (C & 1)) >> 1;
  for (int r = a0; r < a1; ++r) {
    double u[4];
    float dv[4];
    load4(U + e9(r, q0, pitch), u);
    load4(D + e9(r, q0, pitch), dv);
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if ((q0 + v) <= blim) u[v] = __dadd_rn(u[v], widen_f32(dv[v]));  // the widening is exact
    store4(U + e9(r, q0, pitch), u);
  }
}

// CORRECT (the inner sweeps of the defect correction, FP32): the phase of the
// last iteration also adds the quarter's final d to u, and the last tile of
// colour 3 counts the correction.
template <typename T, int C, bool CORRECT = false>
__global__ void __launch_bounds__(kThreads) k_sweep9(const Desc9* __restrict__ dp, SlotState* st,
                                                     const Tile* __restrict__ tiles, int ntiles) {
  __shared__ unsigned long long red[kWarpsY];
  __shared__ int ctl[3];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const Desc9& d = *dp;
  const int alim = (d.n + (C >> 1)) >> 1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    if (threadIdx.x == 0) {
      const int kk = *((volatile int*)&st->iters) + 1;
      ctl[0] = *((volatile int*)&st->done);
      ctl[1] = kk;
      ctl[2] = ((kk % d.K) == 0) || (kk >= d.max_iters);
      if (!ctl[0] && !dbg_tile9(st, tl.row0 - 1, tl.row0 + tl.nrows + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1, d.n,
                                d.pitch))
        ctl[0] = 1;
    }
    __syncthreads();
    const int skip = ctl[0], kk = ctl[1], measure = ctl[2];
    __syncthreads();
    if (skip) continue;
    const int q0 = tl.col0 + lane * kVec;
    const int rpw = (tl.nrows + kWarpsY - 1) / kWarpsY;
    const int a0 = tl.row0 + wy * rpw;
    const int a1 = min(min(a0 + rpw, tl.row0 + tl.nrows), alim + 1);
    unsigned long long dm = 0;
    // the source term is a compile-time choice (as a runtime test its
    // addition is issued speculatively)
    const bool has_g = d.g[C] != nullptr;
    if (measure)
      dm = has_g ? sweep9_rows<T, C, true, true>(d, q0, a0, a1, lane) : sweep9_rows<T, C, true, false>(d, q0, a0, a1, lane);
    else if (has_g)
      (void)sweep9_rows<T, C, false, true>(d, q0, a0, a1, lane);
    else
      (void)sweep9_rows<T, C, false, false>(d, q0, a0, a1, lane);
    if (CORRECT && kk == d.max_iters) correct9_rows<C>(d, (const float*)d.x[C], q0, a0, a1);
    if (measure) block_max_to(dm, &st->dmax_bits, red);
    if (C == 3) {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        if (prev == (unsigned)d.tiles - 1u) {
          __threadfence();
          finalize9(d, st, kk, measure);
          if (CORRECT && kk == d.max_iters) d.outer->outer += 1;
        }
      }
      __syncthreads();
    }
  }
}

template <typename T, bool FAST, int C, bool HAS_G>
__device__ __forceinline__ unsigned long long rows9(const Desc9& d, bool measure, int q0, int a0, int a1, int lane) {
  if (FAST) {
    return measure ? sweep9_fast_rows<C, true, HAS_G>(d, q0, a0, a1, lane)
                   : sweep9_fast_rows<C, false, HAS_G>(d, q0, a0, a1, lane);
  }
  return measure ? sweep9_rows<T, C, true, HAS_G>(d, q0, a0, a1, lane)
                 : sweep9_rows<T, C, false, HAS_G>(d, q0, a0, a1, lane);
}

// A chunk of 4L colour phases in one launch, scheduled as a data flow (the
// cube kernels' schedule): work items (phase p, strip t) are claimed in the
// order p * strips + t; item (p, t) waits until strip t and the eight strips
// around it (row bands above and below, column tiles left and right, and the
// four corners, which the diagonal couplings reach) -- the only ones whose
// cells its stencil reads (in the three other quarters) or whose readers it
// could overwrite -- have finished phase p-1 (progress[t]
// counts the phases a strip has finished, so phases p-2 and p-3 are done
// too).  Every dependency has a smaller number than the item waiting for it,
// so the smallest unfinished item can always run.  Waits are bounded (an
// error in the slot state, then return); the last strip of the last phase
// closes the chunk, which ends at a tested iteration.
template <typename T, bool FAST, bool HAS_G>
__global__ void __launch_bounds__(kThreads) k_9_flow(const Desc9* __restrict__ dp, SlotState* st,
                                                     const Tile* __restrict__ strips, int nstrips, int ct,
                                                     int nphases, unsigned* progress) {
  const int lane = threadIdx.x & 31;
  const Desc9& d = *dp;
  int skip = 0, k0 = 0;
  if (lane == 0) {
    skip = *((volatile int*)&st->done);
    k0 = *((volatile int*)&st->iters);
  }
  skip = __shfl_sync(0xffffffffu, skip, 0);
  if (skip) return;  // done changes inside a launch only after its last item
  k0 = __shfl_sync(0xffffffffu, k0, 0);
  const long long items = (long long)nphases * nstrips;
  unsigned* claim = progress + nstrips;
  const int bands = nstrips / ct;
  const int last_it = k0 + (nphases >> 2);
  for (;;) {
    long long g = 0;
    if (lane == 0) g = (long long)atomicAdd(claim, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= items) break;
    const int p = (int)(g / nstrips), t = (int)(g - (long long)p * nstrips);
    const int C = p & 3;
    const int kk = k0 + (p >> 2) + 1;
    const bool measure = ((kk % d.K) == 0) || (kk >= d.max_iters);
    if (measure && kk != last_it) {  // the host plan must end launches at tested iterations
      if (lane == 0) {
        st->error = 1;
        st->done = 1;
      }
      return;
    }
    if (p > 0) {
      int nb[9];
      flow9_neighbours(t, bands, ct, nb);
      if (!flow_wait<9>(progress, nb, (unsigned)p, lane)) {
        if (lane == 0) {
          st->error = 1;
          st->done = 1;
        }
        return;
      }
    }
    const Tile tl = strips[t];
    if (!dbg_tile9(st, tl.row0 - 1, tl.row0 + tl.nrows + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1, d.n, d.pitch))
      return;
    const int q0 = tl.col0 + lane * kVec;
    const int a0 = tl.row0;
    const int a1 = min(tl.row0 + tl.nrows, ((d.n + (C >> 1)) >> 1) + 1);
    unsigned long long dm;
    switch (C) {
      case 0: dm = rows9<T, FAST, 0, HAS_G>(d, measure, q0, a0, a1, lane); break;
      case 1: dm = rows9<T, FAST, 1, HAS_G>(d, measure, q0, a0, a1, lane); break;
      case 2: dm = rows9<T, FAST, 2, HAS_G>(d, measure, q0, a0, a1, lane); break;
      default: dm = rows9<T, FAST, 3, HAS_G>(d, measure, q0, a0, a1, lane); break;
    }
    if (measure) {
      dm = warp_max64(dm);
      if (lane == 0 && dm) atomicMax(&st->dmax_bits, dm);
    }
    __threadfence();  // this lane's cells are visible before the strip's progress is
    __syncwarp();
    if (lane == 0) {
      flow_st_release(progress + t, (unsigned)(p + 1));
      if (p == nphases - 1) {
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        if (prev == (unsigned)nstrips - 1u) {
          __threadfence();
          finalize9(d, st, last_it, measure);
        }
      }
    }
    __syncwarp();
  }
}

// Residual rows of quarter C: max |(g + (4 s4 + sd)) - 20 u| in FP64; WRITE
// (the defect correction): r~ rounded to FP32 into rhs32[C].
template <typename T, int C, bool WRITE>
__device__ __forceinline__ unsigned long long resid9_rows(const Desc9& d, int q0, int a0, int a1, int lane) {
  constexpr int PI = C >> 1, PJ = C & 1;
  unsigned long long rm = 0;
  const T* X = (const T*)d.x[C];
  const T* Q1 = (const T*)d.x[C ^ 1];
  const T* Q2 = (const T*)d.x[C ^ 2];
  const T* Q3 = (const T*)d.x[C ^ 3];
  const double* G = d.g64[C];
  const int pitch = d.pitch;
  const int blim = (d.n + PJ) >> 1;
  a1 = min(a1, ((d.n + PI) >> 1) + 1);
  for (int r = a0; r < a1; ++r) {
    T n2[4], s2[4], n3[4], s3[4], w1[4], own[4];
    load4(Q2 + e9(r - PI, q0, pitch), n2);
    load4(Q2 + e9(r + 1 - PI, q0, pitch), s2);
    load4(Q3 + e9(r - PI, q0, pitch), n3);
    load4(Q3 + e9(r + 1 - PI, q0, pitch), s3);
    load4(Q1 + e9(r, q0, pitch), w1);
    load4(X + e9(r, q0, pitch), own);
    double gv[4] = {0.0, 0.0, 0.0, 0.0};
    if (G) load4(G + e9(r, q0, pitch), gv);
    T W[4], E[4], NW[4], NE[4], SW[4], SE[4];
    we_of<T, PJ>(w1, Q1 + (size_t)r * pitch, q0, lane, W, E);
    we_of<T, PJ>(n3, Q3 + (size_t)(r - PI) * pitch, q0, lane, NW, NE);
    we_of<T, PJ>(s3, Q3 + (size_t)(r + 1 - PI) * pitch, q0, lane, SW, SE);
    float r32[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double s4 =
          __dadd_rn(__dadd_rn((double)n2[v], (double)s2[v]), __dadd_rn((double)W[v], (double)E[v]));
      const double sd =
          __dadd_rn(__dadd_rn((double)NW[v], (double)NE[v]), __dadd_rn((double)SW[v], (double)SE[v]));
      const double res = __dadd_rn(__dadd_rn(gv[v], __dadd_rn(__dmul_rn(4.0, s4), sd)),
                                   -__dmul_rn(20.0, (double)own[v]));
      const bool in = (q0 + v) <= blim;
      if (in) rm = umax64(rm, abs_bits(res));
      r32[v] = in ? narrow_f64(res) : 0.0f;  // round to nearest even, on the integer units
    }
    if (WRITE) store4(d.rhs32[C] + e9(r, q0, pitch), r32);
  }
  return rm;
}

// ROLE kResidCheck: the residual stop on iterations that are multiples of K;
// kResidRefine: the defect correction's test after every correction, with r~
// rounded to FP32 into rhs32; kResidFinal: only rho is recorded.
template <typename T, int ROLE>
__global__ void __launch_bounds__(kThreads) k_resid9(const Desc9* __restrict__ dp, SlotState* st,
                                                     const Tile* __restrict__ tiles, int ntiles) {
  __shared__ unsigned long long red[kWarpsY];
  __shared__ int ctl[2];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const Desc9& d = *dp;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    if (threadIdx.x == 0) {
      const int it = *((volatile int*)&st->iters);
      int skip = 0;
      if (ROLE == kResidCheck)
        skip = *((volatile int*)&st->converged) || it == 0 || (it % d.K) != 0 ||
               it == *((volatile int*)&st->checked_iter);
      if (!skip && !dbg_tile9(st, tl.row0 - 1, tl.row0 + tl.nrows + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1, d.n,
                             d.pitch))
        skip = 1;
      ctl[0] = skip;
      ctl[1] = it;
    }
    __syncthreads();
    const int skip = ctl[0], it = ctl[1];
    __syncthreads();
    if (skip) continue;
    const int q0 = tl.col0 + lane * kVec;
    const int rpw = (tl.nrows + kWarpsY - 1) / kWarpsY;
    const int a0 = tl.row0 + wy * rpw;
    const int a1 = min(a0 + rpw, tl.row0 + tl.nrows);
    constexpr bool W = ROLE == kResidRefine;
    unsigned long long rm = resid9_rows<T, 0, W>(d, q0, a0, a1, lane);
    rm = umax64(rm, resid9_rows<T, 1, W>(d, q0, a0, a1, lane));
    rm = umax64(rm, resid9_rows<T, 2, W>(d, q0, a0, a1, lane));
    rm = umax64(rm, resid9_rows<T, 3, W>(d, q0, a0, a1, lane));
    block_max_to(rm, &st->rmax_bits, red);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(&st->arrive_res, 1u);
      if (prev == (unsigned)d.tiles - 1u) {
        __threadfence();
        st->arrive_res = 0;
        const double rmax = bits_to_double(atomicExch(&st->rmax_bits, 0ull));
        const double bmax = bits_to_double(*((volatile unsigned long long*)&st->bmax_bits));
        const double rho = bmax > 0.0 ? __ddiv_rn(rmax, bmax) : rmax;
        st->last_rho = rho;
        if (ROLE == kResidCheck) {
          st->checked_iter = it;
          if (rho < d.tol) {
            st->done = 1;
            st->converged = 1;
          } else if (rho < st->best_rho) {
            st->best_rho = rho;
            st->stall_run = 0;
          } else if (rho < 4.0 * st->best_rho) {  // a plateau near the smallest residual so far
            st->stall_run += 1;
            if (d.stall > 0 && st->stall_run >= d.stall) st->done = 1;  // the floor: tol is out of reach
          } else {
            st->stall_run = 0;  // far above it: still the early growth, not a plateau
          }
        }
        if (ROLE == kResidRefine) {
          if (rho < d.tol) {
            st->done = 1;
            st->converged = 1;
            d.inner->done = 1;  // the inner sweeps of this step are skipped
          } else if (rho < st->best_rho) {
            st->best_rho = rho;
            st->stall_run = 0;
          } else if (rho < 4.0 * st->best_rho) {  // the stall rule, as in the plain solve
            st->stall_run += 1;
            if (d.stall > 0 && st->stall_run >= d.stall) {
              st->done = 1;
              d.inner->done = 1;
            }
          } else {
            st->stall_run = 0;
          }
        }
      }
    }
    __syncthreads();
  }
}

#define SOR9_CK(ctx, expr)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      std::ostringstream os_;                                                                 \
      os_ << #expr << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
      (ctx)->set_error(os_.str());                                                            \
      return SOR_ERR_CUDA;                                                                    \
    }                                                                                         \
  } while (0)

constexpr int kMax9N = 32768;

struct Buffers9 {
  Ctx* c = nullptr;
  std::vector<void*> ptrs;
  size_t reserved = 0;
  void* get(size_t bytes) {
    void* p = ctx_dev_alloc(c, bytes);
    if (p) ptrs.push_back(p);
    return p;
  }
  ~Buffers9() {
    for (void* p : ptrs) ctx_dev_free(c, p);
    if (reserved) ctx_release(c, reserved);
  }
};

template <typename T, bool CORRECT = false>
void launch_sweep9(int colour, int grid, cudaStream_t s, const Desc9* d, SlotState* st, const Tile* t, int nt) {
  switch (colour) {
    case 0: k_sweep9<T, 0, CORRECT><<<grid, kThreads, 0, s>>>(d, st, t, nt); break;
    case 1: k_sweep9<T, 1, CORRECT><<<grid, kThreads, 0, s>>>(d, st, t, nt); break;
    case 2: k_sweep9<T, 2, CORRECT><<<grid, kThreads, 0, s>>>(d, st, t, nt); break;
    default: k_sweep9<T, 3, CORRECT><<<grid, kThreads, 0, s>>>(d, st, t, nt); break;
  }
}

template <typename T, bool FAST>
int flow9_blocks_per_sm(bool has_g) {
  int nb = 0;
  cudaError_t e = has_g ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_9_flow<T, FAST, true>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_9_flow<T, FAST, false>, kThreads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <typename T, bool FAST>
cudaError_t launch_9_flow(const Desc9* d, SlotState* st, const Tile* strips, int nstrips, int ct, int grid,
                          int nphases, unsigned* progress, bool has_g, cudaStream_t s) {
  if (has_g)
    k_9_flow<T, FAST, true><<<grid, kThreads, 0, s>>>(d, st, strips, nstrips, ct, nphases, progress);
  else
    k_9_flow<T, FAST, false><<<grid, kThreads, 0, s>>>(d, st, strips, nstrips, ct, nphases, progress);
  return cudaGetLastError();
}

template <typename T>
sor_status run9(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out, sor_result* res) {
  const double t0 = now_s();
  const int n = p->n, m = n + 2;
  const Layout L = Layout::make(n);
  const int pitch = L.pitch;
  const int qrows = ((n + 1) >> 1) + 2;  // quarter rows 0 .. (n+2)/2
  const size_t qelems = (size_t)qrows * pitch;
  const size_t nnat = (size_t)m * m, nf = (size_t)n * n;
  const bool has_f = f != nullptr;
  const bool in_dev = is_device_ptr(u0), f_dev = has_f && is_device_ptr(f), out_dev = is_device_ptr(u_out);
  const double w = p->omega <= 0.0 ? sor_omega_opt(n) : p->omega;
  const int stop = p->stop == SOR_STOP_MAXDELTA ? kStopDelta : kStopResid;

  // tiles over quarter rows 1 .. (n+1)/2 and columns 1 .. (n+1)/2 (each
  // phase masks the cells beyond its own quarter's interior)
  std::vector<Tile> tiles;
  const int arows = (n + 1) >> 1;
  for (int r = 1; r <= arows; r += kTileRows)
    for (int t = 0; t < L.col_tiles(); ++t)
      tiles.push_back(Tile{0, r, 1 + t * kWarpCols, std::min(kTileRows, arows - r + 1)});
  const int nt = (int)tiles.size();
  // FP64 default: the shared-triple phases (within 1e-12 of the exact
  // order); SOR_FLAG_EXACT_ORDER or FP32: the exact-order phases
  // FP64 phases run a launch per run of iterations up to the next test
  // (data-flow schedule); the short FP32 phases a launch per phase
  const bool fast = sizeof(T) == 8 && !(p->flags & SOR_FLAG_EXACT_ORDER);
  const bool flow = sizeof(T) == 8;
  const int bps = !flow ? 1 : fast ? flow9_blocks_per_sm<double, true>(has_f) : flow9_blocks_per_sm<T, false>(has_f);
  if (bps < 1) {
    c->set_error("9-point phase kernel does not fit on an SM");
    return SOR_ERR_CUDA;
  }
  std::vector<Tile> strips;
  const int ct = L.col_tiles();
  if (flow) build_strips9(n, ct, c->sm_count * bps * kWarpsY, &strips);
  const int nst = (int)strips.size();
  const int flow_grid = c->sm_count * bps;

  size_t bytes = 4 * qelems * sizeof(T) + sizeof(Desc9) + sizeof(SlotState) + sizeof(Tile) * nt + 1024 +
                 sizeof(Tile) * nst + sizeof(unsigned) * (nst + 1);
  if (has_f) bytes += 4 * qelems * sizeof(T) + (sizeof(T) == 4 ? 4 * qelems * sizeof(double) : 0);
  const bool stage_u = !in_dev || !out_dev;
  if (stage_u) bytes += nnat * sizeof(double);
  if (has_f && !f_dev) bytes += nf * sizeof(double);
  Buffers9 B;
  B.c = c;
  sor_status rs = ctx_reserve(c, bytes, false, 0.0);
  if (rs != SOR_OK) {
    c->set_error("9-point solve does not fit the device-memory budget");
    return rs;
  }
  B.reserved = bytes;
  T* x[4];
  T* g[4] = {nullptr, nullptr, nullptr, nullptr};
  double* g64[4] = {nullptr, nullptr, nullptr, nullptr};
  bool ok = true;
  for (int q = 0; q < 4; ++q) {
    x[q] = (T*)B.get(qelems * sizeof(T));
    ok = ok && x[q];
    if (has_f) {
      g[q] = (T*)B.get(qelems * sizeof(T));
      g64[q] = sizeof(T) == 4 ? (double*)B.get(qelems * sizeof(double)) : (double*)g[q];
      ok = ok && g[q] && g64[q];
    }
  }
  Desc9* d_desc = (Desc9*)B.get(sizeof(Desc9));
  SlotState* d_state = (SlotState*)B.get(sizeof(SlotState));
  Tile* d_tiles = (Tile*)B.get(sizeof(Tile) * nt);
  Tile* d_strips = (Tile*)B.get(sizeof(Tile) * std::max(1, nst));
  unsigned* d_progress = (unsigned*)B.get(sizeof(unsigned) * (nst + 1));
  double* d_u = stage_u ? (double*)B.get(nnat * sizeof(double)) : nullptr;
  double* d_f = (has_f && !f_dev) ? (double*)B.get(nf * sizeof(double)) : nullptr;
  if (!ok || !d_desc || !d_state || !d_tiles || !d_strips || !d_progress || (stage_u && !d_u) ||
      (has_f && !f_dev && !d_f)) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  cudaStream_t s = c->stream;

  Desc9 d;
  std::memset(&d, 0, sizeof(d));
  for (int q = 0; q < 4; ++q) {
    d.x[q] = x[q];
    d.g[q] = g[q];
    d.g64[q] = g64[q];
  }
  d.n = n;
  d.pitch = pitch;
  d.K = p->check_every;
  d.max_iters = p->max_iters;
  d.stop = stop;
  d.tiles = nt;
  d.a64 = 1.0 - w;
  d.b64 = w / 20.0;
  d.a32 = (float)(1.0 - w);
  d.b32 = (float)(w / 20.0);
  d.tol = p->tol;
  d.stall = p->stall_window;
  SlotState st;
  std::memset(&st, 0, sizeof(st));
  st.checked_iter = -1;
  st.last_dmax = -1.0;
  st.last_rho = -1.0;
  st.best_rho = HUGE_VAL;
  st.done = p->max_iters == 0;

  for (int q = 0; q < 4; ++q) {
    SOR9_CK(c, cudaMemsetAsync(x[q], 0, qelems * sizeof(T), s));
    if (has_f) SOR9_CK(c, cudaMemsetAsync(g[q], 0, qelems * sizeof(T), s));
    if (has_f && sizeof(T) == 4) SOR9_CK(c, cudaMemsetAsync(g64[q], 0, qelems * sizeof(double), s));
  }
  SOR9_CK(c, cudaMemcpyAsync(d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, s));
  SOR9_CK(c, cudaMemcpyAsync(d_state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  SOR9_CK(c, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, s));
  if (nst > 0) SOR9_CK(c, cudaMemcpyAsync(d_strips, strips.data(), sizeof(Tile) * nst, cudaMemcpyHostToDevice, s));
  const double* u_src = u0;
  if (!in_dev) {
    SOR9_CK(c, cudaMemcpyAsync(d_u, u0, nnat * sizeof(double), cudaMemcpyHostToDevice, s));
    u_src = d_u;
  }
  const double* f_src = f;
  if (has_f && !f_dev) {
    SOR9_CK(c, cudaMemcpyAsync(d_f, f, nf * sizeof(double), cudaMemcpyHostToDevice, s));
    f_src = d_f;
  }
  const double h = 1.0 / (double)(n + 1);
  const dim3 pgrid((m + kWarpCols - 1) / kWarpCols, m);
  const bool f32 = sizeof(T) == 4;
  k_pack9<T><<<pgrid, kWarpCols, 0, s>>>(u_src, f_src, n, pitch, 6.0 * (h * h), x[0], x[1], x[2], x[3], g[0], g[1],
                                         g[2], g[3], f32 ? g64[0] : nullptr, f32 ? g64[1] : nullptr,
                                         f32 ? g64[2] : nullptr, f32 ? g64[3] : nullptr, d_state);
  SOR9_CK(c, cudaGetLastError());

  const int grid = std::min(nt, c->sm_count * 8);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SOR9_CK(c, cudaEventCreate(&ev0));
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
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    ~Cleanup() {
      for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaFreeHost(hs);
    }
  } cl{ev0, ev1, h_state, {}};

  // a batch of Lc iterations after iteration `first`: one flow launch per
  // run of iterations up to the next tested one (a multiple of K or the cap),
  // the residual test after those at multiples of K
  auto enqueue = [&](int first, int Lc) -> sor_status {
    if (!flow) {
      for (int it = 1; it <= Lc; ++it) {
        for (int col = 0; col < 4; ++col) launch_sweep9<T>(col, grid, s, d_desc, d_state, d_tiles, nt);
        if (stop == kStopResid && (first + it) % d.K == 0)
          k_resid9<T, kResidCheck><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
      }
      SOR9_CK(c, cudaGetLastError());
      return SOR_OK;
    }
    int done_it = 0;
    while (done_it < Lc) {
      const long long at = first + done_it;
      const long long next_m = std::min<long long>((at / d.K + 1) * d.K, p->max_iters);
      // the claim counter numbers 4 L x strips items in 32 bits: L stays below 2^28 / strips
      const int Ls = (int)std::min<long long>({next_m - at, (long long)(Lc - done_it),
                                               std::max(1LL, (1LL << 28) / std::max(1, nst))});
      SOR9_CK(c, cudaMemsetAsync(d_progress, 0, sizeof(unsigned) * (nst + 1), s));
      if (fast)
        SOR9_CK(c, (launch_9_flow<double, true>(d_desc, d_state, d_strips, nst, ct, flow_grid, 4 * Ls, d_progress,
                                                has_f, s)));
      else
        SOR9_CK(c, (launch_9_flow<T, false>(d_desc, d_state, d_strips, nst, ct, flow_grid, 4 * Ls, d_progress,
                                           has_f, s)));
      done_it += Ls;
      if (stop == kStopResid && (first + done_it) % d.K == 0)
        k_resid9<T, kResidCheck><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
    }
    SOR9_CK(c, cudaGetLastError());
    return SOR_OK;
  };
  // iterations per host check: a whole number of test intervals when K fits,
  // so every batch starts at a tested iteration and one graph serves them all
  const int chunk0 = c->opt_chunk.load() > 0 ? c->opt_chunk.load() : 64;
  const int chunk = d.K <= chunk0 ? (chunk0 / d.K) * d.K : chunk0;
  const bool use_graphs = c->opt_graphs.load() != 0;
  SOR9_CK(c, cudaEventRecord(ev0, s));
  long long planned = 0;
  bool finished = st.done != 0;
  while (!finished && planned < p->max_iters) {
    int Lc = (int)std::min<long long>(chunk, p->max_iters - planned);
    if (d.K > chunk0)  // batches end at tested iterations: few distinct launch plans
      Lc = (int)std::min<long long>(Lc, std::min<long long>((planned / d.K + 1) * d.K, p->max_iters) - planned);
    if (use_graphs) {
      // the launch ends and the residual tests depend on where the tested
      // iterations fall in the batch
      const std::pair<int, int> key(Lc, (int)(planned % d.K));
      auto itg = cl.graphs.find(key);
      if (itg == cl.graphs.end()) {
        cudaGraph_t gr = nullptr;
        SOR9_CK(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const sor_status es = enqueue((int)planned, Lc);
        const cudaError_t ce = cudaStreamEndCapture(s, &gr);
        if (es != SOR_OK) {
          if (gr) cudaGraphDestroy(gr);
          return es;
        }
        SOR9_CK(c, ce);
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        SOR9_CK(c, ie);
        itg = cl.graphs.emplace(key, ex).first;
      }
      SOR9_CK(c, cudaGraphLaunch(itg->second, s));
    } else {
      const sor_status es = enqueue((int)planned, Lc);
      if (es != SOR_OK) return es;
    }
    planned += Lc;
    SOR9_CK(c, cudaMemcpyAsync(h_state, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR9_CK(c, cudaStreamSynchronize(s));
    finished = h_state->done != 0;
  }
  SOR9_CK(c, cudaEventRecord(ev1, s));
  k_resid9<T, kResidFinal><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
  SOR9_CK(c, cudaGetLastError());
  double* out_dst = out_dev ? u_out : d_u;
  k_unpack9<T><<<pgrid, kWarpCols, 0, s>>>(x[0], x[1], x[2], x[3], n, pitch, out_dst);
  SOR9_CK(c, cudaGetLastError());
  if (!out_dev) SOR9_CK(c, cudaMemcpyAsync(u_out, d_u, nnat * sizeof(double), cudaMemcpyDeviceToHost, s));
  SOR9_CK(c, cudaMemcpyAsync(h_state, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
  SOR9_CK(c, cudaStreamSynchronize(s));
  float ms = 0.0f;
  SOR9_CK(c, cudaEventElapsedTime(&ms, ev0, ev1));
  if (h_state->error) {
    c->set_error("device-side consistency check failed");
    return SOR_ERR_INTERNAL;
  }
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->iterations = h_state->iters;
    res->converged = h_state->converged;
    res->final_maxdelta = h_state->last_dmax;
    res->final_resid_rel = h_state->last_rho;
    res->latency_s = now_s() - t0;
    res->device_s = ms * 1e-3;
  }
  return SOR_OK;
}

// Defect correction with the four-colour sweeps (SOR_FP32_REFINE): per outer
// step the FP64 residual test, which also rounds r~ to FP32 as the right
// side; inner_sweeps FP32 four-colour iterations on A d = r~ from d = 0 (a
// launch per phase), whose last phase of each colour also adds d to u in
// FP64.  One step is a graph replayed up to max_iters / inner times; once the
// test passes, the device skips the queued sweeps and the host stops at its
// next poll.
sor_status run9_refine(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                       sor_result* res) {
  const double t0 = now_s();
  const int n = p->n, m = n + 2;
  const Layout L = Layout::make(n);
  const int pitch = L.pitch;
  const int qrows = ((n + 1) >> 1) + 2;
  const size_t qelems = (size_t)qrows * pitch;
  const size_t nnat = (size_t)m * m, nf = (size_t)n * n;
  const bool has_f = f != nullptr;
  const bool in_dev = is_device_ptr(u0), f_dev = has_f && is_device_ptr(f), out_dev = is_device_ptr(u_out);
  const double w = p->omega <= 0.0 ? sor_omega_opt(n) : p->omega;
  const int inner = p->inner_sweeps > 0 ? p->inner_sweeps : 20;
  const int max_outer = p->max_iters / inner;

  std::vector<Tile> tiles;
  const int arows = (n + 1) >> 1;
  for (int r = 1; r <= arows; r += kTileRows)
    for (int t = 0; t < L.col_tiles(); ++t)
      tiles.push_back(Tile{0, r, 1 + t * kWarpCols, std::min(kTileRows, arows - r + 1)});
  const int nt = (int)tiles.size();

  const bool stage_u = !in_dev || !out_dev;
  size_t bytes = 4 * qelems * (sizeof(double) + 2 * sizeof(float)) + 2 * sizeof(Desc9) + 3 * sizeof(SlotState) +
                 sizeof(Tile) * nt + 1024;
  if (has_f) bytes += 4 * qelems * sizeof(double);
  if (stage_u) bytes += nnat * sizeof(double);
  if (has_f && !f_dev) bytes += nf * sizeof(double);
  Buffers9 B;
  B.c = c;
  sor_status rs = ctx_reserve(c, bytes, false, 0.0);
  if (rs != SOR_OK) {
    c->set_error("9-point solve does not fit the device-memory budget");
    return rs;
  }
  B.reserved = bytes;
  double* u64 = (double*)B.get(4 * qelems * sizeof(double));
  float* dbuf = (float*)B.get(4 * qelems * sizeof(float));  // the correction, four quarters
  float* rbuf = (float*)B.get(4 * qelems * sizeof(float));  // the rounded residual, four quarters
  double* g64 = has_f ? (double*)B.get(4 * qelems * sizeof(double)) : nullptr;
  Desc9* d_desc = (Desc9*)B.get(2 * sizeof(Desc9));                // [0] u, [1] d
  SlotState* d_state = (SlotState*)B.get(3 * sizeof(SlotState));  // [0] outer, [1] inner, [2] inner at rest
  Tile* d_tiles = (Tile*)B.get(sizeof(Tile) * nt);
  double* d_u = stage_u ? (double*)B.get(nnat * sizeof(double)) : nullptr;
  double* d_f = (has_f && !f_dev) ? (double*)B.get(nf * sizeof(double)) : nullptr;
  if (!u64 || !dbuf || !rbuf || (has_f && !g64) || !d_desc || !d_state || !d_tiles || (stage_u && !d_u) ||
      (has_f && !f_dev && !d_f)) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  cudaStream_t s = c->stream;

  Desc9 du, dd;
  std::memset(&du, 0, sizeof(du));
  std::memset(&dd, 0, sizeof(dd));
  for (int q = 0; q < 4; ++q) {
    du.x[q] = u64 + q * qelems;
    du.g[q] = has_f ? g64 + q * qelems : nullptr;
    du.g64[q] = has_f ? g64 + q * qelems : nullptr;
    du.rhs32[q] = rbuf + q * qelems;
    dd.x[q] = dbuf + q * qelems;
    dd.g[q] = rbuf + q * qelems;
    dd.ucorr[q] = u64 + q * qelems;
  }
  du.n = dd.n = n;
  du.pitch = dd.pitch = pitch;
  du.tiles = dd.tiles = nt;
  du.K = 1;
  du.max_iters = 1 << 30;
  du.stop = kStopResid;
  du.tol = p->tol;
  du.stall = p->stall_window;
  du.inner = d_state + 1;
  dd.K = inner;
  dd.max_iters = inner;  // one run of `inner` iterations; its change test never stops it
  dd.stop = kStopDelta;
  dd.tol = -1.0;
  dd.a32 = (float)(1.0 - w);
  dd.b32 = (float)(w / 20.0);
  dd.a64 = 1.0 - w;
  dd.b64 = w / 20.0;
  dd.outer = d_state;
  SlotState st[3];
  std::memset(st, 0, sizeof(st));
  for (auto& x : st) {
    x.checked_iter = -1;
    x.last_dmax = -1.0;
    x.last_rho = -1.0;
    x.best_rho = HUGE_VAL;
  }
  SOR9_CK(c, cudaMemsetAsync(u64, 0, 4 * qelems * sizeof(double), s));
  if (has_f) SOR9_CK(c, cudaMemsetAsync(g64, 0, 4 * qelems * sizeof(double), s));
  SOR9_CK(c, cudaMemsetAsync(dbuf, 0, 4 * qelems * sizeof(float), s));
  SOR9_CK(c, cudaMemsetAsync(rbuf, 0, 4 * qelems * sizeof(float), s));
  const Desc9 descs[2] = {du, dd};
  SOR9_CK(c, cudaMemcpyAsync(d_desc, descs, sizeof(descs), cudaMemcpyHostToDevice, s));
  SOR9_CK(c, cudaMemcpyAsync(d_state, st, sizeof(st), cudaMemcpyHostToDevice, s));
  SOR9_CK(c, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, s));
  const double* u_src = u0;
  if (!in_dev) {
    SOR9_CK(c, cudaMemcpyAsync(d_u, u0, nnat * sizeof(double), cudaMemcpyHostToDevice, s));
    u_src = d_u;
  }
  const double* f_src = f;
  if (has_f && !f_dev) {
    SOR9_CK(c, cudaMemcpyAsync(d_f, f, nf * sizeof(double), cudaMemcpyHostToDevice, s));
    f_src = d_f;
  }
  const double h = 1.0 / (double)(n + 1);
  const dim3 pgrid((m + kWarpCols - 1) / kWarpCols, m);
  double* gq[4] = {nullptr, nullptr, nullptr, nullptr};
  if (has_f)
    for (int q = 0; q < 4; ++q) gq[q] = g64 + q * qelems;
  k_pack9<double><<<pgrid, kWarpCols, 0, s>>>(u_src, f_src, n, pitch, 6.0 * (h * h), u64, u64 + qelems,
                                              u64 + 2 * qelems, u64 + 3 * qelems, gq[0], gq[1], gq[2], gq[3],
                                              nullptr, nullptr, nullptr, nullptr, d_state);
  SOR9_CK(c, cudaGetLastError());

  const int grid = std::min(nt, c->sm_count * 8);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SOR9_CK(c, cudaEventCreate(&ev0));
  if (cudaEventCreate(&ev1) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(ev0);
    c->set_error("event creation failed");
    return SOR_ERR_CUDA;
  }
  SlotState* h_state = nullptr;  // [0], [1]: the outer state after alternate batches
  if (cudaMallocHost(&h_state, 2 * sizeof(SlotState)) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    c->set_error("pinned allocation failed");
    return SOR_ERR_OOM;
  }
  cudaEvent_t pev[2] = {nullptr, nullptr};
  struct Cleanup {
    cudaEvent_t a, b;
    SlotState* hs;
    cudaGraphExec_t g;
    cudaEvent_t* pe;
    ~Cleanup() {
      if (g) cudaGraphExecDestroy(g);
      for (int k = 0; k < 2; ++k)
        if (pe[k]) cudaEventDestroy(pe[k]);
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaFreeHost(hs);
    }
  } cl{ev0, ev1, h_state, nullptr, pev};
  for (int k = 0; k < 2; ++k) SOR9_CK(c, cudaEventCreateWithFlags(&pev[k], cudaEventDisableTiming));

  // one outer step: inner state back to rest, d = 0, the residual test (and
  // right side), the inner sweeps (the last phase of each colour corrects u)
  auto enqueue_step = [&]() -> sor_status {
    SOR9_CK(c, cudaMemcpyAsync(d_state + 1, d_state + 2, sizeof(SlotState), cudaMemcpyDeviceToDevice, s));
    SOR9_CK(c, cudaMemsetAsync(dbuf, 0, 4 * qelems * sizeof(float), s));
    k_resid9<double, kResidRefine><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
    for (int it = 0; it < inner; ++it)
      for (int col = 0; col < 4; ++col) launch_sweep9<float, true>(col, grid, s, d_desc + 1, d_state + 1, d_tiles, nt);
    SOR9_CK(c, cudaGetLastError());
    return SOR_OK;
  };
  const bool use_graphs = c->opt_graphs.load() != 0;
  if (use_graphs && max_outer > 0) {
    cudaGraph_t gr = nullptr;
    SOR9_CK(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const sor_status es = enqueue_step();
    const cudaError_t ce = cudaStreamEndCapture(s, &gr);
    if (es != SOR_OK) {
      if (gr) cudaGraphDestroy(gr);
      return es;
    }
    SOR9_CK(c, ce);
    const cudaError_t ie = cudaGraphInstantiate(&cl.g, gr, 0);
    cudaGraphDestroy(gr);
    SOR9_CK(c, ie);
  }
  SOR9_CK(c, cudaEventRecord(ev0, s));
  // batches of about a millisecond of steps; the host reads the state after
  // batch b while batch b+1 runs (steps queued past convergence only repeat
  // the residual test)
  const double step_s = (double)n * n * inner / 3.0e11 + 20e-6;
  const int per_poll = (int)std::max(1.0, std::min(32.0, std::floor(1e-3 / step_s)));
  int planned = 0, batch = 0;
  while (planned < max_outer) {
    const int kk = std::min(per_poll, max_outer - planned);
    for (int j = 0; j < kk; ++j) {
      if (use_graphs) {
        SOR9_CK(c, cudaGraphLaunch(cl.g, s));
      } else {
        const sor_status es = enqueue_step();
        if (es != SOR_OK) return es;
      }
    }
    planned += kk;
    SOR9_CK(c, cudaMemcpyAsync(h_state + (batch & 1), d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR9_CK(c, cudaEventRecord(pev[batch & 1], s));
    if (batch > 0) {
      SOR9_CK(c, cudaEventSynchronize(pev[(batch - 1) & 1]));
      const SlotState& prev = h_state[(batch - 1) & 1];
      if (prev.done || prev.error) break;  // converged, or stalled at the floor
    }
    ++batch;
  }
  // the test after the last correction (a no-op repeat once converged)
  k_resid9<double, kResidRefine><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
  SOR9_CK(c, cudaGetLastError());
  SOR9_CK(c, cudaEventRecord(ev1, s));
  double* out_dst = out_dev ? u_out : d_u;
  k_unpack9<double><<<pgrid, kWarpCols, 0, s>>>(u64, u64 + qelems, u64 + 2 * qelems, u64 + 3 * qelems, n, pitch,
                                                out_dst);
  SOR9_CK(c, cudaGetLastError());
  if (!out_dev) SOR9_CK(c, cudaMemcpyAsync(u_out, d_u, nnat * sizeof(double), cudaMemcpyDeviceToHost, s));
  SOR9_CK(c, cudaMemcpyAsync(h_state, d_state, 2 * sizeof(SlotState), cudaMemcpyDeviceToHost, s));
  SOR9_CK(c, cudaStreamSynchronize(s));
  const SlotState fin = h_state[0], fin_inner = h_state[1];
  float ms = 0.0f;
  SOR9_CK(c, cudaEventElapsedTime(&ms, ev0, ev1));
  if (fin.error || fin_inner.error) {
    c->set_error("device-side consistency check failed");
    return SOR_ERR_INTERNAL;
  }
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->iterations = fin.outer * inner;
    res->converged = fin.converged;
    res->outer_steps = fin.outer;
    res->final_maxdelta = -1.0;
    res->final_resid_rel = fin.last_rho;
    res->latency_s = now_s() - t0;
    res->device_s = ms * 1e-3;
  }
  return SOR_OK;
}

}  // namespace

sor_status solve9_blocking(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                           sor_result* res) {
  NvtxRange nvtx("sor_solve9");
  if (!p || !u0 || !u_out) {
    c->set_error("params, u0 and u_out must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  std::ostringstream why;
  if (p->n < 1 || p->n > kMax9N) why << "n must be in [1, " << kMax9N << "]";
  else if (p->precision != SOR_FP64 && p->precision != SOR_FP32 && p->precision != SOR_FP32_REFINE)
    why << "9-point solves run in FP64, FP32 or FP32_REFINE";
  else if (p->inner_sweeps < 0) why << "inner_sweeps must be >= 0";
  else if (p->stop != SOR_STOP_MAXDELTA && p->stop != SOR_STOP_RESID_REL) why << "unknown stop rule";
  else if (p->max_iters < 0 || p->check_every < 1) why << "max_iters >= 0 and check_every >= 1 required";
  else if (p->flags & ~SOR_FLAG_EXACT_ORDER) why << "unknown flags";
  else if (p->stall_window < 0) why << "stall_window must be >= 0";
  else if (std::isnan(p->tol) || std::isnan(p->omega)) why << "tol and omega must not be NaN";
  else if (p->omega > 0.0 && !(p->omega < 2.0)) why << "omega must be in (0, 2)";
  if (!why.str().empty()) {
    c->set_error(why.str());
    return SOR_ERR_INVALID_ARG;
  }
  if (p->precision == SOR_FP32_REFINE) return run9_refine(c, p, u0, f, u_out, res);
  return p->precision == SOR_FP64 ? run9<double>(c, p, u0, f, u_out, res) : run9<float>(c, p, u0, f, u_out, res);
}

}  // namespace sorgb
