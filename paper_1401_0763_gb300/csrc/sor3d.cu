// Red-black SOR on 3D grids (7-point stencil): the grids the paper names as
// the next step of its study (Section 5), solved by the same method --
// Algorithm 1 with the cell update of Eq. 1, the Gauss-Seidel value taken
// from the six face neighbours:
//   U <- (1-w) U + (w/6) ((((N + S) + (W + E)) + (D + U)) + g),  g = h^2 f,
// red = (i + j + k) even, red phase first, convergence test every K
// iterations on max|change| or on the scaled residual
//   r~ = (g + (((N + S) + (W + E)) + (D + U))) - 6 u.
// Every product and sum is rounded on its own in that order, so FP64 and FP32
// results equal the CPU oracle's bit for bit.
//
// Storage.  Plane k and row i of the (N+2)^3 cube form row r = k (N+2) + i of
// a colour array laid out like the 2D one: cell (k, i, j) has colour
// c = (i + j + k) & 1 and sits at packed column q = (j + 1) >> 1, element
// r * pitch + q + kOff.  With s = (i + k + c) & 1 the in-plane neighbours are
// those of the 2D layout (N = o[r-1][q], S = o[r+1][q], W = o[r][q-s],
// E = o[r][q-s+1]) and the neighbours below / above the plane are
// D = o[r - (N+2)][q], U = o[r + (N+2)][q] (same packed column: moving one
// plane flips the colour and keeps j).  Interior: 1 <= k, i <= N and
// 1 <= q <= (N + s) / 2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <sstream>
#include <utility>
#include <vector>

#include "sor_devfn.cuh"
#include "sor_strips.cuh"
#include "sor_bits.cuh"
#include "sor_runtime.h"

namespace sorgb {
namespace {

__device__ __forceinline__ size_t e3(int k, int i, int q, int m, int pitch) {
  return ((size_t)k * (size_t)m + (size_t)i) * (size_t)pitch + (size_t)(q + kOff);
}

// Debug check (SOR_DEBUG_BOUNDS) of a work item that touches planes [k0, k1),
// rows [i0, i1) and packed columns [q0, q1) of the colour arrays: on failure
// the state records kErrBounds and stops; release builds compile it to true.
__device__ __forceinline__ bool dbg_tile3(SlotState* st, int k0, int k1, int i0, int i1, int q0, int q1, int m,
                                          int pitch) {
  if (dbg_range(k0, k1, m, st) && dbg_range(i0, i1, m, st) &&
      dbg_range((long long)q0 + kOff, (long long)q1 + kOff, pitch, st))
    return true;
  st->done = 1;
  return false;
}

// Solve description in device memory (constant while the solve runs).
struct Desc3 {
  void* x[2];            // colour arrays (FP64 or FP32); with blocked FP32 sweeps, the current pair
  void* xalt[2];         // blocked FP32 sweeps: the other pair (written by each launch, then made current)
  const void* g[2];      // h^2 f in the sweep type, or null
  const double* g64[2];  // h^2 f in FP64 for the residual, or null
  int n, m, pitch, K, max_iters, stop, tiles;
  float a32, b32;        // (float)(1 - w), (float)(w / 6)
  double a64, b64;       // 1 - w, w / 6
  double tol;
  int stall;             // residual stop: stall window (0 = off), the 2D rule
  float* rhs32[2];       // defect correction, residual pass: r~ rounded to FP32, per colour (else null)
  SlotState* inner;      // defect correction, residual pass: the inner solve's state (skipped once converged)
  double* ucorr[2];      // defect correction, inner sweeps: u, corrected by the final d (else null)
  SlotState* outer;      // defect correction, inner sweeps: the outer state (counts corrections)
};

// Thread (k, i, q) moves the natural cells j = 2q-1 and j = 2q of row i of
// plane k into the colour arrays; interior cells also receive h^2 f and
// contribute |b~| = |h^2 f + (shell neighbours)| to ||b~||_inf.
template <typename T>
__global__ void k_pack3d(const double* __restrict__ u0, const double* __restrict__ f, int n, int pitch, double h2,
                         T* x0, T* x1, T* g0, T* g1, double* g64_0, double* g64_1, SlotState* st) {
  __shared__ unsigned long long red[kWarpsY];
  const int m = n + 2;
  const int qw = (n + 1) / 2 + 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, k = blockIdx.z;
  unsigned long long bb = 0, ub = 0, gb = 0;
  if (q < qw) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int j = 2 * q - 1 + t;
      if (j < 0 || j >= m) continue;
      const int c = (i + j + k) & 1;
      const size_t nat = ((size_t)k * m + i) * m + j;
      const size_t e = e3(k, i, q, m, pitch);
      (c ? x1 : x0)[e] = (T)u0[nat];
      ub = umax64(ub, abs_bits(u0[nat]));
      const bool interior = i >= 1 && i <= n && j >= 1 && j <= n && k >= 1 && k <= n;
      double gc = 0.0;
      if (interior && f) gc = __dmul_rn(h2, f[((size_t)(k - 1) * n + (i - 1)) * n + (j - 1)]);
      gb = umax64(gb, abs_bits(gc));
      T* gg = c ? g1 : g0;
      if (gg) gg[e] = (T)gc;
      double* g6 = c ? g64_1 : g64_0;
      if (g6) g6[e] = gc;
      if (interior) {
        // b~ = g + shell neighbours, summed in the order N, S, W, E, D, U
        double bnd = 0.0;
        if (i == 1) bnd = __dadd_rn(bnd, u0[nat - m]);
        if (i == n) bnd = __dadd_rn(bnd, u0[nat + m]);
        if (j == 1) bnd = __dadd_rn(bnd, u0[nat - 1]);
        if (j == n) bnd = __dadd_rn(bnd, u0[nat + 1]);
        if (k == 1) bnd = __dadd_rn(bnd, u0[nat - (size_t)m * m]);
        if (k == n) bnd = __dadd_rn(bnd, u0[nat + (size_t)m * m]);
        bb = umax64(bb, abs_bits(__dadd_rn(gc, bnd)));
      }
    }
  }
  block_max_to(bb, &st->bmax_bits, red);
  block_max_to(ub, &st->umax_bits, red);  // magnitudes that bound the rescaled phases' chunk length
  block_max_to(gb, &st->gmax_bits, red);
}

template <typename T>
__global__ void k_unpack3d(const T* __restrict__ x0, const T* __restrict__ x1, int n, int pitch, double* u) {
  const int m = n + 2;
  const int qw = (n + 1) / 2 + 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, k = blockIdx.z;
  if (q >= qw) return;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int j = 2 * q - 1 + t;
    if (j < 0 || j >= m) continue;
    const int c = (i + j + k) & 1;
    u[((size_t)k * m + i) * m + j] = (double)(c ? x1 : x0)[e3(k, i, q, m, pitch)];
  }
}

// Rows [i0, i1) of plane k for one warp, one colour phase, exact order.  The
// loads of row i+1 are issued before row i is computed (register double
// buffering), so a warp waits for memory once per strip instead of once per
// row; the arithmetic and its order do not change.
template <typename T>
struct Row3 {
  T op[4], own[4], dn[4], up[4], gv[4];
  T left, right;  // the in-row neighbours beyond the warp's columns (lanes 0 / 31)
};
template <typename T, bool HAS_G>
__device__ __forceinline__ void row3_load(Row3<T>& r, const T* __restrict__ X, const T* __restrict__ O,
                                          const T* __restrict__ G, int k, int i, int m, int pitch, int q0, int lane) {
  load4(O + e3(k, i + 1, q0, m, pitch), r.op);
  load4(X + e3(k, i, q0, m, pitch), r.own);
  load4(O + e3(k - 1, i, q0, m, pitch), r.dn);
  load4(O + e3(k + 1, i, q0, m, pitch), r.up);
  if (HAS_G) load4(G + e3(k, i, q0, m, pitch), r.gv);
  r.left = lane == 0 ? O[e3(k, i, q0 - 1, m, pitch)] : T(0);
  r.right = lane == 31 ? O[e3(k, i, q0 + kVec, m, pitch)] : T(0);
}

template <typename T, bool MEASURE, bool HAS_G>
__device__ __forceinline__ unsigned long long sweep3_rows(T* __restrict__ X, const T* __restrict__ O,
                                                          const T* __restrict__ G, T a, T b, int pitch, int m, int n,
                                                          int colour, int k, int q0, int i0, int i1, int lane) {
  unsigned long long dm = 0;
  unsigned dm32 = 0;
  if (i0 >= i1) return 0;
  T om[4], oc[4];
  load4(O + e3(k, i0 - 1, q0, m, pitch), om);
  load4(O + e3(k, i0, q0, m, pitch), oc);
  Row3<T> cur;
  row3_load<T, HAS_G>(cur, X, O, G, k, i0, m, pitch, q0, lane);
  for (int i = i0; i < i1; ++i) {
    Row3<T> nxt;
    row3_load<T, HAS_G>(nxt, X, O, G, k, min(i + 1, i1 - 1), m, pitch, q0, lane);  // the last row reloads itself
    T left = __shfl_up_sync(0xffffffffu, oc[3], 1);
    T right = __shfl_down_sync(0xffffffffu, oc[0], 1);
    if (lane == 0) left = cur.left;
    if (lane == 31) right = cur.right;
    const int s = (i + k + colour) & 1;
    const int qlim = (n + s) >> 1;
    T W[4], E[4];
    if (s == 0) {
      W[0] = oc[0]; W[1] = oc[1]; W[2] = oc[2]; W[3] = oc[3];
      E[0] = oc[1]; E[1] = oc[2]; E[2] = oc[3]; E[3] = right;
    } else {
      W[0] = left; W[1] = oc[0]; W[2] = oc[1]; W[3] = oc[2];
      E[0] = oc[0]; E[1] = oc[1]; E[2] = oc[2]; E[3] = oc[3];
    }
    T nv[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T sum = radd(radd(radd(om[v], cur.op[v]), radd(W[v], E[v])), radd(cur.dn[v], cur.up[v]));
      if (HAS_G) sum = radd(sum, cur.gv[v]);
      const T nu = radd(rmul(a, cur.own[v]), rmul(b, sum));
      const bool in = (q0 + v) <= qlim;
      // cells past the interior keep their value (the whole vector is written back)
      nv[v] = in ? nu : cur.own[v];
      if (MEASURE && in) {
        if (sizeof(T) == 4)
          dm32 = max(dm32, abs_bits32((float)radd(nu, -cur.own[v])));
        else
          dm = umax64(dm, abs_bits((double)radd(nu, -cur.own[v])));
      }
    }
    store4(X + e3(k, i, q0, m, pitch), nv);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      om[v] = oc[v];
      oc[v] = cur.op[v];
    }
    cur = nxt;
  }
  if (sizeof(T) == 4 && MEASURE) dm = abs_bits_of(__uint_as_float(dm32));
  return dm;
}

// After the black phase of iteration k (Algorithm 1): count it, test the
// change on check iterations, stop at the cap.
__device__ __forceinline__ void finalize3(const Desc3& d, SlotState* st, int k, int measure) {
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

// Scaled residual over tiles, both colours, in FP64.  ROLE kResidCheck: the
// residual stop of Algorithm 1's test on iterations that are multiples of K
// (decided by the last tile); kResidRefine: the defect correction's test
// after every correction, with r~ rounded to FP32 into rhs32 for the inner
// sweeps; kResidFinal: only rho of the current iterate is recorded.
template <typename T, int ROLE>
__global__ void __launch_bounds__(kThreads) k_resid3d(const Desc3* __restrict__ dp, SlotState* st,
                                                      const Tile* __restrict__ tiles, int ntiles) {
  __shared__ unsigned long long red[kWarpsY];
  __shared__ int ctl[2];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const Desc3& d = *dp;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    if (threadIdx.x == 0) {
      const int it = *((volatile int*)&st->iters);
      int skip = 0;
      if (ROLE == kResidCheck)
        skip = *((volatile int*)&st->converged) || it == 0 || (it % d.K) != 0 ||
               it == *((volatile int*)&st->checked_iter);
      const int kt = tl.row0 / d.m, it0 = tl.row0 - kt * d.m;
      if (!skip && !dbg_tile3(st, kt - 1, kt + 2, it0 - 1, it0 + tl.nrows + 1, tl.col0 - 1,
                              tl.col0 + kWarpCols + 1, d.m, d.pitch))
        skip = 1;
      ctl[0] = skip;
      ctl[1] = it;
    }
    __syncthreads();
    const int skip = ctl[0], it = ctl[1];
    __syncthreads();
    if (skip) continue;
    const int m = d.m, n = d.n, pitch = d.pitch;
    const int k = tl.row0 / m, ib = tl.row0 - k * m;
    const int q0 = tl.col0 + lane * kVec;
    const int rpw = (tl.nrows + kWarpsY - 1) / kWarpsY;
    const int i0 = ib + wy * rpw;
    const int i1 = min(i0 + rpw, ib + tl.nrows);
    unsigned long long rm = 0;
    for (int i = i0; i < i1; ++i) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T* Xs = (const T*)d.x[c];
        const T* Xo = (const T*)d.x[c ^ 1];
        const double* G = d.g64[c];
        T own[4], nm[4], nc[4], np[4], dn[4], up[4];
        load4(Xs + e3(k, i, q0, m, pitch), own);
        load4(Xo + e3(k, i - 1, q0, m, pitch), nm);
        load4(Xo + e3(k, i, q0, m, pitch), nc);
        load4(Xo + e3(k, i + 1, q0, m, pitch), np);
        load4(Xo + e3(k - 1, i, q0, m, pitch), dn);
        load4(Xo + e3(k + 1, i, q0, m, pitch), up);
        double gv[4] = {0.0, 0.0, 0.0, 0.0};
        if (G) load4(G + e3(k, i, q0, m, pitch), gv);
        T left = __shfl_up_sync(0xffffffffu, nc[3], 1);
        T right = __shfl_down_sync(0xffffffffu, nc[0], 1);
        if (lane == 0) left = Xo[e3(k, i, q0 - 1, m, pitch)];
        if (lane == 31) right = Xo[e3(k, i, q0 + kVec, m, pitch)];
        const int s = (i + k + c) & 1;
        const int qlim = (n + s) >> 1;
        T W[4], E[4];
        if (s == 0) {
          W[0] = nc[0]; W[1] = nc[1]; W[2] = nc[2]; W[3] = nc[3];
          E[0] = nc[1]; E[1] = nc[2]; E[2] = nc[3]; E[3] = right;
        } else {
          W[0] = left; W[1] = nc[0]; W[2] = nc[1]; W[3] = nc[2];
          E[0] = nc[0]; E[1] = nc[1]; E[2] = nc[2]; E[3] = nc[3];
        }
        float r32[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const double nb =
              __dadd_rn(__dadd_rn(__dadd_rn((double)nm[v], (double)np[v]), __dadd_rn((double)W[v], (double)E[v])),
                        __dadd_rn((double)dn[v], (double)up[v]));
          const double r = __dadd_rn(__dadd_rn(gv[v], nb), -__dmul_rn(6.0, (double)own[v]));
          const bool in = (q0 + v) <= qlim;
          if (in) rm = umax64(rm, abs_bits(r));
          r32[v] = in ? narrow_f64(r) : 0.0f;  // round to nearest even, on the integer units
        }
        if (ROLE == kResidRefine) store4(d.rhs32[c] + e3(k, i, q0, m, pitch), r32);
      }
    }
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

// ------------------------------------------------------------------------------------------------
// FP64 default phases on cubes: shared in-plane pair sums and rescaled unknowns
// ------------------------------------------------------------------------------------------------
//
// The reformulation of the 2D default path carried to the cube, with w = w/6:
// within plane k the four in-plane neighbours split into an upper-left and a
// lower-right pair, each formed once and used by two cells (s = (i + k + c) & 1
// plays the role of the 2D row parity); the neighbours below and above form a
// third pair; red values after step t of a chunk are carried as
// w^-(2t-1) u and black ones as w^-2t u, so the update is one FMA,
// X' = alpha X + ((DU + DL) + (D + U)) [+ gamma g].  The phase that updates a
// colour rewrites that colour's shell cells next to its strip at the scale the
// next phase reads them (from a copy saved after packing); chunks end at
// every tested iteration with unscaled values.  5 FP64 operations per update
// instead of 8.

struct Phase3 {
  double alpha, beta, gamma, dscale, nscale;
  int last;
};

constexpr int kF3Stages = 4;  // row buffers per warp
constexpr int kF3Ahead = 3;   // rows fetched ahead of the row being updated

template <bool HAS_G>
struct Stage3 {
  double op[32 * kVec];   // neighbour colour, row i + 1
  double own[32 * kVec];  // own colour, row i
  double dn[32 * kVec];   // neighbour colour, plane k - 1
  double up[32 * kVec];   // neighbour colour, plane k + 1
  double g[HAS_G ? 32 * kVec : 2];
  double edge[2];
};
template <bool HAS_G>
constexpr size_t f3_smem() {
  return (size_t)kWarpsY * kF3Stages * sizeof(Stage3<HAS_G>);
}

__device__ __forceinline__ void c3_copy16(void* dst, const void* src, int nbytes) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(src), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void c3_copy8_if(void* dst, const void* src, int nbytes, bool pred) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n @p cp.async.ca.shared.global [%0], [%1], 8, %2;\n}\n" ::"r"(saddr),
      "l"(src), "r"(nbytes), "r"((int)pred)
      : "memory");
}
template <int N>
__device__ __forceinline__ void c3_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copies row i of plane k (and its neighbours) into a stage; zero-fill when
// !valid; one group per row either way.
template <bool HAS_G>
__device__ __forceinline__ void f3_issue(Stage3<HAS_G>* st, int k, int i, bool valid, const double* O,
                                         const double* X, const double* G, int m, int pitch, int q0, int lane) {
  const int nb = valid ? 16 : 0;
  const double* o = valid ? O + e3(k, i + 1, q0, m, pitch) : O;
  const double* x = valid ? X + e3(k, i, q0, m, pitch) : X;
  const double* d = valid ? O + e3(k - 1, i, q0, m, pitch) : O;
  const double* u = valid ? O + e3(k + 1, i, q0, m, pitch) : O;
  c3_copy16(st->op + lane * kVec, o, nb);
  c3_copy16(st->op + lane * kVec + 2, o + 2, nb);
  c3_copy16(st->own + lane * kVec, x, nb);
  c3_copy16(st->own + lane * kVec + 2, x + 2, nb);
  c3_copy16(st->dn + lane * kVec, d, nb);
  c3_copy16(st->dn + lane * kVec + 2, d + 2, nb);
  c3_copy16(st->up + lane * kVec, u, nb);
  c3_copy16(st->up + lane * kVec + 2, u + 2, nb);
  if (HAS_G) {
    const double* gp = valid ? G + e3(k, i, q0, m, pitch) : G;
    c3_copy16(st->g + lane * kVec, gp, nb);
    c3_copy16(st->g + lane * kVec + 2, gp + 2, nb);
  }
  const bool right = lane == 31;
  const double* e = valid ? O + e3(k, i, right ? q0 + kVec : q0 - 1, m, pitch) : O;
  c3_copy8_if(&st->edge[right ? 1 : 0], e, valid ? 8 : 0, lane == 0 || right);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

struct Walk3 {
  double om[4], oc[4], dlp[4];
  double edge;  // lane r: the strip-edge pair of the r-th parity-1 row of the current group
  int ek;       // parity-1 rows of the group already taken
};

// Lane 0's upper-left pair in a parity-1 row, O[k][i-1][col0] +
// O[k][i][col0-1], reaches past the strip; formed row by row it costs a whole
// warp instruction on the FP64 pipe.  The pairs of 32 parity-1 rows i,
// i+2, ... are formed together (lane r: row i + 2r) and taken by shuffles.
__device__ __forceinline__ void f3_edges(Walk3& w, const double* __restrict__ O, int k, int m, int pitch, int col0,
                                         int i, int i1, int lane) {
  const int r = i + 2 * lane;
  double e = 0.0;
  if (r < i1) e = __dadd_rn(O[e3(k, r - 1, col0, m, pitch)], O[e3(k, r, col0 - 1, m, pitch)]);
  w.edge = e;
  w.ek = 0;
}
__device__ __forceinline__ double f3_edge(Walk3& w, const double* __restrict__ O, int k, int m, int pitch, int q0,
                                          int i, int i1, int lane) {
  if (w.ek == 32) f3_edges(w, O, k, m, pitch, q0 - lane * kVec, i, i1, lane);
  const double e = __shfl_sync(0xffffffffu, w.edge, w.ek);
  ++w.ek;
  return e;
}

// One row i of plane k (parity S = (i + k + colour) & 1 fixed at compile
// time; FIRST: no previous row, form the upper-left pairs directly; FULL:
// every cell of the strip is interior, no mask).
template <bool UNIT_BETA, bool HAS_G, bool MEASURE, bool FULL, int S, bool FIRST>
__device__ __forceinline__ void f3_row(Walk3& w, int k, int i, int i0, int i1, Stage3<HAS_G>* stages,
                                       const double* O, double* X, const double* G, int n, int m, int pitch, int q0,
                                       int lane, const Phase3& ph, unsigned long long& dm) {
  const int ahead = i + kF3Ahead;
  f3_issue<HAS_G>(stages + ((ahead - i0) & (kF3Stages - 1)), k, ahead, ahead < i1, O, X, G, m, pitch, q0, lane);
  c3_wait<kF3Ahead>();  // the buffer refilled above was read one row ago
  const Stage3<HAS_G>* st = stages + ((i - i0) & (kF3Stages - 1));
  double op[4], own[4], dn[4], up[4], gv[4];
  load4(st->op + lane * kVec, op);
  load4(st->own + lane * kVec, own);
  load4(st->dn + lane * kVec, dn);
  load4(st->up + lane * kVec, up);
  if (HAS_G) load4(st->g + lane * kVec, gv);
  double left = __shfl_up_sync(0xffffffffu, w.oc[3], 1);
  double right = __shfl_down_sync(0xffffffffu, w.oc[0], 1);
  if (lane == 0) left = st->edge[0];
  if (lane == 31) right = st->edge[1];
  double W[4], E[4];
  if (S == 0) {
    W[0] = w.oc[0]; W[1] = w.oc[1]; W[2] = w.oc[2]; W[3] = w.oc[3];
    E[0] = w.oc[1]; E[1] = w.oc[2]; E[2] = w.oc[3]; E[3] = right;
  } else {
    W[0] = left; W[1] = w.oc[0]; W[2] = w.oc[1]; W[3] = w.oc[2];
    E[0] = w.oc[0]; E[1] = w.oc[1]; E[2] = w.oc[2]; E[3] = w.oc[3];
  }
  double DL[4], DU[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) DL[v] = __dadd_rn(E[v], op[v]);
  if (FIRST) {
#pragma unroll
    for (int v = 0; v < 4; ++v) DU[v] = __dadd_rn(w.om[v], W[v]);
  } else if (S == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) DU[v] = w.dlp[v];
  } else {
    double d0 = __shfl_up_sync(0xffffffffu, w.dlp[3], 1);
    const double e0 = f3_edge(w, O, k, m, pitch, q0, i, i1, lane);  // om[0] + left, formed with the others
    if (lane == 0) d0 = e0;
    DU[0] = d0; DU[1] = w.dlp[0]; DU[2] = w.dlp[1]; DU[3] = w.dlp[2];
  }
  const int qlim = (n + S) >> 1;
  double nv[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double sum = __dadd_rn(__dadd_rn(DU[v], DL[v]), __dadd_rn(dn[v], up[v]));
    double t2;
    if (UNIT_BETA)
      t2 = HAS_G ? __fma_rn(ph.gamma, gv[v], sum) : sum;
    else
      t2 = HAS_G ? __fma_rn(ph.gamma, gv[v], __dmul_rn(ph.beta, sum)) : __dmul_rn(ph.beta, sum);
    const double nu = __fma_rn(ph.alpha, own[v], t2);
    const bool inside = FULL || (q0 + v) <= qlim;
    nv[v] = inside ? nu : own[v];  // cells past the interior keep their value
    if (MEASURE && inside) dm = umax64(dm, abs_bits(__fma_rn(-ph.dscale, own[v], nu)));
  }
  store4(X + e3(k, i, q0, m, pitch), nv);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    w.dlp[v] = DL[v];
    w.om[v] = w.oc[v];
    w.oc[v] = op[v];
  }
}

template <bool UNIT_BETA, bool HAS_G, bool MEASURE, bool FULL, int S0>
__device__ __forceinline__ void f3_rows(Walk3& w, int k, int i0, int i1, Stage3<HAS_G>* stages, const double* O,
                                        double* X, const double* G, int n, int m, int pitch, int q0, int lane,
                                        const Phase3& ph, unsigned long long& dm) {
  int i = i0;
  f3_row<UNIT_BETA, HAS_G, MEASURE, FULL, S0, true>(w, k, i, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph,
                                                    dm);
  ++i;
  for (; i + 1 < i1; i += 2) {
    f3_row<UNIT_BETA, HAS_G, MEASURE, FULL, 1 - S0, false>(w, k, i, i0, i1, stages, O, X, G, n, m, pitch, q0, lane,
                                                           ph, dm);
    f3_row<UNIT_BETA, HAS_G, MEASURE, FULL, S0, false>(w, k, i + 1, i0, i1, stages, O, X, G, n, m, pitch, q0, lane,
                                                       ph, dm);
  }
  if (i < i1)
    f3_row<UNIT_BETA, HAS_G, MEASURE, FULL, 1 - S0, false>(w, k, i, i0, i1, stages, O, X, G, n, m, pitch, q0, lane,
                                                           ph, dm);
}

// Saved unscaled shell of one colour array: planes 0 and N+1 (m rows of pitch
// elements each), rows 0 and N+1 of every plane (m x pitch each), and the
// column q = 0 and the east shell column of every row (m x m each).
__host__ __device__ __forceinline__ size_t shell3_elems(int m, int pitch) {
  return 4 * (size_t)m * pitch + 2 * (size_t)m * m;
}
__device__ __forceinline__ int east3(int n, int k, int i, int c) { return ((n + ((i + k + c) & 1)) >> 1) + 1; }

__global__ void k_shell_save3(const Desc3* __restrict__ dp, double* shell0, double* shell1) {
  const Desc3& d = *dp;
  const int n = d.n, m = d.m, pitch = d.pitch;
  const int c = blockIdx.y;
  const double* X = (const double*)d.x[c];
  double* R = c ? shell1 : shell0;
  const size_t mp = (size_t)m * pitch, mm = (size_t)m * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < shell3_elems(m, pitch);
       e += (size_t)gridDim.x * blockDim.x) {
    double v;
    if (e < mp) {
      v = X[e];  // plane 0
    } else if (e < 2 * mp) {
      v = X[(size_t)(n + 1) * mp + (e - mp)];  // plane N+1
    } else if (e < 3 * mp) {
      const size_t r = e - 2 * mp;  // row 0 of plane r / pitch
      v = X[((r / pitch) * m + 0) * pitch + r % pitch];
    } else if (e < 4 * mp) {
      const size_t r = e - 3 * mp;  // row N+1 of plane r / pitch
      v = X[((r / pitch) * m + (n + 1)) * pitch + r % pitch];
    } else if (e < 4 * mp + mm) {
      const size_t r = e - 4 * mp;
      v = X[e3((int)(r / m), (int)(r % m), 0, m, pitch)];
    } else {
      const size_t r = e - 4 * mp - mm;
      const int k = (int)(r / m), i = (int)(r % m);
      v = X[e3(k, i, east3(n, k, i, c), m, pitch)];
    }
    R[e] = v;
  }
}

// Rewrites this phase's colour's shell cells next to the strip at scale ns.
__device__ __forceinline__ void f3_shell(const Desc3& d, const double* __restrict__ R, double* __restrict__ X,
                                         int colour, int k, int i0, int i1, int col0, int q0, int lane, double ns) {
  const int n = d.n, m = d.m, pitch = d.pitch;
  const size_t mp = (size_t)m * pitch, mm = (size_t)m * m;
  __syncwarp();
  // the shell plane below (k = 1) and / or above (k = N), this strip's rows
  // and columns (both for N = 1)
  for (int side = 0; side < 2; ++side) {
    if (side == 0 ? k != 1 : k != n) continue;
    const size_t base = side == 0 ? 0 : mp;
    const int kk = side == 0 ? 0 : n + 1;
    for (int i = i0; i < i1; ++i) {
      double v[4];
      load4(R + base + (size_t)i * pitch + q0 + kOff, v);
#pragma unroll
      for (int t = 0; t < 4; ++t) v[t] = __dmul_rn(v[t], ns);
      store4(X + e3(kk, i, q0, m, pitch), v);
    }
  }
  if (i0 == 1) {  // row 0 of plane k
    double v[4];
    load4(R + 2 * mp + (size_t)k * pitch + q0 + kOff, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = __dmul_rn(v[t], ns);
    store4(X + e3(k, 0, q0, m, pitch), v);
  }
  if (i1 == n + 1) {  // row N+1 of plane k
    double v[4];
    load4(R + 3 * mp + (size_t)k * pitch + q0 + kOff, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = __dmul_rn(v[t], ns);
    store4(X + e3(k, n + 1, q0, m, pitch), v);
  }
  const bool west = col0 == 1, east = col0 + kWarpCols > ((n + 1) >> 1);
  if (west || east) {
    for (int i = i0 + lane; i < i1; i += 32) {
      if (west) X[e3(k, i, 0, m, pitch)] = __dmul_rn(R[4 * mp + (size_t)k * m + i], ns);
      if (east) X[e3(k, i, east3(n, k, i, colour), m, pitch)] = __dmul_rn(R[4 * mp + mm + (size_t)k * m + i], ns);
    }
  }
}

// A whole chunk of 2L phases in one launch, scheduled as a data flow.  The
// work items are (phase p, strip t), numbered p * nstrips + t; warps claim
// them in that order from a counter.  Item (p, t) may start once strip t and
// its neighbours -- the strips of the planes below and above, the row bands
// above and below and the column tiles left and right, the only ones whose
// cells its stencil reads or whose readers it could overwrite -- have
// finished phase p-1 (progress[t] counts the phases a strip has finished).
// Every dependency has a smaller number than the item that waits for it, so
// the smallest unfinished item can always run: the schedule cannot
// deadlock, needs no co-residency, lets fast SMs take more items and lets
// phase p+1 start on planes whose neighbours are done while phase p is
// still draining.  A strip publishes its progress with a release store after
// fencing its writes; every lane of a waiting warp reads the counters with
// acquire loads.  Every wait is bounded: past kFlowSpins polls the warp
// records an error in the slot state and returns (the host reports
// SOR_ERR_INTERNAL).  The last strip to finish the last phase closes the
// chunk's iterations.

template <bool HAS_G>
__global__ void __launch_bounds__(kThreads, 2) k_f3_flow(const Desc3* __restrict__ dp, SlotState* st,
                                                         const Tile* __restrict__ strips, int nstrips, int bands,
                                                         int ct, const double* __restrict__ shell0,
                                                         const double* __restrict__ shell1,
                                                         const Phase3* __restrict__ phases, int nphases,
                                                         unsigned* progress) {
  extern __shared__ __align__(16) unsigned char f3_mem[];
  const int lane = threadIdx.x & 31;
  Stage3<HAS_G>* stages = reinterpret_cast<Stage3<HAS_G>*>(f3_mem) + (threadIdx.x >> 5) * kF3Stages;
  const Desc3& d = *dp;
  int skip = 0, k0 = 0;
  if (lane == 0) {
    skip = *((volatile int*)&st->done);
    k0 = *((volatile int*)&st->iters);
  }
  skip = __shfl_sync(0xffffffffu, skip, 0);
  if (skip) return;  // done changes inside a launch only after its last item
  k0 = __shfl_sync(0xffffffffu, k0, 0);
  const int n = d.n, m = d.m, pitch = d.pitch;
  const long long items = (long long)nphases * nstrips;
  unsigned* claim = progress + nstrips;
  for (;;) {
    long long g = 0;
    if (lane == 0) g = (long long)atomicAdd(claim, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= items) break;
    const int p = (int)(g / nstrips), t = (int)(g - (long long)p * nstrips);
    const int colour = p & 1;
    const int kk = k0 + (p >> 1) + 1;
    const Phase3 ph = phases[p];
    const int measure = ((kk % d.K) == 0) || (kk >= d.max_iters);
    if (measure && !ph.last) {  // the host plan must end chunks at measured iterations
      if (lane == 0) {
        st->error = 1;
        st->done = 1;
      }
      return;
    }
    if (p > 0) {
      int nb[7];
      flow3_neighbours(t, n, bands, ct, nb);
      if (!flow_wait<7>(progress, nb, (unsigned)p, lane)) {
        if (lane == 0) {
          st->error = 1;
          st->done = 1;
        }
        return;
      }
    }
    const Tile tl = strips[t];
    const int k = tl.row0 / m, i0 = tl.row0 - k * m, i1 = i0 + tl.nrows;
    if (!dbg_tile3(st, k - 1, k + 2, i0 - 1, i1 + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1, m, pitch)) return;
    double* X = (double*)d.x[colour];
    const double* O = (const double*)d.x[colour ^ 1];
    const double* G = (const double*)d.g[colour];
    const int q0 = tl.col0 + lane * kVec;
    for (int a = 0; a < kF3Ahead; ++a)
      f3_issue<HAS_G>(stages + a, k, i0 + a, i0 + a < i1, O, X, G, m, pitch, q0, lane);
    Walk3 w;
    load4(O + e3(k, i0 - 1, q0, m, pitch), w.om);
    load4(O + e3(k, i0, q0, m, pitch), w.oc);
#pragma unroll
    for (int v = 0; v < 4; ++v) w.dlp[v] = 0.0;
    unsigned long long dm = 0;
    const int s0 = (i0 + k + colour) & 1;
    // the edge pairs of the first 32 parity-1 rows after the first row
    f3_edges(w, O, k, m, pitch, tl.col0, s0 ? i0 + 2 : i0 + 1, i1, lane);
    const bool unit = ph.beta == 1.0;
    if (measure) {  // the last iteration of the chunk: unscaled, change measured
      if (s0 == 0) f3_rows<false, HAS_G, true, false, 0>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
      else f3_rows<false, HAS_G, true, false, 1>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
    } else if (unit && tl.col0 + kWarpCols - 1 <= (n >> 1)) {  // every column of the strip interior in both parities
      if (s0 == 0) f3_rows<true, HAS_G, false, true, 0>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
      else f3_rows<true, HAS_G, false, true, 1>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
    } else if (unit) {
      if (s0 == 0) f3_rows<true, HAS_G, false, false, 0>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
      else f3_rows<true, HAS_G, false, false, 1>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
    } else {
      if (s0 == 0) f3_rows<false, HAS_G, false, false, 0>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
      else f3_rows<false, HAS_G, false, false, 1>(w, k, i0, i1, stages, O, X, G, n, m, pitch, q0, lane, ph, dm);
    }
    c3_wait<0>();
    f3_shell(d, colour ? shell1 : shell0, X, colour, k, i0, i1, tl.col0, q0, lane, ph.nscale);
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
          finalize3(d, st, k0 + (nphases >> 1), measure);
        }
      }
    }
    __syncwarp();
  }
}

// u += (double)d over the interior cells of colour c in rows [i0, i1) of
// plane k (this lane's packed columns), d just written by this lane.
__device__ __forceinline__ void correct3_rows(double* __restrict__ U, const float* __restrict__ D, int pitch,
                                              int m, int n, int colour, int k, int q0, int i0, int i1) {
  for (int i = i0; i < i1; ++i) {
    const int qlim = (n + ((i + k + colour) & 1)) >> 1;
    double u[4];
    float dv[4];
    load4(U + e3(k, i, q0, m, pitch), u);
    load4(D + e3(k, i, q0, m, pitch), dv);
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if ((q0 + v) <= qlim) u[v] = __dadd_rn(u[v], widen_f32(dv[v]));  // the widening is exact
    store4(U + e3(k, i, q0, m, pitch), u);
  }
}

// The exact-order phases (FP32, and FP64 with SOR_FLAG_EXACT_ORDER) under the
// same data-flow schedule: items (phase, strip) claimed in order, each
// waiting for its strip and the six neighbouring strips to finish the
// previous phase; the rows of a strip are swept by sweep3_rows.  A launch
// covers the iterations up to the next tested one, whose change it measures.
// CORRECT (the inner sweeps of the defect correction): each colour's last
// phase also adds its final d to u (d of that colour changes no more), and
// the last strip counts the correction.
template <typename T, bool HAS_G, bool CORRECT = false>
__global__ void __launch_bounds__(kThreads) k_3_flow(const Desc3* __restrict__ dp, SlotState* st,
                                                     const Tile* __restrict__ strips, int nstrips, int bands, int ct,
                                                     int nphases, unsigned* progress) {
  const int lane = threadIdx.x & 31;
  const Desc3& d = *dp;
  int skip = 0, k0 = 0;
  if (lane == 0) {
    skip = *((volatile int*)&st->done);
    k0 = *((volatile int*)&st->iters);
  }
  skip = __shfl_sync(0xffffffffu, skip, 0);
  if (skip) return;  // done changes inside a launch only after its last item
  k0 = __shfl_sync(0xffffffffu, k0, 0);
  const int n = d.n, m = d.m, pitch = d.pitch;
  const T a = sizeof(T) == 4 ? (T)d.a32 : (T)d.a64;
  const T b = sizeof(T) == 4 ? (T)d.b32 : (T)d.b64;
  const long long items = (long long)nphases * nstrips;
  unsigned* claim = progress + nstrips;
  const int last_it = k0 + (nphases >> 1);
  for (;;) {
    long long g = 0;
    if (lane == 0) g = (long long)atomicAdd(claim, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= items) break;
    const int p = (int)(g / nstrips), t = (int)(g - (long long)p * nstrips);
    const int colour = p & 1;
    const int kk = k0 + (p >> 1) + 1;
    const int measure = ((kk % d.K) == 0) || (kk >= d.max_iters);
    if (measure && kk != last_it) {  // the host plan must end launches at tested iterations
      if (lane == 0) {
        st->error = 1;
        st->done = 1;
      }
      return;
    }
    if (p > 0) {
      int nb[7];
      flow3_neighbours(t, n, bands, ct, nb);
      if (!flow_wait<7>(progress, nb, (unsigned)p, lane)) {
        if (lane == 0) {
          st->error = 1;
          st->done = 1;
        }
        return;
      }
    }
    const Tile tl = strips[t];
    const int k = tl.row0 / m, i0 = tl.row0 - k * m, i1 = i0 + tl.nrows;
    if (!dbg_tile3(st, k - 1, k + 2, i0 - 1, i1 + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1, m, pitch)) return;
    T* X = (T*)d.x[colour];
    const T* O = (const T*)d.x[colour ^ 1];
    const T* G = (const T*)d.g[colour];
    const int q0 = tl.col0 + lane * kVec;
    if (measure) {
      unsigned long long dm = sweep3_rows<T, true, HAS_G>(X, O, G, a, b, pitch, m, n, colour, k, q0, i0, i1, lane);
      dm = warp_max64(dm);
      if (lane == 0 && dm) atomicMax(&st->dmax_bits, dm);
    } else {
      (void)sweep3_rows<T, false, HAS_G>(X, O, G, a, b, pitch, m, n, colour, k, q0, i0, i1, lane);
    }
    if (CORRECT && p >= nphases - 2)
      correct3_rows(d.ucorr[colour], (const float*)X, pitch, m, n, colour, k, q0, i0, i1);
    __threadfence();  // this lane's cells are visible before the strip's progress is
    __syncwarp();
    if (lane == 0) {
      flow_st_release(progress + t, (unsigned)(p + 1));
      if (p == nphases - 1) {
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        if (prev == (unsigned)nstrips - 1u) {
          __threadfence();
          finalize3(d, st, last_it, measure);
          if (CORRECT) d.outer->outer += 1;
        }
      }
    }
    __syncwarp();
  }
}

// Constants of phase (t, colour) of a chunk of L iterations for w = omega/6.
Phase3 phase3_of(double omega, int t, int L, int colour) {
  const double w6 = omega / 6.0, omc = 1.0 - omega;
  Phase3 a;
  if (colour == 0)
    a.nscale = t == L ? 1.0 : std::pow(w6, -(2 * t - 1));
  else
    a.nscale = t == L ? 1.0 : std::pow(w6, -(2 * t));
  if (colour == 0) {
    if (t == L) {
      const double inv_a = t == 1 ? 1.0 : std::pow(w6, 2 * t - 3);
      const double inv_b = t == 1 ? 1.0 : std::pow(w6, 2 * t - 2);
      a.alpha = omc * inv_a;
      a.beta = w6 * inv_b;
      a.gamma = w6;
      a.dscale = inv_a;
      a.last = 1;
    } else {
      a.alpha = t == 1 ? omc / w6 : omc / (w6 * w6);
      a.beta = 1.0;
      a.gamma = std::pow(w6, -(2 * t - 2));
      a.dscale = 0.0;
      a.last = 0;
    }
  } else {
    if (t == L) {
      const double inv_b = t == 1 ? 1.0 : std::pow(w6, 2 * t - 2);
      a.alpha = omc * inv_b;
      a.beta = w6;
      a.gamma = w6;
      a.dscale = inv_b;
      a.last = 1;
    } else {
      a.alpha = omc / (w6 * w6);
      a.beta = 1.0;
      a.gamma = std::pow(w6, -(2 * t - 1));
      a.dscale = 0.0;
      a.last = 0;
    }
  }
  return a;
}

// Longest chunk whose carried scale stays below 2^400.
int fast3_lmax(double omega) {
  const double bits = 2.0 * std::log2(6.0 / omega);
  const int L = bits > 0.0 ? (int)std::floor(400.0 / bits) : 256;
  return std::max(1, std::min(L, 256));
}

// Opts both instantiations into their dynamic shared memory (before any
// capture: attribute calls stay out of graph capture).
cudaError_t fast3_prepare() {
  static cudaError_t state = cudaErrorNotReady;
  if (state == cudaErrorNotReady) {
    cudaError_t e = cudaFuncSetAttribute(k_f3_flow<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)f3_smem<false>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_f3_flow<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f3_smem<true>());
    state = e;
  }
  return state;
}

// Resident blocks per SM of the flow kernel (0 on failure).
int fast3_blocks_per_sm(bool has_g) {
  int nb = 0;
  cudaError_t e = has_g ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_f3_flow<true>, kThreads, f3_smem<true>())
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_f3_flow<false>, kThreads,
                                                                       f3_smem<false>());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_f3_flow(const Desc3* d, SlotState* st, const Tile* strips, int nstrips, int bands, int ct,
                           int grid, const double* shell0, const double* shell1, const Phase3* phases, int nphases,
                           unsigned* progress, bool has_g, cudaStream_t s) {
  const size_t sm = has_g ? f3_smem<true>() : f3_smem<false>();
  if (has_g)
    k_f3_flow<true><<<grid, kThreads, sm, s>>>(d, st, strips, nstrips, bands, ct, shell0, shell1, phases, nphases,
                                               progress);
  else
    k_f3_flow<false><<<grid, kThreads, sm, s>>>(d, st, strips, nstrips, bands, ct, shell0, shell1, phases, nphases,
                                                progress);
  return cudaGetLastError();
}

template <typename T>
int exact3_blocks_per_sm(bool has_g) {
  int nb = 0;
  cudaError_t e = has_g ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_3_flow<T, true>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_3_flow<T, false>, kThreads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <typename T>
cudaError_t launch_3_flow(const Desc3* d, SlotState* st, const Tile* strips, int nstrips, int bands, int ct,
                          int grid, int nphases, unsigned* progress, bool has_g, cudaStream_t s,
                          bool correct = false) {
  if (correct)
    k_3_flow<T, true, true><<<grid, kThreads, 0, s>>>(d, st, strips, nstrips, bands, ct, nphases, progress);
  else if (has_g)
    k_3_flow<T, true><<<grid, kThreads, 0, s>>>(d, st, strips, nstrips, bands, ct, nphases, progress);
  else
    k_3_flow<T, false><<<grid, kThreads, 0, s>>>(d, st, strips, nstrips, bands, ct, nphases, progress);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// FP32 iterations fused per tile, streamed through the planes (temporal blocking on cubes)
// ------------------------------------------------------------------------------------------------
//
// The 2D tile family's temporal blocking carried to the cube.  A tile is a
// block of TY rows x OQ packed columns over a run of up to TZ planes.  Its
// block walks the planes in order; at step s it stages plane s + 2 (both
// colours: TY + 2 HR rows x 128 packed columns, HR = 2T halo rows and HQ
// halo packed columns each side) into a ring of 2T + 3 plane slots in shared
// memory and runs phase p = 1 .. 2T (red first; the exact update of k_3_flow)
// on plane s - p + 1, in place.  When phase p reaches plane z, phase p - 1
// has already passed planes z - 1, z and z + 1, and phase p + 1 has not yet
// touched z - 1, so every read sees the values of the right phase.  Phase p
// covers only the rows and planes within 2T - p of the tile's output (a cell
// after t iterations depends on cells at most 2t rows or planes and t packed
// columns away), so the stale band that grows inward from the staged border
// never reaches the output.  Finished planes go to the other buffer pair
// (neighbouring tiles read their halos from the previous iterate), which the
// last block then makes the current one by swapping the descriptor's
// pointers.  Traffic per cell: one read and one write per T iterations, plus
// the halo re-reads.
//
// Measured on GB300 it is slower than the per-phase data-flow kernel on
// cubes up to 514^3 (depth 2: 121 and 181 GLUP/s on 258^3 and 514^3, depth
// 1: 140 and 220, per phase: 462 and 423).  A plane's band of about 22 rows
// per phase is spread over 16 warps, so a warp updates one or two rows and
// reuses no row in registers: the launch executes about 166 instructions per
// update with the issue slots 61 % busy, while the per-phase kernel is not
// bound by memory traffic at these sizes.  It is kept behind
// SOR_OPT_CUBE_DEPTH = 1 or 2; results are identical to the per-phase form.

template <int TD>
struct Tb3Geom {
  static constexpr int HR = 2 * TD;                    // halo rows
  static constexpr int HQ = TD <= 3 ? 4 : 8;           // halo packed columns (a multiple of 4, >= TD + 1)
  static constexpr int C = 128;                        // staged packed columns
  static constexpr int OQ = C - 2 * HQ;                // output packed columns
  static constexpr int TY = 16;                        // output rows
  static constexpr int RY = TY + 2 * HR;               // staged rows
  static constexpr int TZ = 32;                        // output planes
  static constexpr int NS = 2 * TD + 3;                // plane slots
  static constexpr int THREADS = TD == 1 ? 256 : 512;  // one block per SM at depth >= 2
  static constexpr size_t smem = (size_t)NS * 2 * RY * C * sizeof(float);
};

// One tile: output planes [k0, k0 + nz), rows [row0, row0 + nrows), packed
// columns [col0, col0 + OQ).
struct Tile3 {
  int k0, nz, row0, nrows, col0;
};

__device__ __forceinline__ void tb3_cp16(float* sdst, const float* gsrc, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(valid ? gsrc : nullptr),
               "r"(valid ? 16 : 0)
               : "memory");
}

// Row r of plane z, colour c, on the staged tile (this lane's 4 packed
// columns).  Sc: own colour of plane z; So / Sd / Su: the other colour of
// planes z, z - 1, z + 1.  out_cells: bit v set for cells of the tile's output
// whose change is measured (0 when not measured).
__device__ __forceinline__ void tb3_row(float* __restrict__ Sc, const float* __restrict__ So,
                                        const float* __restrict__ Sd, const float* __restrict__ Su,
                                        const float* __restrict__ Gp, int r, int S, int qf, int qlim, float a,
                                        float b, unsigned out_cells, unsigned& dm32, int lane) {
  constexpr int C = 128;
  const int o = r * C + 4 * lane;
  float own[4], om[4], oc[4], op[4], dn[4], up[4];
  load4(Sc + o, own);
  load4(So + o - C, om);
  load4(So + o, oc);
  load4(So + o + C, op);
  load4(Sd + o, dn);
  load4(Su + o, up);
  float W[4], E[4];
  if (S == 0) {
    const float side = __shfl_down_sync(0xffffffffu, oc[0], 1);
    W[0] = oc[0]; W[1] = oc[1]; W[2] = oc[2]; W[3] = oc[3];
    E[0] = oc[1]; E[1] = oc[2]; E[2] = oc[3]; E[3] = side;
  } else {
    const float side = __shfl_up_sync(0xffffffffu, oc[3], 1);
    W[0] = side; W[1] = oc[0]; W[2] = oc[1]; W[3] = oc[2];
    E[0] = oc[0]; E[1] = oc[1]; E[2] = oc[2]; E[3] = oc[3];
  }
  float gv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (Gp) {
    const float4 g4 = __ldg(reinterpret_cast<const float4*>(Gp));
    gv[0] = g4.x; gv[1] = g4.y; gv[2] = g4.z; gv[3] = g4.w;
  }
  // cells of staged columns 0 and 127 see a wrong W or E: like every cell
  // near the staged border they are stale, and the stale band never reaches
  // the output
  float nv[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float sum = radd(radd(radd(om[v], op[v]), radd(W[v], E[v])), radd(dn[v], up[v]));
    if (Gp) sum = radd(sum, gv[v]);
    const float nu = radd(rmul(a, own[v]), rmul(b, sum));
    const bool in = qf + v >= 1 && qf + v <= qlim;
    nv[v] = in ? nu : own[v];
    if (in && ((out_cells >> v) & 1u)) dm32 = max(dm32, abs_bits32(radd(nu, -own[v])));
  }
  store4(Sc + o, nv);
}

template <int TD>
__global__ void __launch_bounds__(Tb3Geom<TD>::THREADS) k_sweep3_tb(Desc3* dp, SlotState* st,
                                                                    const Tile3* __restrict__ tiles, int ntiles,
                                                                    int nt_req) {
  using Gm = Tb3Geom<TD>;
  constexpr int NW = Gm::THREADS / 32;
  constexpr int C = Gm::C;
  extern __shared__ __align__(16) float t3s[];
  __shared__ unsigned long long red[NW];
  __shared__ int ctl[4];  // skip, iterations, last iteration, measured
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = dp->n, m = dp->m, pitch = dp->pitch;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile3 tl = tiles[t];
    if (threadIdx.x == 0) {
      int skip = *((volatile int*)&st->done);
      const int k0 = *((volatile int*)&st->iters);
      const int nt = min(nt_req, dp->max_iters - k0);
      const int k_end = k0 + nt;
      const int measure = (k_end % dp->K) == 0 || k_end >= dp->max_iters;
      for (int j = k0 + 1; j < k_end && !skip; ++j)  // the host plan ends launches at tested iterations
        if ((j % dp->K) == 0) {
          st->error = 1;
          st->done = 1;
          skip = 1;
        }
      if (nt <= 0) skip = 1;
      // the tile's output planes, rows and columns lie inside the arrays
      if (!skip && !dbg_tile3(st, tl.k0, tl.k0 + tl.nz, tl.row0, tl.row0 + tl.nrows, tl.col0, tl.col0 + Gm::OQ,
                              dp->m, dp->pitch))
        skip = 1;
      ctl[0] = skip;
      ctl[1] = nt;
      ctl[2] = k_end;
      ctl[3] = measure;
    }
    __syncthreads();
    const int skip = ctl[0], nt = ctl[1], k_end = ctl[2], measure = ctl[3];
    __syncthreads();
    if (skip) continue;

    const float* X0 = (const float*)dp->x[0];  // the current pair: staged from
    const float* X1 = (const float*)dp->x[1];
    float* Y0 = (float*)dp->xalt[0];  // the other pair: the tile's output goes here
    float* Y1 = (float*)dp->xalt[1];
    const float* G0 = (const float*)dp->g[0];
    const float* G1 = (const float*)dp->g[1];
    const float a = dp->a32, b = dp->b32;
    const int base_r = tl.row0 - Gm::HR;
    const int base_q = tl.col0 - Gm::HQ;
    const int base_e = base_q + kOff;  // element of staged column 0 (a multiple of 4)
    const int zlo = tl.k0, zhi = tl.k0 + tl.nz;  // output planes [zlo, zhi)
    const int z_first = max(1, zlo - 2 * nt + 1);  // the first plane of phase 1 (the first step)
    const int z_last = zhi - 1 + 2 * nt - 1;       // the step of phase 2nt on the last output plane
    const int z_in = min(m - 1, zhi + 2 * nt - 1);  // the last plane staged
    auto plane = [&](int z, int c) -> float* {
      return t3s + ((size_t)((z + 8 * Gm::NS) % Gm::NS) * 2 + c) * Gm::RY * C;
    };
    // plane z of both colours into its slot, rows and columns outside the
    // array reading as 0; one copy group per call
    auto stage = [&](int z) {
      if (z <= z_in) {
        for (int idx = threadIdx.x; idx < 2 * Gm::RY * 32; idx += blockDim.x) {
          const int c = idx / (Gm::RY * 32);
          const int rr = (idx >> 5) - c * Gm::RY;
          const int ln = idx & 31;
          const int i = base_r + rr;
          const int e = base_e + 4 * ln;
          const bool valid = i >= 0 && i < m && e >= 0 && e + 4 <= pitch;
          const float* gp = valid ? (c ? X1 : X0) + ((size_t)z * m + i) * pitch + e : nullptr;
          tb3_cp16(plane(z, c) + rr * C + 4 * ln, gp, valid);
        }
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    stage(z_first - 1);
    stage(z_first);
    stage(z_first + 1);
    unsigned dm32 = 0;
    for (int s = z_first; s <= z_last; ++s) {
      stage(s + 2);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // plane s + 1 has arrived
      __syncthreads();
#pragma unroll 1
      for (int p = 1; p <= 2 * nt; ++p) {
        const int z = s - p + 1;
        const int reach = 2 * nt - p;
        const int c = (p - 1) & 1;
        if (z >= max(1, zlo - reach) && z <= min(n, zhi - 1 + reach)) {
          const bool lastm = measure && p >= 2 * nt - 1 && z >= zlo && z < zhi;
          const int r_lo = max(Gm::HR - reach, 1 - base_r);
          const int r_hi = min(Gm::HR + tl.nrows + reach, n + 1 - base_r);
          float* Sc = plane(z, c);
          const float* So = plane(z, c ^ 1);
          const float* Sd = plane(z - 1, c ^ 1);
          const float* Su = plane(z + 1, c ^ 1);
          const float* Gc = c ? G1 : G0;
          const int qf = base_q + 4 * lane;
          unsigned outc = 0;
          if (lastm)
#pragma unroll
            for (int v = 0; v < 4; ++v)
              outc |= (unsigned)(4 * lane + v >= Gm::HQ && 4 * lane + v < Gm::HQ + Gm::OQ) << v;
          for (int r = r_lo + warp; r < r_hi; r += NW) {
            const int i = base_r + r;
            const int S = (i + z + c) & 1;
            const int qlim = (n + S) >> 1;
            const float* Gp = (Gc && qf <= qlim && qf + 3 >= 1) ? Gc + ((size_t)z * m + i) * pitch + qf + kOff : nullptr;
            const bool out_row = r >= Gm::HR && r < Gm::HR + tl.nrows;
            tb3_row(Sc, So, Sd, Su, Gp, r, S, qf, qlim, a, b, out_row ? outc : 0u, dm32, lane);
          }
        }
        __syncthreads();
      }
      // plane s - 2nt + 1 has had its last phase: its output rows and columns to the other pair
      const int zo = s - 2 * nt + 1;
      if (zo >= zlo && zo < zhi) {
        for (int idx = threadIdx.x; idx < 2 * tl.nrows * 32; idx += blockDim.x) {
          const int c = idx / (tl.nrows * 32);
          const int rr = (idx >> 5) - c * tl.nrows;
          const int col = 4 * (idx & 31);
          if (col < Gm::HQ || col >= Gm::HQ + Gm::OQ) continue;
          const int i = tl.row0 + rr;
          const int qlim = (n + ((i + zo + c) & 1)) >> 1;
          const int qf = base_q + col;
          if (qf > qlim) continue;
          float v4[4];
          load4(plane(zo, c) + (Gm::HR + rr) * C + col, v4);
          float* Yd = (c ? Y1 : Y0) + ((size_t)zo * m + i) * pitch + qf + kOff;
          if (qf + 3 <= qlim) {
            store4(Yd, v4);
          } else {
#pragma unroll
            for (int v = 0; v < 4; ++v)
              if (qf + v <= qlim) Yd[v] = v4[v];
          }
        }
      }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // the groups past the last plane are empty
    if (measure) {
      unsigned long long dm = warp_max64(abs_bits_of(__uint_as_float(dm32)));
      if (lane == 0) red[warp] = dm;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long mm = 0;
        for (int w = 0; w < NW; ++w) mm = umax64(mm, red[w]);
        if (mm) atomicMax(&st->dmax_bits, mm);
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(&st->arrive, 1u);
      if (prev == (unsigned)ntiles - 1u) {  // every tile is written: the other pair becomes the current one
        __threadfence();
        void* t0 = dp->x[0];
        void* t1 = dp->x[1];
        dp->x[0] = dp->xalt[0];
        dp->x[1] = dp->xalt[1];
        dp->xalt[0] = t0;
        dp->xalt[1] = t1;
        finalize3(*dp, st, k_end, measure);
      }
    }
    __syncthreads();  // the next tile reuses the plane slots
  }
}

template <int TD>
cudaError_t tb3_prepare() {
  return cudaFuncSetAttribute(k_sweep3_tb<TD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tb3Geom<TD>::smem);
}

template <int TD>
int tb3_blocks_per_sm() {
  int nb = 0;
  if (tb3_prepare<TD>() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep3_tb<TD>, Tb3Geom<TD>::THREADS, Tb3Geom<TD>::smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <int TD>
cudaError_t launch_sweep3_tb(Desc3* d, SlotState* st, const Tile3* tiles, int ntiles, int grid, int nt,
                             cudaStream_t s) {
  count_kernel_launches(1);
  k_sweep3_tb<TD><<<grid, Tb3Geom<TD>::THREADS, Tb3Geom<TD>::smem, s>>>(d, st, tiles, ntiles, nt);
  return cudaGetLastError();
}

// The tiles of a cube for depth TD.
template <int TD>
std::vector<Tile3> tb3_tiles(int n) {
  using Gm = Tb3Geom<TD>;
  std::vector<Tile3> out;
  const int qmax = (n + 1) / 2;
  for (int k0 = 1; k0 <= n; k0 += Gm::TZ)
    for (int r0 = 1; r0 <= n; r0 += Gm::TY)
      for (int q0 = 1; q0 <= qmax; q0 += Gm::OQ)
        out.push_back(Tile3{k0, std::min(Gm::TZ, n - k0 + 1), r0, std::min(Gm::TY, n - r0 + 1), q0});
  return out;
}

// Unpacks the descriptor's current pair (the blocked sweeps swap pairs on the device).
template <typename T>
__global__ void k_unpack3d_cur(const Desc3* __restrict__ dp, double* u) {
  const int n = dp->n, pitch = dp->pitch, m = n + 2;
  const T* x0 = (const T*)dp->x[0];
  const T* x1 = (const T*)dp->x[1];
  const int qw = (n + 1) / 2 + 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, k = blockIdx.z;
  if (q >= qw) return;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int j = 2 * q - 1 + t;
    if (j < 0 || j >= m) continue;
    const int c = (i + j + k) & 1;
    u[((size_t)k * m + i) * m + j] = (double)(c ? x1 : x0)[e3(k, i, q, m, pitch)];
  }
}

#define SOR3_CK(ctx, expr)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      std::ostringstream os_;                                                                 \
      os_ << #expr << ": " << cudaGetErrorString(e_) << " (" << __FILE__ << ":" << __LINE__ << ")"; \
      (ctx)->set_error(os_.str());                                                            \
      return SOR_ERR_CUDA;                                                                    \
    }                                                                                         \
  } while (0)

constexpr int kMax3dN = 1200;  // interior side limit (int row indices, sizes far below the budget)

// Device buffers of one 3D solve, released in the destructor.
struct Buffers3 {
  Ctx* c = nullptr;
  std::vector<void*> ptrs;
  size_t reserved = 0;
  void* get(size_t bytes) {
    void* p = ctx_dev_alloc(c, bytes);
    if (p) ptrs.push_back(p);
    return p;
  }
  ~Buffers3() {
    for (void* p : ptrs) ctx_dev_free(c, p);
    if (reserved) ctx_release(c, reserved);
  }
};

// One cube solve on stream s (the context's stream for sor_solve3d, a worker's
// own stream for batched cube requests).  wait_budget: wait for device memory
// under the context's budget instead of failing (batched requests).
template <typename T>
sor_status run3d(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out, sor_result* res,
                 cudaStream_t s, bool wait_budget) {
  const double t0 = now_s();
  const int n = p->n, m = n + 2;
  const Layout L = Layout::make(n);
  const int pitch = L.pitch;
  const size_t elems = (size_t)m * m * pitch;
  const size_t ncube = (size_t)m * m * m, nf = (size_t)n * n * n;
  const bool has_f = f != nullptr;
  const bool in_dev = is_device_ptr(u0), f_dev = has_f && is_device_ptr(f), out_dev = is_device_ptr(u_out);
  const double w = p->omega <= 0.0 ? sor_omega_opt(n) : p->omega;
  const int stop = p->stop == SOR_STOP_MAXDELTA ? kStopDelta : kStopResid;
  // FP64 default: the rescaled phases with shared pair sums (within 1e-12 of
  // the exact order); SOR_FLAG_EXACT_ORDER or FP32: the exact-order phases
  bool fast = sizeof(T) == 8 && !(p->flags & SOR_FLAG_EXACT_ORDER);
  if (fast) SOR3_CK(c, fast3_prepare());
  // FP32: blocked sweeps of SOR_OPT_CUBE_DEPTH iterations per launch (0, the
  // default: the per-phase flow kernel, faster here); same results either way
  const int tbd = sizeof(T) == 4 ? c->opt_cube_depth.load() : 0;
  const int tb_bps = tbd == 1 ? tb3_blocks_per_sm<1>() : tbd == 2 ? tb3_blocks_per_sm<2>() : 0;
  const bool tb = tbd > 0 && tb_bps > 0;
  std::vector<Tile3> tb_tiles;
  if (tb) tb_tiles = tbd == 1 ? tb3_tiles<1>(n) : tb3_tiles<2>(n);
  const int ntb = (int)tb_tiles.size();
  const int tb_grid = std::max(1, std::min(ntb, c->sm_count * std::max(1, tb_bps)));
  const int bps = fast ? fast3_blocks_per_sm(has_f) : exact3_blocks_per_sm<T>(has_f);
  if (bps < 1) {
    c->set_error("3D phase kernel does not fit on an SM");
    return SOR_ERR_CUDA;
  }
  std::vector<Tile> strips;
  const int bands = build_strips3(L, c->sm_count * bps * kWarpsY, &strips);
  const int flow_grid = c->sm_count * bps;
  const int nst = (int)strips.size();
  const size_t shell_elems = shell3_elems(m, pitch);
  const int lmax = fast3_lmax(w);
  constexpr int kTables = 16;  // phase tables of distinct chunk lengths held at once

  // tiles: plane k, rows of 32, columns of 128 packed cells
  std::vector<Tile> tiles;
  for (int k = 1; k <= n; ++k)
    for (int r = 0; r < L.row_tiles(); ++r)
      for (int t = 0; t < L.col_tiles(); ++t)
        tiles.push_back(Tile{0, k * m + 1 + r * kTileRows, 1 + t * kWarpCols, std::min(kTileRows, n - r * kTileRows)});
  const int nt = (int)tiles.size();

  size_t bytes = 2 * elems * sizeof(T) + sizeof(Desc3) + sizeof(SlotState) + sizeof(Tile) * nt + 1024;
  bytes += sizeof(Tile) * nst + sizeof(unsigned) * (nst + 1);
  if (fast) bytes += 2 * shell_elems * sizeof(double) + sizeof(Phase3) * 2 * (size_t)lmax * kTables;
  if (has_f) bytes += 2 * elems * sizeof(T) + (sizeof(T) == 4 ? 2 * elems * sizeof(double) : 0);
  if (tb) bytes += 2 * elems * sizeof(T) + sizeof(Tile3) * (size_t)ntb;
  const bool stage_u = !in_dev || !out_dev;
  if (stage_u) bytes += ncube * sizeof(double);
  if (has_f && !f_dev) bytes += nf * sizeof(double);
  Buffers3 B;
  B.c = c;
  sor_status rs = ctx_reserve(c, bytes, wait_budget, -1.0);
  if (rs != SOR_OK) {
    c->set_error("3D solve does not fit the device-memory budget");
    return rs;
  }
  B.reserved = bytes;
  T* x[2] = {(T*)B.get(elems * sizeof(T)), (T*)B.get(elems * sizeof(T))};
  T* g[2] = {nullptr, nullptr};
  double* g64[2] = {nullptr, nullptr};
  if (has_f) {
    g[0] = (T*)B.get(elems * sizeof(T));
    g[1] = (T*)B.get(elems * sizeof(T));
    if (sizeof(T) == 4) {
      g64[0] = (double*)B.get(elems * sizeof(double));
      g64[1] = (double*)B.get(elems * sizeof(double));
    } else {
      g64[0] = (double*)g[0];
      g64[1] = (double*)g[1];
    }
  }
  Desc3* d_desc = (Desc3*)B.get(sizeof(Desc3));
  SlotState* d_state = (SlotState*)B.get(sizeof(SlotState));
  Tile* d_tiles = (Tile*)B.get(sizeof(Tile) * nt);
  Tile* d_strips = (Tile*)B.get(sizeof(Tile) * nst);
  double* d_shell0 = fast ? (double*)B.get(shell_elems * sizeof(double)) : nullptr;
  unsigned* d_progress = (unsigned*)B.get(sizeof(unsigned) * (nst + 1));
  Phase3* d_tables = fast ? (Phase3*)B.get(sizeof(Phase3) * 2 * (size_t)lmax * kTables) : nullptr;
  double* d_shell1 = fast ? (double*)B.get(shell_elems * sizeof(double)) : nullptr;
  double* d_u = stage_u ? (double*)B.get(ncube * sizeof(double)) : nullptr;
  double* d_f = (has_f && !f_dev) ? (double*)B.get(nf * sizeof(double)) : nullptr;
  T* xalt[2] = {tb ? (T*)B.get(elems * sizeof(T)) : nullptr, tb ? (T*)B.get(elems * sizeof(T)) : nullptr};
  Tile3* d_tb = tb ? (Tile3*)B.get(sizeof(Tile3) * (size_t)ntb) : nullptr;
  if ((tb && (!xalt[0] || !xalt[1] || !d_tb)) ||
      !x[0] || !x[1] || (has_f && (!g[0] || !g[1] || !g64[0] || !g64[1])) || !d_desc || !d_state || !d_tiles ||
      (stage_u && !d_u) || (has_f && !f_dev && !d_f) || !d_strips || !d_progress || (fast && (!d_shell0 || !d_shell1 || !d_tables))) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }

  Desc3 d;
  std::memset(&d, 0, sizeof(d));
  d.x[0] = x[0];
  d.x[1] = x[1];
  d.xalt[0] = xalt[0];
  d.xalt[1] = xalt[1];
  d.g[0] = g[0];
  d.g[1] = g[1];
  d.g64[0] = g64[0];
  d.g64[1] = g64[1];
  d.n = n;
  d.m = m;
  d.pitch = pitch;
  d.K = p->check_every;
  d.max_iters = p->max_iters;
  d.stop = stop;
  d.tiles = nt;
  d.a64 = 1.0 - w;
  d.b64 = w / 6.0;
  d.a32 = (float)(1.0 - w);
  d.b32 = (float)(w / 6.0);
  d.tol = p->tol;
  d.stall = p->stall_window;
  SlotState st;
  std::memset(&st, 0, sizeof(st));
  st.checked_iter = -1;
  st.last_dmax = -1.0;
  st.last_rho = -1.0;
  st.best_rho = HUGE_VAL;
  st.done = p->max_iters == 0;

  for (int k = 0; k < 2; ++k) {
    SOR3_CK(c, cudaMemsetAsync(x[k], 0, elems * sizeof(T), s));
    if (has_f) SOR3_CK(c, cudaMemsetAsync(g[k], 0, elems * sizeof(T), s));
    if (has_f && sizeof(T) == 4) SOR3_CK(c, cudaMemsetAsync(g64[k], 0, elems * sizeof(double), s));
  }
  SOR3_CK(c, cudaMemcpyAsync(d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, s));
  SOR3_CK(c, cudaMemcpyAsync(d_state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  SOR3_CK(c, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, s));
  SOR3_CK(c, cudaMemcpyAsync(d_strips, strips.data(), sizeof(Tile) * nst, cudaMemcpyHostToDevice, s));
  if (tb) SOR3_CK(c, cudaMemcpyAsync(d_tb, tb_tiles.data(), sizeof(Tile3) * ntb, cudaMemcpyHostToDevice, s));
  const double* u_src = u0;
  if (!in_dev) {
    SOR3_CK(c, cudaMemcpyAsync(d_u, u0, ncube * sizeof(double), cudaMemcpyHostToDevice, s));
    u_src = d_u;
  }
  const double* f_src = f;
  if (has_f && !f_dev) {
    SOR3_CK(c, cudaMemcpyAsync(d_f, f, nf * sizeof(double), cudaMemcpyHostToDevice, s));
    f_src = d_f;
  }
  const double h = 1.0 / (double)(n + 1);
  const dim3 pgrid((L.qw + kWarpCols - 1) / kWarpCols, m, m);
  k_pack3d<T><<<pgrid, kWarpCols, 0, s>>>(u_src, f_src, n, pitch, h * h, x[0], x[1], g[0], g[1],
                                          sizeof(T) == 4 ? g64[0] : nullptr, sizeof(T) == 4 ? g64[1] : nullptr,
                                          d_state);
  SOR3_CK(c, cudaGetLastError());
  if (tb)  // the other pair starts as a copy (its shell never changes; every launch rewrites the interior)
    for (int k = 0; k < 2; ++k)
      SOR3_CK(c, cudaMemcpyAsync(xalt[k], x[k], elems * sizeof(T), cudaMemcpyDeviceToDevice, s));
  int lrun = lmax;  // chunk cap of the rescaled phases for these inputs
  if (fast) {
    // input magnitudes bound the rescaled phases' chunk length; inputs they
    // cannot carry take the exact-order phases (the same strips and grid:
    // the exact flow kernel needs no co-residency)
    SlotState hs;
    SOR3_CK(c, cudaMemcpyAsync(&hs, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR3_CK(c, cudaStreamSynchronize(s));
    double umax = 0.0, gmax = 0.0;
    std::memcpy(&umax, &hs.umax_bits, sizeof(double));
    std::memcpy(&gmax, &hs.gmax_bits, sizeof(double));
    const int cap = rescaled_lcap(umax, gmax, n, 3, w);
    if (cap == 0)
      fast = false;
    else
      lrun = std::min(lmax, cap);
  }
  if (fast) {  // unscaled copy of both colours' shells, for the per-phase rewrite
    const int sb = (int)std::min<size_t>((shell_elems + 255) / 256, (size_t)c->sm_count * 8);
    k_shell_save3<<<dim3(sb, 2), 256, 0, s>>>(d_desc, d_shell0, d_shell1);
    SOR3_CK(c, cudaGetLastError());
  }

  const int grid = std::min(nt, c->sm_count * 8);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SOR3_CK(c, cudaEventCreate(&ev0));
  SOR3_CK(c, cudaEventCreate(&ev1));
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

  // A batch of Lc iterations after iteration `first` runs as chunks that end
  // at every tested iteration (a multiple of K or the cap), one flow launch
  // each; on the FP64 default path chunks also stay within the scale cap and
  // take their phase constants from a device table per chunk length
  // (the claim counter numbers 2 L x strips items in 32 bits: L is capped
  // to keep that below 2^30)
  const long long lcap = std::min<long long>(fast ? lrun : (1LL << 30), std::max(1LL, (1LL << 29) / nst));
  auto plan_chunks = [&](long long first, int Lc) {
    std::vector<int> out;
    int done_it = 0;
    while (done_it < Lc) {
      const long long at = first + done_it;
      const long long next_m = std::min<long long>((at / d.K + 1) * d.K, p->max_iters);
      const int Ls = (int)std::min<long long>({lcap, next_m - at, (long long)(Lc - done_it)});
      out.push_back(Ls);
      done_it += Ls;
    }
    return out;
  };
  std::map<int, int> table_of;  // chunk length -> table slot
  std::vector<std::vector<Phase3>> host_tables(kTables);
  // uploads the tables the batch needs (outside any capture); when the slots
  // run out, the captured graphs that name them are dropped first
  auto ensure_tables = [&](const std::vector<int>& lens) -> sor_status {
    for (int Ls : lens) {
      if (table_of.count(Ls)) continue;
      if ((int)table_of.size() == kTables) {
        SOR3_CK(c, cudaStreamSynchronize(s));
        for (auto& kv : cl.graphs) cudaGraphExecDestroy(kv.second);
        cl.graphs.clear();
        table_of.clear();
      }
      const int slot = (int)table_of.size();
      std::vector<Phase3>& h = host_tables[slot];
      h.resize(2 * (size_t)Ls);
      for (int t = 1; t <= Ls; ++t)
        for (int colour = 0; colour < 2; ++colour) h[2 * (t - 1) + colour] = phase3_of(w, t, Ls, colour);
      SOR3_CK(c, cudaMemcpyAsync(d_tables + (size_t)slot * 2 * lmax, h.data(), sizeof(Phase3) * h.size(),
                                 cudaMemcpyHostToDevice, s));
      table_of[Ls] = slot;
    }
    return SOR_OK;
  };
  auto enqueue = [&](int first, int Lc) -> sor_status {
    int done_it = 0;
    for (int Ls : plan_chunks(first, Lc)) {
      if (tb) {  // blocks of tbd iterations, the last one ending the chunk
        for (int it = 0; it < Ls; it += tbd) {
          const int nit = std::min(tbd, Ls - it);
          SOR3_CK(c, tbd == 1 ? launch_sweep3_tb<1>(d_desc, d_state, d_tb, ntb, tb_grid, nit, s)
                              : launch_sweep3_tb<2>(d_desc, d_state, d_tb, ntb, tb_grid, nit, s));
        }
        done_it += Ls;
        if (stop == kStopResid && (first + done_it) % d.K == 0)
          k_resid3d<T, kResidCheck><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
        continue;
      }
      SOR3_CK(c, cudaMemsetAsync(d_progress, 0, sizeof(unsigned) * (nst + 1), s));
      if (fast)
        SOR3_CK(c, launch_f3_flow(d_desc, d_state, d_strips, nst, bands, L.col_tiles(), flow_grid, d_shell0,
                                  d_shell1, d_tables + (size_t)table_of.at(Ls) * 2 * lmax, 2 * Ls, d_progress,
                                  has_f, s));
      else
        SOR3_CK(c, launch_3_flow<T>(d_desc, d_state, d_strips, nst, bands, L.col_tiles(), flow_grid, 2 * Ls,
                                    d_progress, has_f, s));
      done_it += Ls;
      if (stop == kStopResid && (first + done_it) % d.K == 0)
        k_resid3d<T, kResidCheck><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
    }
    SOR3_CK(c, cudaGetLastError());
    return SOR_OK;
  };
  // iterations per host check: a whole number of test intervals when K fits,
  // so every batch starts at a tested iteration and one graph serves them all
  const int chunk0 = c->opt_chunk.load() > 0 ? c->opt_chunk.load() : 64;
  const int chunk = d.K <= chunk0 ? (chunk0 / d.K) * d.K : chunk0;
  const bool use_graphs = c->opt_graphs.load() != 0;
  SOR3_CK(c, cudaEventRecord(ev0, s));
  long long planned = 0;
  bool finished = st.done != 0;
  while (!finished && planned < p->max_iters) {
    if (c->closing.load()) return SOR_ERR_CANCELLED;  // the context is being destroyed
    int Lc = (int)std::min<long long>(chunk, p->max_iters - planned);
    if (d.K > chunk0)  // batches end at tested iterations: few distinct chunk lengths
      Lc = (int)std::min<long long>(Lc, std::min<long long>((planned / d.K + 1) * d.K, p->max_iters) - planned);
    if (fast) {
      const sor_status ts = ensure_tables(plan_chunks(planned, Lc));
      if (ts != SOR_OK) return ts;
    }
    if (use_graphs) {
      // the chunk ends and the residual launches depend on where the tested
      // iterations fall in the batch
      const std::pair<int, int> key(Lc, (int)(planned % d.K));
      auto itg = cl.graphs.find(key);
      if (itg == cl.graphs.end()) {
        cudaGraph_t gr = nullptr;
        SOR3_CK(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const sor_status es = enqueue((int)planned, Lc);
        const cudaError_t ce = cudaStreamEndCapture(s, &gr);
        if (es != SOR_OK) {
          if (gr) cudaGraphDestroy(gr);
          return es;
        }
        SOR3_CK(c, ce);
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        SOR3_CK(c, ie);
        itg = cl.graphs.emplace(key, ex).first;
      }
      SOR3_CK(c, cudaGraphLaunch(itg->second, s));
    } else {
      const sor_status es = enqueue((int)planned, Lc);
      if (es != SOR_OK) return es;
    }
    planned += Lc;
    SOR3_CK(c, cudaMemcpyAsync(h_state, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR3_CK(c, cudaStreamSynchronize(s));
    finished = h_state->done != 0;
  }
  SOR3_CK(c, cudaEventRecord(ev1, s));
  k_resid3d<T, kResidFinal><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
  SOR3_CK(c, cudaGetLastError());
  double* out_dst = out_dev ? u_out : d_u;
  if (tb)  // the current pair is the descriptor's (the blocked launches swap pairs on the device)
    k_unpack3d_cur<T><<<pgrid, kWarpCols, 0, s>>>(d_desc, out_dst);
  else
    k_unpack3d<T><<<pgrid, kWarpCols, 0, s>>>(x[0], x[1], n, pitch, out_dst);
  SOR3_CK(c, cudaGetLastError());
  if (!out_dev) SOR3_CK(c, cudaMemcpyAsync(u_out, d_u, ncube * sizeof(double), cudaMemcpyDeviceToHost, s));
  SOR3_CK(c, cudaMemcpyAsync(h_state, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
  SOR3_CK(c, cudaStreamSynchronize(s));
  float ms = 0.0f;
  SOR3_CK(c, cudaEventElapsedTime(&ms, ev0, ev1));
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

// The bounded wait of the flow kernels on one progress counter: one warp
// waits for counter >= 1 and records whether it gave up.
__global__ void k_flow_wait_probe(const unsigned* progress, int polls, int* timed_out) {
  const int lane = threadIdx.x & 31;
  const int nb[1] = {0};
  const bool ok = flow_wait<1>(progress, nb, 1u, lane, polls);
  if (lane == 0) *timed_out = ok ? 0 : 1;
}

// Defect correction on a cube (SOR_FP32_REFINE): per outer step the FP64
// residual test, which also rounds r~ to FP32 as the right side; inner
// red-black FP32 sweeps on A d = r~ from d = 0 (the exact-order flow
// kernel, whose last phase of each colour also adds d to u in FP64).  One step is a graph replayed up to max_iters /
// inner times; once the test passes, the device skips the remaining sweeps
// and corrections, and the host stops at its next poll.
sor_status run3d_refine(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                        sor_result* res, cudaStream_t s, bool wait_budget) {
  const double t0 = now_s();
  const int n = p->n, m = n + 2;
  const Layout L = Layout::make(n);
  const int pitch = L.pitch;
  const size_t elems = (size_t)m * m * pitch;
  const size_t ncube = (size_t)m * m * m, nf = (size_t)n * n * n;
  const bool has_f = f != nullptr;
  const bool in_dev = is_device_ptr(u0), f_dev = has_f && is_device_ptr(f), out_dev = is_device_ptr(u_out);
  const double w = p->omega <= 0.0 ? sor_omega_opt(n) : p->omega;
  const int inner = p->inner_sweeps > 0 ? p->inner_sweeps : 20;
  const int max_outer = p->max_iters / inner;

  const int bps = exact3_blocks_per_sm<float>(true);
  if (bps < 1) {
    c->set_error("3D phase kernel does not fit on an SM");
    return SOR_ERR_CUDA;
  }
  std::vector<Tile> strips;
  const int bands = build_strips3(L, c->sm_count * bps * kWarpsY, &strips);
  const int flow_grid = c->sm_count * bps, nst = (int)strips.size();
  std::vector<Tile> tiles;
  for (int k = 1; k <= n; ++k)
    for (int r = 0; r < L.row_tiles(); ++r)
      for (int t = 0; t < L.col_tiles(); ++t)
        tiles.push_back(Tile{0, k * m + 1 + r * kTileRows, 1 + t * kWarpCols, std::min(kTileRows, n - r * kTileRows)});
  const int nt = (int)tiles.size();

  const bool stage_u = !in_dev || !out_dev;
  size_t bytes = 2 * elems * (sizeof(double) + 2 * sizeof(float)) + 2 * sizeof(Desc3) + 3 * sizeof(SlotState) +
                 sizeof(Tile) * (nt + nst) + sizeof(unsigned) * (nst + 1) + 1024;
  if (has_f) bytes += 2 * elems * sizeof(double);
  if (stage_u) bytes += ncube * sizeof(double);
  if (has_f && !f_dev) bytes += nf * sizeof(double);
  Buffers3 B;
  B.c = c;
  sor_status rs = ctx_reserve(c, bytes, wait_budget, -1.0);
  if (rs != SOR_OK) {
    c->set_error("3D solve does not fit the device-memory budget");
    return rs;
  }
  B.reserved = bytes;
  double* u64[2] = {(double*)B.get(elems * sizeof(double)), (double*)B.get(elems * sizeof(double))};
  float* dbuf = (float*)B.get(2 * elems * sizeof(float));  // the correction, both colours
  float* rbuf = (float*)B.get(2 * elems * sizeof(float));  // the rounded residual, both colours
  double* g64[2] = {nullptr, nullptr};
  if (has_f) {
    g64[0] = (double*)B.get(elems * sizeof(double));
    g64[1] = (double*)B.get(elems * sizeof(double));
  }
  Desc3* d_desc = (Desc3*)B.get(2 * sizeof(Desc3));  // [0] u (residual, correction), [1] d (inner sweeps)
  SlotState* d_state = (SlotState*)B.get(3 * sizeof(SlotState));  // [0] outer, [1] inner, [2] inner at rest
  Tile* d_tiles = (Tile*)B.get(sizeof(Tile) * nt);
  Tile* d_strips = (Tile*)B.get(sizeof(Tile) * nst);
  unsigned* d_progress = (unsigned*)B.get(sizeof(unsigned) * (nst + 1));
  double* d_u = stage_u ? (double*)B.get(ncube * sizeof(double)) : nullptr;
  double* d_f = (has_f && !f_dev) ? (double*)B.get(nf * sizeof(double)) : nullptr;
  if (!u64[0] || !u64[1] || !dbuf || !rbuf || (has_f && (!g64[0] || !g64[1])) || !d_desc || !d_state ||
      !d_tiles || !d_strips || !d_progress || (stage_u && !d_u) || (has_f && !f_dev && !d_f)) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  float* dcol[2] = {dbuf, dbuf + elems};
  float* rcol[2] = {rbuf, rbuf + elems};

  Desc3 du, dd;
  std::memset(&du, 0, sizeof(du));
  std::memset(&dd, 0, sizeof(dd));
  du.x[0] = u64[0];
  du.x[1] = u64[1];
  du.g[0] = g64[0];
  du.g[1] = g64[1];
  du.g64[0] = g64[0];
  du.g64[1] = g64[1];
  du.n = dd.n = n;
  du.m = dd.m = m;
  du.pitch = dd.pitch = pitch;
  du.tiles = dd.tiles = nt;
  du.K = 1;
  du.max_iters = 1 << 30;
  du.stop = kStopResid;
  du.tol = p->tol;
  du.stall = p->stall_window;
  du.rhs32[0] = rcol[0];
  du.rhs32[1] = rcol[1];
  du.inner = d_state + 1;
  dd.x[0] = dcol[0];
  dd.x[1] = dcol[1];
  dd.g[0] = rcol[0];
  dd.g[1] = rcol[1];
  dd.K = inner;
  dd.max_iters = inner;  // one launch of `inner` iterations; its change test never stops it
  dd.stop = kStopDelta;
  dd.tol = -1.0;
  dd.a32 = (float)(1.0 - w);
  dd.b32 = (float)(w / 6.0);
  dd.a64 = 1.0 - w;
  dd.b64 = w / 6.0;
  dd.ucorr[0] = u64[0];
  dd.ucorr[1] = u64[1];
  dd.outer = d_state;
  SlotState st[3];
  std::memset(st, 0, sizeof(st));
  for (auto& x : st) {
    x.checked_iter = -1;
    x.last_dmax = -1.0;
    x.last_rho = -1.0;
    x.best_rho = HUGE_VAL;
  }
  for (int k = 0; k < 2; ++k) {
    SOR3_CK(c, cudaMemsetAsync(u64[k], 0, elems * sizeof(double), s));
    if (has_f) SOR3_CK(c, cudaMemsetAsync(g64[k], 0, elems * sizeof(double), s));
  }
  SOR3_CK(c, cudaMemsetAsync(dbuf, 0, 2 * elems * sizeof(float), s));
  SOR3_CK(c, cudaMemsetAsync(rbuf, 0, 2 * elems * sizeof(float), s));
  const Desc3 descs[2] = {du, dd};
  SOR3_CK(c, cudaMemcpyAsync(d_desc, descs, sizeof(descs), cudaMemcpyHostToDevice, s));
  SOR3_CK(c, cudaMemcpyAsync(d_state, st, sizeof(st), cudaMemcpyHostToDevice, s));
  SOR3_CK(c, cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, s));
  SOR3_CK(c, cudaMemcpyAsync(d_strips, strips.data(), sizeof(Tile) * nst, cudaMemcpyHostToDevice, s));
  const double* u_src = u0;
  if (!in_dev) {
    SOR3_CK(c, cudaMemcpyAsync(d_u, u0, ncube * sizeof(double), cudaMemcpyHostToDevice, s));
    u_src = d_u;
  }
  const double* f_src = f;
  if (has_f && !f_dev) {
    SOR3_CK(c, cudaMemcpyAsync(d_f, f, nf * sizeof(double), cudaMemcpyHostToDevice, s));
    f_src = d_f;
  }
  const double h = 1.0 / (double)(n + 1);
  const dim3 pgrid((L.qw + kWarpCols - 1) / kWarpCols, m, m);
  k_pack3d<double><<<pgrid, kWarpCols, 0, s>>>(u_src, f_src, n, pitch, h * h, u64[0], u64[1], g64[0], g64[1],
                                               nullptr, nullptr, d_state);
  SOR3_CK(c, cudaGetLastError());

  const int grid = std::min(nt, c->sm_count * 8);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  SOR3_CK(c, cudaEventCreate(&ev0));
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
  for (int k = 0; k < 2; ++k) SOR3_CK(c, cudaEventCreateWithFlags(&pev[k], cudaEventDisableTiming));

  // one outer step: inner state back to rest, d = 0, the residual test (and
  // right side), the inner sweeps, the correction
  auto enqueue_step = [&]() -> sor_status {
    SOR3_CK(c, cudaMemcpyAsync(d_state + 1, d_state + 2, sizeof(SlotState), cudaMemcpyDeviceToDevice, s));
    SOR3_CK(c, cudaMemsetAsync(dbuf, 0, 2 * elems * sizeof(float), s));
    k_resid3d<double, kResidRefine><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
    SOR3_CK(c, cudaGetLastError());
    SOR3_CK(c, cudaMemsetAsync(d_progress, 0, sizeof(unsigned) * (nst + 1), s));
    SOR3_CK(c, launch_3_flow<float>(d_desc + 1, d_state + 1, d_strips, nst, bands, L.col_tiles(), flow_grid,
                                    2 * inner, d_progress, true, s, true));
    return SOR_OK;
  };
  const bool use_graphs = c->opt_graphs.load() != 0;
  if (use_graphs && max_outer > 0) {
    cudaGraph_t gr = nullptr;
    SOR3_CK(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const sor_status es = enqueue_step();
    const cudaError_t ce = cudaStreamEndCapture(s, &gr);
    if (es != SOR_OK) {
      if (gr) cudaGraphDestroy(gr);
      return es;
    }
    SOR3_CK(c, ce);
    const cudaError_t ie = cudaGraphInstantiate(&cl.g, gr, 0);
    cudaGraphDestroy(gr);
    SOR3_CK(c, ie);
  }
  SOR3_CK(c, cudaEventRecord(ev0, s));
  // batches of about a millisecond of steps; the host reads the state after
  // batch b while batch b+1 runs, so the device never waits for the poll
  // (steps queued past convergence only repeat the residual test)
  const double step_s = (double)n * n * n * inner / 4.0e11 + 20e-6;
  const int per_poll = (int)std::max(1.0, std::min(32.0, std::floor(1e-3 / step_s)));
  int planned = 0, batch = 0;
  while (planned < max_outer) {
    if (c->closing.load()) return SOR_ERR_CANCELLED;  // the context is being destroyed
    const int kk = std::min(per_poll, max_outer - planned);
    for (int j = 0; j < kk; ++j) {
      if (use_graphs) {
        SOR3_CK(c, cudaGraphLaunch(cl.g, s));
      } else {
        const sor_status es = enqueue_step();
        if (es != SOR_OK) return es;
      }
    }
    planned += kk;
    SOR3_CK(c, cudaMemcpyAsync(h_state + (batch & 1), d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
    SOR3_CK(c, cudaEventRecord(pev[batch & 1], s));
    if (batch > 0) {  // the previous batch's state
      SOR3_CK(c, cudaEventSynchronize(pev[(batch - 1) & 1]));
      const SlotState& prev = h_state[(batch - 1) & 1];
      if (prev.done || prev.error) break;  // converged, or stalled at the floor
    }
    ++batch;
  }
  // the test after the last correction (a no-op repeat once converged)
  k_resid3d<double, kResidRefine><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
  SOR3_CK(c, cudaGetLastError());
  SOR3_CK(c, cudaEventRecord(ev1, s));
  double* out_dst = out_dev ? u_out : d_u;
  k_unpack3d<double><<<pgrid, kWarpCols, 0, s>>>(u64[0], u64[1], n, pitch, out_dst);
  SOR3_CK(c, cudaGetLastError());
  if (!out_dev) SOR3_CK(c, cudaMemcpyAsync(u_out, d_u, ncube * sizeof(double), cudaMemcpyDeviceToHost, s));
  SlotState fin[2];
  SOR3_CK(c, cudaMemcpyAsync(h_state, d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
  SOR3_CK(c, cudaStreamSynchronize(s));
  fin[0] = h_state[0];
  SOR3_CK(c, cudaMemcpy(&fin[1], d_state + 1, sizeof(SlotState), cudaMemcpyDeviceToHost));
  float ms = 0.0f;
  SOR3_CK(c, cudaEventElapsedTime(&ms, ev0, ev1));
  if (fin[0].error || fin[1].error) {
    c->set_error("device-side consistency check failed");
    return SOR_ERR_INTERNAL;
  }
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->iterations = fin[0].outer * inner;
    res->converged = fin[0].converged;
    res->outer_steps = fin[0].outer;
    res->final_maxdelta = -1.0;
    res->final_resid_rel = fin[0].last_rho;
    res->latency_s = now_s() - t0;
    res->device_s = ms * 1e-3;
  }
  return SOR_OK;
}

}  // namespace

sor_status diag_flow_wait(Ctx* c, int polls, int preset, int* timed_out) {
  if (!timed_out || polls < 1 || polls > kFlowSpins || (preset != 0 && preset != 1)) {
    c->set_error("polls must be in [1, 2^21], preset 0 or 1, timed_out non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  Buffers3 B;
  B.c = c;
  unsigned* buf = (unsigned*)B.get(2 * sizeof(unsigned));
  if (!buf) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  cudaStream_t s = c->stream;
  const unsigned host[2] = {(unsigned)preset, 2u};
  int out = -1;
  SOR3_CK(c, cudaMemcpyAsync(buf, host, sizeof(host), cudaMemcpyHostToDevice, s));
  k_flow_wait_probe<<<1, 32, 0, s>>>(buf, polls, (int*)(buf + 1));
  SOR3_CK(c, cudaGetLastError());
  SOR3_CK(c, cudaMemcpyAsync(&out, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  SOR3_CK(c, cudaStreamSynchronize(s));
  if (out != 0 && out != 1) {
    c->set_error("wait probe did not report");
    return SOR_ERR_INTERNAL;
  }
  *timed_out = out;
  return SOR_OK;
}

sor_status check_params3d(Ctx* c, const sor_params* p, const double* u0, const double* u_out) {
  if (!p || !u0 || !u_out) {
    c->set_error("params, u0 and u_out must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  std::ostringstream why;
  if (p->n < 1 || p->n > kMax3dN) why << "n must be in [1, " << kMax3dN << "]";
  else if (p->precision != SOR_FP64 && p->precision != SOR_FP32 && p->precision != SOR_FP32_REFINE)
    why << "3D solves run in FP64, FP32 or FP32_REFINE";
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
  return SOR_OK;
}

sor_status run_cube(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out, sor_result* res,
                    cudaStream_t s, bool wait_budget) {
  if (p->precision == SOR_FP32_REFINE) return run3d_refine(c, p, u0, f, u_out, res, s, wait_budget);
  return p->precision == SOR_FP64 ? run3d<double>(c, p, u0, f, u_out, res, s, wait_budget)
                                  : run3d<float>(c, p, u0, f, u_out, res, s, wait_budget);
}

// Device bytes a cube solve reserves at most (the sum run3d and run3d_refine
// reserve, taken for the larger of the two and with every staging copy).
size_t cube_bytes(const sor_params* p, bool has_f) {
  const int n = p->n, m = n + 2;
  const Layout L = Layout::make(n);
  const size_t elems = (size_t)m * m * L.pitch;
  const size_t ncube = (size_t)m * m * m, nf = (size_t)n * n * n;
  size_t b = 4 * elems * sizeof(double);      // iterate or solution ping-pong pairs
  b += 4 * elems * sizeof(float);              // correction pair and its right side
  if (has_f) b += 2 * elems * sizeof(double) + nf * sizeof(double);
  b += ncube * sizeof(double);                 // staging
  b += 2 * 2 * ((size_t)m * L.pitch * 4 + (size_t)m * m * 4) * sizeof(double);  // shells
  b += (size_t)64 << 20;                       // tile, strip and phase tables, counters
  return b;
}

sor_status solve3d_blocking(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                            sor_result* res) {
  NvtxRange nvtx("sor_solve3d");
  const sor_status rs = check_params3d(c, p, u0, u_out);
  if (rs != SOR_OK) return rs;
  return run_cube(c, p, u0, f, u_out, res, c->stream, false);
}

}  // namespace sorgb
