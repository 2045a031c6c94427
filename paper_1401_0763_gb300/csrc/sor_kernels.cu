// Red-black SOR kernels for sm_103a (GB300).
//
//   k_pack / k_unpack     natural (N+2)^2 <-> colour-split storage, h^2 f, ||b~||_inf
//   k_sweep<T>            one colour phase (Section 3.1, Algorithm 1 updateGridRed /
//                         updateGridBlack) over a list of tiles of one or many slots,
//                         with the fused max|change| reduction (Section 2.1,
//                         Section 3.3) and the per-iteration bookkeeping of Algorithm 1
//   k_sweep_fast64        FP64 phase with shared neighbour pair sums and rescaled
//                         unknowns (fewer FP64 instructions per update)
//   k_resid<T>            scaled residual r~ = h^2 f + sum_nb(u) - 4u in FP64 with
//                         the relative-residual test and, for defect correction,
//                         u += d fused in
//
// Arithmetic: k_sweep and k_resid evaluate every expression in the order
//   (1-w)*u + (w/4)*(((N+S)+(W+E))+g)   and   (g + ((N+S)+(W+E))) - 4u
// with each product and sum rounded on its own (__fmul_rn / __fadd_rn and the
// FP64 forms), so their results do not depend on compiler contraction.
#include <cuda_runtime.h>

#include <cstring>

#include "sor_bits.cuh"
#include "sor_device.cuh"
#include "sor_devfn.cuh"
#include "sor_kernels.h"

namespace sorgb {

// Kernel launches issued by this host thread (statistics; captured launches
// are counted once at capture, their replays by the runtime).
static thread_local unsigned long long t_launches = 0;
unsigned long long kernel_launch_count() { return t_launches; }
void count_kernel_launches(int k) { t_launches += (unsigned long long)k; }

// ------------------------------------------------------------------------------------------------
// pack / unpack
// ------------------------------------------------------------------------------------------------

// Thread (i, q) moves the natural cells j = 2q-1 and j = 2q of row i (one of
// each colour) into the colour arrays; interior cells also receive h^2 f and
// contribute |b~| = |h^2 f + (ring neighbours)| to ||b~||_inf.  The largest
// |u0| and |h^2 f| are reduced as well: they bound the values the rescaled
// FP64 phases carry, whose chunk length the host derives from them.
template <typename T>
__global__ void k_pack(const double* __restrict__ u0, const double* __restrict__ f, int n, int pitch, double h2,
                       T* x00, T* x01, T* x10, T* x11, T* g0, T* g1, double* g64_0, double* g64_1,
                       double* u00, double* u01, double* u10, double* u11, SlotState* st) {
  __shared__ unsigned long long red[kWarpsY];
  const int m = n + 2;
  const int qw = (n + 1) / 2 + 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  unsigned long long bb = 0, ub = 0, gb = 0;
  if (q < qw) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int j = 2 * q - 1 + t;
      if (j < 0 || j >= m) continue;
      const int c = (i + j) & 1;
      if (!dbg_range((long long)i * m + j, (long long)i * m + j + 1, (long long)m * m, st) ||
          !dbg_range((long long)eidx(i, q, pitch), (long long)eidx(i, q, pitch) + 1, (long long)m * pitch, st))
        continue;
      const double v = u0[(size_t)i * m + j];
      ub = umax64(ub, abs_bits(v));
      const size_t e = eidx(i, q, pitch);
      T* xa = c ? x01 : x00;
      T* xb = c ? x11 : x10;
      if (xa) xa[e] = (T)v;
      if (xb) xb[e] = (T)v;
      double* ua = c ? u01 : u00;
      double* ub = c ? u11 : u10;
      if (ua) ua[e] = v;
      if (ub) ub[e] = v;
      const bool interior = (i >= 1 && i <= n && j >= 1 && j <= n);
      double gij = 0.0;
      if (interior && f) gij = __dmul_rn(h2, f[(size_t)(i - 1) * n + (j - 1)]);
      gb = umax64(gb, abs_bits(gij));
      T* gg = c ? g1 : g0;
      if (gg) gg[e] = (T)gij;
      double* g6 = c ? g64_1 : g64_0;
      if (g6) g6[e] = gij;
      if (interior) {
        // b~ = g + ring neighbours, summed in the order N, S, W, E
        double bnd = 0.0;
        if (i == 1) bnd = __dadd_rn(bnd, u0[(size_t)0 * m + j]);
        if (i == n) bnd = __dadd_rn(bnd, u0[(size_t)(n + 1) * m + j]);
        if (j == 1) bnd = __dadd_rn(bnd, u0[(size_t)i * m + 0]);
        if (j == n) bnd = __dadd_rn(bnd, u0[(size_t)i * m + (n + 1)]);
        bb = umax64(bb, abs_bits(__dadd_rn(gij, bnd)));
      }
    }
  }
  block_max_to(bb, &st->bmax_bits, red);
  block_max_to(ub, &st->umax_bits, red);
  block_max_to(gb, &st->gmax_bits, red);
}

// Inverse of k_pack for the iterate in colour arrays c0 / c1 (type T).
template <typename T>
__global__ void k_unpack(const T* __restrict__ c0, const T* __restrict__ c1, int n, int pitch,
                         double* __restrict__ out) {
  const int m = n + 2;
  const int qw = (n + 1) / 2 + 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (q >= qw) return;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int j = 2 * q - 1 + t;
    if (j < 0 || j >= m) continue;
    const int c = (i + j) & 1;
    out[(size_t)i * m + j] = (double)(c ? c1 : c0)[eidx(i, q, pitch)];
  }
}

// ------------------------------------------------------------------------------------------------
// one colour phase, exact operation order
// ------------------------------------------------------------------------------------------------

// Per-slot decisions taken once per tile by thread 0.
struct TileCtl {
  int skip, k, measure, xbuf;
};

// Rows [i0, i1) of one warp's share of a tile for k_sweep (one colour phase,
// exact operation order).  MEASURE: also return max |change| (as the bits of
// a non-negative double); a compile-time flag so that no |change| work is
// issued on the iterations that do not test it.
template <typename T, int MODE, bool MEASURE, bool HAS_G>
__device__ __forceinline__ unsigned long long sweep_rows(T* __restrict__ X, const T* __restrict__ O,
                                                         const T* __restrict__ G, T a, T b, int pitch, int n,
                                                         int colour, int q0, int i0, int i1, int lane, bool zero_all,
                                                         bool zero_own) {
  unsigned long long dm = 0;
  unsigned dm32 = 0;
  if (i0 < i1) {
    T om[4], oc[4], op[4];
    if (zero_all) {
#pragma unroll
      for (int v = 0; v < 4; ++v) { om[v] = T(0); oc[v] = T(0); }
    } else {
      load4(O + eidx(i0 - 1, q0, pitch), om);
      load4(O + eidx(i0, q0, pitch), oc);
    }
    for (int i = i0; i < i1; ++i) {
      T own[4], gv[4];
      if (zero_all) {
#pragma unroll
        for (int v = 0; v < 4; ++v) op[v] = T(0);
      } else {
        load4(O + eidx(i + 1, q0, pitch), op);
      }
      if (zero_own) {
#pragma unroll
        for (int v = 0; v < 4; ++v) own[v] = T(0);
      } else {
        load4(X + eidx(i, q0, pitch), own);
      }
      if (HAS_G) load4(G + eidx(i, q0, pitch), gv);
      T left = __shfl_up_sync(0xffffffffu, oc[3], 1);
      T right = __shfl_down_sync(0xffffffffu, oc[0], 1);
      if (!zero_all) {
        if (lane == 0) left = O[eidx(i, q0 - 1, pitch)];
        if (lane == 31) right = O[eidx(i, q0 + kVec, pitch)];
      } else {
        left = T(0); right = T(0);
      }
      const int s = (i + colour) & 1;
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
      bool all_in = true;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        T sum = radd(radd(om[v], op[v]), radd(W[v], E[v]));
        if (HAS_G) sum = radd(sum, gv[v]);
        const T nu = radd(rmul(a, own[v]), rmul(b, sum));
        const bool in = (q0 + v) <= qlim;
        all_in = all_in && in;
        nv[v] = in ? nu : own[v];
        if (MEASURE && in) {
          if (sizeof(T) == 4)
            dm32 = max(dm32, abs_bits32((float)radd(nu, -own[v])));
          else
            dm = umax64(dm, abs_bits((double)radd(nu, -own[v])));
        }
      }
      if (all_in) {
        store4(X + eidx(i, q0, pitch), nv);
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if ((q0 + v) <= qlim) X[eidx(i, q0 + v, pitch)] = nv[v];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) { om[v] = oc[v]; oc[v] = op[v]; }
    }
  }
  if (sizeof(T) == 4 && MEASURE) dm = abs_bits_of(__uint_as_float(dm32));
  return dm;
}

// MODE 0: plain iteration on x (type T) with optional rhs g (type T).
// MODE 1: inner sweep of defect correction on d (FP32) with rhs r~ (FP32);
//         `sweep` is the index of this iteration within the correction; at
//         sweep 0 the correction starts from d = 0.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_sweep(const SlotDesc* __restrict__ slots, SlotState* states,
                                                    const Tile* __restrict__ tiles, int ntiles, int colour,
                                                    int sweep) {
  __shared__ unsigned long long red[kWarpsY];
  __shared__ TileCtl ctl;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const SlotDesc& sd = slots[tl.slot];
    SlotState* st = states + tl.slot;
    if (threadIdx.x == 0) {
      TileCtl c;
      c.skip = *((volatile int*)&st->done);
      if (MODE == 1 && sweep >= sd.inner) c.skip = 1;
      c.k = *((volatile int*)&st->iters) + 1;
      c.measure = (MODE == 0) && (((c.k % sd.K) == 0) || (c.k >= sd.max_iters));
      c.xbuf = (MODE == 0) ? *((volatile int*)&st->xbuf) : 0;
      if (!dbg_tile(sd, st, tl.row0 - 1, tl.row0 + tl.nrows + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1)) c.skip = 1;
      ctl = c;
    }
    __syncthreads();
    const TileCtl c = ctl;
    __syncthreads();
    if (c.skip) continue;

    const int pitch = sd.pitch, n = sd.n;
    T* X = (T*)sd.x[c.xbuf][colour];
    const T* O = (const T*)sd.x[c.xbuf][colour ^ 1];
    const T* G = (const T*)sd.g[colour];
    T a, b;
    if (sizeof(T) == 4) { a = (T)sd.a32; b = (T)sd.b32; } else { a = (T)sd.a64; b = (T)sd.b64; }
    const bool zero_all = (MODE == 1) && sweep == 0 && colour == 0;  // d = 0 before the first red phase
    const bool zero_own = (MODE == 1) && sweep == 0;                // black cells still 0 in the first black phase

    const int q0 = tl.col0 + lane * kVec;
    const int rows_per_warp = (tl.nrows + kWarpsY - 1) / kWarpsY;
    const int i0 = tl.row0 + wy * rows_per_warp;
    const int i1 = min(i0 + rows_per_warp, tl.row0 + tl.nrows);
    unsigned long long dm = 0;
    // the source term is a compile-time choice: as a runtime test the compiler
    // issues its addition speculatively, one more FP64 operation per cell
    if (MODE == 0 && c.measure) {
      dm = G ? sweep_rows<T, MODE, true, true>(X, O, G, a, b, pitch, n, colour, q0, i0, i1, lane, zero_all, zero_own)
             : sweep_rows<T, MODE, true, false>(X, O, G, a, b, pitch, n, colour, q0, i0, i1, lane, zero_all,
                                                zero_own);
    } else if (G) {
      (void)sweep_rows<T, MODE, false, true>(X, O, G, a, b, pitch, n, colour, q0, i0, i1, lane, zero_all, zero_own);
    } else {
      (void)sweep_rows<T, MODE, false, false>(X, O, G, a, b, pitch, n, colour, q0, i0, i1, lane, zero_all,
                                              zero_own);
    }
    if (MODE == 0) {
      if (c.measure) block_max_to(dm, &st->dmax_bits, red);
      if (colour == 1) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
          const unsigned prev = atomicAdd(&st->arrive, 1u);
          if (prev == (unsigned)sd.sweep_tiles - 1u) {
            __threadfence();
            finalize_plain(sd, st, c.k, c.measure);
          }
        }
        __syncthreads();
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// one colour phase in FP64 with fewer FP64 instructions per update
// ------------------------------------------------------------------------------------------------
//
// GB300 issues FP64 at about 1/64 of its FP32 rate, so this phase is bound by
// FP64 instruction issue, not by HBM.  Two reformulations of the same update
// cut the FP64 instructions from 6 to about 3.1 per cell (no sources):
//
// (a) Shared pair sums.  With s = (i + c) & 1 the four neighbours of (i, q)
//     split into an upper-left pair DU(i,q) = N + W and a lower-right pair
//     DL(i,q) = E + S, and DU(i+1, q) = DL(i, q + s_i - 1): walking down a
//     column strip, each pair sum is formed once and used by two cells, so the
//     neighbour sum costs 2 additions instead of 3.
// (b) Rescaled unknowns inside a chunk of L iterations.  Red values after the
//     red phase of iteration t of the chunk are carried as a_t * u with
//     a_t = (w/4)^-(2t-1), black values as b_t * u with b_t = (w/4)^-2t.  Then
//     both phases read  X' = alpha * X + (sum of the four neighbours)  with
//     alpha = (1-w)/(w/4)^2 (one FMA), and the sources enter as gamma * g.
//     The first red phase starts from unscaled values and the last iteration
//     of the chunk returns to unscaled values (X' = alpha X + beta Sigma),
//     so between chunks -- where convergence is tested, max|change| measured
//     and the result read -- the arrays hold u itself.
//     The Dirichlet ring cells must be read at the scale of their colour in
//     each phase.  The phase that updates colour c (and never reads colour
//     c's ring) rewrites colour c's ring cells as (unscaled value) x (the scale
//     the next phase reads colour c at), from a copy saved after packing; the
//     last phases of a chunk write scale 1, so between chunks the ring is
//     unscaled again.  Readers never rescale, and every strip does the same
//     work per row.
// Every cell's expression depends only on its own neighbours and the launch
// constants, never on the tiling, so results are reproducible bit for bit
// across tile shapes and batch compositions.
struct FastPhase {
  double alpha, beta, gamma, dscale;
  double nscale;  // scale at which the next phase reads this phase's colour: this phase writes its
                  // colour's Dirichlet ring cells as (unscaled value) x nscale
  int last;       // this phase belongs to the last iteration of its chunk (values unscaled after it)
};

// Register state of one warp walking down a strip of rows: the neighbour-colour
// rows i-1 and i, the lower-right pair sums of the previous row, and the
// strip-edge pairs of the coming parity-1 rows (below).
struct FastWalk {
  double om[4], oc[4], dlp[4];
  double edge;  // lane r: the edge pair of the r-th parity-1 row of the current group
  int ek;       // parity-1 rows of the group already taken
};

// In a parity-1 row, lane 0's upper-left pair N + W = O[i-1][col0] +
// O[i][col0-1] reaches one column left of the strip, past what the previous
// row formed.  Formed row by row it cost a whole warp instruction on the FP64
// pipe (predicating it to one lane costs the same), 1 of 25 per row pair.  So
// the pairs of 32 parity-1 rows i, i+2, ... are formed together, lane r taking
// row i + 2r, and each row takes its value by a shuffle.
__device__ __forceinline__ void fast_edges(FastWalk& w, const double* __restrict__ O, int pitch, int col0, int i,
                                           int i1, int lane) {
  const int r = i + 2 * lane;
  double e = 0.0;
  if (r < i1) e = __dadd_rn(O[eidx(r - 1, col0, pitch)], O[eidx(r, col0 - 1, pitch)]);
  w.edge = e;
  w.ek = 0;
}
// The edge pair of parity-1 row i (rows taken in order; a new group at every
// 32nd).
__device__ __forceinline__ double fast_edge(FastWalk& w, const double* __restrict__ O, int pitch, int q0, int i,
                                            int i1, int lane) {
  if (w.ek == 32) fast_edges(w, O, pitch, q0 - lane * kVec, i, i1, lane);
  const double e = __shfl_sync(0xffffffffu, w.edge, w.ek);
  ++w.ek;
  return e;
}

// Rows are staged through shared memory by asynchronous copies issued
// kFastAhead rows ahead (a per-warp pipeline), so the loads' latency leaves
// the critical path without holding registers.  A stage holds, for row i: the
// neighbour-colour row i+1, the own row i, the source row i and the two
// strip-edge neighbours O[i][q0-1] (lane 0) and O[i][q0+4] (lane 31).  Each
// lane reads back only what it copied itself, so the pipeline needs no
// synchronisation beyond each thread's own wait_group.  A buffer is refilled
// kFastStages - kFastAhead = 2 rows after it was read: by then every value
// read from it has fed an instruction that already issued, so the refill
// cannot overtake the read.
constexpr int kFastStages = 6;
constexpr int kFastAhead = 4;

template <bool HAS_G>
struct FastStage {
  double op[32 * kVec];
  double own[32 * kVec];
  double g[HAS_G ? 32 * kVec : 2];
  double edge[2];
};

template <bool HAS_G>
constexpr size_t fast_smem_bytes() {
  return (size_t)kWarpsY * kFastStages * sizeof(FastStage<HAS_G>);
}

// 16-byte asynchronous copy; nbytes 0 copies nothing and zero-fills.
__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gsrc, int nbytes) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gsrc), "r"(nbytes) : "memory");
}
// 8-byte asynchronous copy by the lanes with pred set (nbytes as above).
__device__ __forceinline__ void cp_async_8_if(void* smem_dst, const void* gsrc, int nbytes, bool pred) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n @p cp.async.ca.shared.global [%0], [%1], 8, %2;\n}\n" ::"r"(saddr),
      "l"(gsrc), "r"(nbytes), "r"((int)pred)
      : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Issue the copies of row i into a stage (zero-fill, no global read, when
// !valid) and close the group, so every row accounts for exactly one group.
template <bool HAS_G>
__device__ __forceinline__ void fast_issue(FastStage<HAS_G>* st, int i, bool valid, const double* __restrict__ O,
                                           const double* __restrict__ X, const double* __restrict__ G, int pitch,
                                           int q0, int lane) {
  const int nb = valid ? 16 : 0;
  const double* o = valid ? O + eidx(i + 1, q0, pitch) : O;
  const double* x = valid ? X + eidx(i, q0, pitch) : X;
  cp_async_16(st->op + lane * kVec, o, nb);
  cp_async_16(st->op + lane * kVec + 2, o + 2, nb);
  cp_async_16(st->own + lane * kVec, x, nb);
  cp_async_16(st->own + lane * kVec + 2, x + 2, nb);
  if (HAS_G) {
    const double* gp = valid ? G + eidx(i, q0, pitch) : G;
    cp_async_16(st->g + lane * kVec, gp, nb);
    cp_async_16(st->g + lane * kVec + 2, gp + 2, nb);
  }
  const bool right = lane == 31;
  const double* e = valid ? O + eidx(i, right ? q0 + kVec : q0 - 1, pitch) : O;
  cp_async_8_if(&st->edge[right ? 1 : 0], e, valid ? 8 : 0, lane == 0 || right);
  cp_async_commit();
}

// One staged row as this lane reads it back.
struct FastIn {
  double op[4], own[4], g[4], el, er;
};

template <bool HAS_G>
__device__ __forceinline__ void fast_read(const FastStage<HAS_G>* st, int lane, FastIn& r) {
  load4(st->op + lane * kVec, r.op);
  load4(st->own + lane * kVec, r.own);
  if (HAS_G) load4(st->g + lane * kVec, r.g);
  r.el = st->edge[0];
  r.er = st->edge[1];
}

// The cells of one row (parity S = (i + colour) & 1, known at compile time,
// which fixes where W / E come from and how the upper-left pair sums follow
// from the previous row's lower-right ones: S == 0 -> the same columns;
// S == 1 -> one column to the left, a shuffle, lane 0 forming the strip-edge
// pair itself).  om / oc: neighbour-colour rows i-1 / i; dlp: lower-right pair
// sums of row i-1; op: neighbour-colour row i+1 (ring values already scaled).
// FIRST: no previous row, form the upper-left pairs directly.  Ring values
// arrive already at the phase's scale.  Pure register work: the caller loads
// and stores, so two rows can be scheduled together.
template <bool UNIT_BETA, bool HAS_G, bool MEASURE, int S, bool FIRST, bool FULL>
__device__ __forceinline__ void fast_cells(const double (&om)[4], const double (&oc)[4], const double (&dlp)[4],
                                           const double (&op)[4], const FastIn& in, int n, int q0, int lane,
                                           const FastPhase& ph, double (&nv)[4], double (&DL)[4],
                                           unsigned long long& dm, double e0) {
  double left = __shfl_up_sync(0xffffffffu, oc[3], 1);
  double right = __shfl_down_sync(0xffffffffu, oc[0], 1);
  if (lane == 0) left = in.el;
  if (lane == 31) right = in.er;
  double W[4], E[4];
  if (S == 0) {
    W[0] = oc[0]; W[1] = oc[1]; W[2] = oc[2]; W[3] = oc[3];
    E[0] = oc[1]; E[1] = oc[2]; E[2] = oc[3]; E[3] = right;
  } else {
    W[0] = left; W[1] = oc[0]; W[2] = oc[1]; W[3] = oc[2];
    E[0] = oc[0]; E[1] = oc[1]; E[2] = oc[2]; E[3] = oc[3];
  }
  double DU[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) DL[v] = __dadd_rn(E[v], op[v]);
  if (FIRST) {
#pragma unroll
    for (int v = 0; v < 4; ++v) DU[v] = __dadd_rn(om[v], W[v]);
  } else if (S == 0) {  // previous row had s = 1: same columns
#pragma unroll
    for (int v = 0; v < 4; ++v) DU[v] = dlp[v];
  } else {  // previous row had s = 0: one column to the left
    double d0 = __shfl_up_sync(0xffffffffu, dlp[3], 1);
    if (lane == 0) d0 = e0;  // om[0] + left, formed with the strip's other edge pairs
    DU[0] = d0; DU[1] = dlp[0]; DU[2] = dlp[1]; DU[3] = dlp[2];
  }
  const int qlim = (n + S) >> 1;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double sum = __dadd_rn(DU[v], DL[v]);
    double t2;
    if (UNIT_BETA)
      t2 = HAS_G ? __fma_rn(ph.gamma, in.g[v], sum) : sum;
    else
      t2 = HAS_G ? __fma_rn(ph.gamma, in.g[v], __dmul_rn(ph.beta, sum)) : __dmul_rn(ph.beta, sum);
    const double nu = __fma_rn(ph.alpha, in.own[v], t2);
    const bool inside = FULL || (q0 + v) <= qlim;
    // cells past the interior (the ring cell, padding) keep their value; the
    // whole vector is written back, so no other lane's or warp's cell is touched
    nv[v] = inside ? nu : in.own[v];
    if (MEASURE && inside) dm = umax64(dm, abs_bits(__fma_rn(-ph.dscale, in.own[v], nu)));
  }
}

__device__ __forceinline__ int wrap_stage(int b) { return b >= kFastStages ? b - kFastStages : b; }

// One row i in buffer b.
template <bool UNIT_BETA, bool HAS_G, bool MEASURE, bool FULL, int S, bool FIRST>
__device__ __forceinline__ void fast_step1(FastWalk& w, int i, int& b, FastStage<HAS_G>* stages, int i1,
                                           const double* __restrict__ O, double* __restrict__ X,
                                           const double* __restrict__ G, int pitch, int n, int q0, int lane,
                                           const FastPhase& ph, unsigned long long& dm) {
  cp_async_wait<kFastAhead - 1>();  // rows up to i + 3 are in flight: row i has landed
  FastIn a;
  fast_read<HAS_G>(stages + b, lane, a);
  double nv[4], DL[4];
  const double e0 = (S == 1 && !FIRST) ? fast_edge(w, O, pitch, q0, i, i1, lane) : 0.0;
  fast_cells<UNIT_BETA, HAS_G, MEASURE, S, FIRST, FULL>(w.om, w.oc, w.dlp, a.op, a, n, q0, lane, ph, nv, DL, dm, e0);
  fast_issue<HAS_G>(stages + wrap_stage(b + kFastAhead), i + kFastAhead, i + kFastAhead < i1, O, X, G, pitch, q0,
                    lane);
  store4(X + eidx(i, q0, pitch), nv);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    w.dlp[v] = DL[v];
    w.om[v] = w.oc[v];
    w.oc[v] = a.op[v];
  }
  b = wrap_stage(b + 1);
}

// Rows i (parity S) and i + 1 (parity 1 - S); both rows' arithmetic is
// independent enough to be interleaved, which doubles the FP64 work in flight
// per warp.
template <bool UNIT_BETA, bool HAS_G, bool MEASURE, bool FULL, int S>
__device__ __forceinline__ void fast_step2(FastWalk& w, int i, int& b, FastStage<HAS_G>* stages, int i1,
                                           const double* __restrict__ O, double* __restrict__ X,
                                           const double* __restrict__ G, int pitch, int n, int q0, int lane,
                                           const FastPhase& ph, unsigned long long& dm) {
  cp_async_wait<kFastAhead - 2>();  // rows i and i + 1 have landed
  FastIn a, c;
  fast_read<HAS_G>(stages + b, lane, a);
  fast_read<HAS_G>(stages + wrap_stage(b + 1), lane, c);
  double nva[4], DLa[4], nvc[4], DLc[4];
  const double e0 = fast_edge(w, O, pitch, q0, S == 1 ? i : i + 1, i1, lane);  // the pair's parity-1 row
  fast_cells<UNIT_BETA, HAS_G, MEASURE, S, false, FULL>(w.om, w.oc, w.dlp, a.op, a, n, q0, lane, ph, nva, DLa, dm,
                                                        e0);
  fast_cells<UNIT_BETA, HAS_G, MEASURE, 1 - S, false, FULL>(w.oc, a.op, DLa, c.op, c, n, q0, lane, ph, nvc, DLc, dm,
                                                            e0);
  fast_issue<HAS_G>(stages + wrap_stage(b + kFastAhead), i + kFastAhead, i + kFastAhead < i1, O, X, G, pitch, q0,
                    lane);
  fast_issue<HAS_G>(stages + wrap_stage(b + kFastAhead + 1), i + kFastAhead + 1, i + kFastAhead + 1 < i1, O, X, G,
                    pitch, q0, lane);
  store4(X + eidx(i, q0, pitch), nva);
  store4(X + eidx(i + 1, q0, pitch), nvc);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    w.dlp[v] = DLc[v];
    w.om[v] = a.op[v];
    w.oc[v] = c.op[v];
  }
  b = wrap_stage(b + 2);
}

// Rows [i0, i1) of one strip: the first row, then pairs (whose first row has
// the parity of i0 + 1, fixed at compile time) and an odd row left over.
template <bool UNIT_BETA, bool HAS_G, bool MEASURE, bool FULL, int S0>
__device__ __forceinline__ void fast_rows(FastWalk& w, FastStage<HAS_G>* stages, const double* __restrict__ O,
                                          double* __restrict__ X, const double* __restrict__ G, int pitch, int n,
                                          int q0, int i0, int i1, int lane, const FastPhase& ph,
                                          unsigned long long& dm) {
  int i = i0, b = 0;
  fast_step1<UNIT_BETA, HAS_G, MEASURE, FULL, S0, true>(w, i, b, stages, i1, O, X, G, pitch, n, q0, lane, ph, dm);
  ++i;
  for (; i + 1 < i1; i += 2)
    fast_step2<UNIT_BETA, HAS_G, MEASURE, FULL, 1 - S0>(w, i, b, stages, i1, O, X, G, pitch, n, q0, lane, ph, dm);
  if (i < i1)
    fast_step1<UNIT_BETA, HAS_G, MEASURE, FULL, 1 - S0, false>(w, i, b, stages, i1, O, X, G, pitch, n, q0, lane, ph,
                                                               dm);
}

template <bool UNIT_BETA, bool HAS_G, bool MEASURE, bool FULL = false>
__device__ __forceinline__ unsigned long long fast_walk(FastStage<HAS_G>* stages, const double* __restrict__ O,
                                                        double* __restrict__ X, const double* __restrict__ G,
                                                        int pitch, int n, int colour, int q0, int i0, int i1,
                                                        int lane, const FastPhase& ph) {
  for (int k = 0; k < kFastAhead; ++k)  // prologue: rows i0 .. i0 + kFastAhead - 1 into buffers 0 ..
    fast_issue<HAS_G>(stages + k, i0 + k, i0 + k < i1, O, X, G, pitch, q0, lane);
  FastWalk w;
  load4(O + eidx(i0 - 1, q0, pitch), w.om);
  load4(O + eidx(i0, q0, pitch), w.oc);
#pragma unroll
  for (int v = 0; v < 4; ++v) w.dlp[v] = 0.0;
  // the edge pairs of the first 32 parity-1 rows after the first row
  fast_edges(w, O, pitch, q0 - lane * kVec, ((i0 + 1 + colour) & 1) ? i0 + 1 : i0 + 2, i1, lane);
  unsigned long long dm = 0;
  if (i0 < i1) {
    if (((i0 + colour) & 1) == 0)
      fast_rows<UNIT_BETA, HAS_G, MEASURE, FULL, 0>(w, stages, O, X, G, pitch, n, q0, i0, i1, lane, ph, dm);
    else
      fast_rows<UNIT_BETA, HAS_G, MEASURE, FULL, 1>(w, stages, O, X, G, pitch, n, q0, i0, i1, lane, ph, dm);
  }
  cp_async_wait<0>();  // no copy may still target the stages when the warp moves on
  return dm;
}

// This phase's colour X: rewrite the Dirichlet ring cells next to the strip
// (ring rows 0 / N+1 above / below its columns, the column q = 0 and the east
// ring column beside its rows) as (unscaled value) x ph.nscale, the scale at
// which the next phase reads this colour.  Row stores of the strip may have
// written the same cells back unchanged just before; the warp barrier orders
// them.  Cells that hold no ring value in a given row (the other parity's
// padding) receive the saved padding value times the scale and are never read.
__device__ __forceinline__ void fast_ring(const SlotDesc& sd, double* __restrict__ X, int colour, const Tile& tl,
                                          int q0, int lane, double ns) {
  const int n = sd.n, pitch = sd.pitch, m = n + 2;
  const double* __restrict__ R = sd.ring[colour];
  __syncwarp();
  if (tl.row0 == 1) {  // ring row 0 above the strip's columns
    double v[4];
    load4(R + q0 + kOff, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __dmul_rn(v[k], ns);
    store4(X + eidx(0, q0, pitch), v);
  }
  if (tl.row0 + tl.nrows == n + 1) {  // ring row N+1 below them
    double v[4];
    load4(R + pitch + q0 + kOff, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __dmul_rn(v[k], ns);
    store4(X + eidx(n + 1, q0, pitch), v);
  }
  const bool west = tl.col0 == 1, east = tl.col0 + kWarpCols > ((n + 1) >> 1);
  if (west || east) {
    for (int r = tl.row0 + lane; r < tl.row0 + tl.nrows; r += 32) {
      if (west) X[eidx(r, 0, pitch)] = __dmul_rn(R[2 * pitch + r], ns);
      if (east) X[eidx(r, ((n + ((r + colour) & 1)) >> 1) + 1, pitch)] = __dmul_rn(R[2 * pitch + m + r], ns);
    }
  }
}

// Warp-per-strip kernel: each warp walks one strip (slot, first row, first
// packed column, rows) of 128 packed columns; a persistent grid strides over
// a strip table cut so that every warp gets the same number of rows.
template <bool UNIT_BETA, bool HAS_G>
__global__ void __launch_bounds__(kThreads, 3) k_sweep_fast(const SlotDesc* __restrict__ slots, SlotState* states,
                                                            const Tile* __restrict__ strips, int nstrips, int colour,
                                                            FastPhase ph) {
  extern __shared__ __align__(16) unsigned char fast_smem[];
  const int lane = threadIdx.x & 31;
  FastStage<HAS_G>* stages = reinterpret_cast<FastStage<HAS_G>*>(fast_smem) + (threadIdx.x >> 5) * kFastStages;
  const int warp = blockIdx.x * kWarpsY + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * kWarpsY;
  for (int t = warp; t < nstrips; t += nwarps) {
    const Tile tl = strips[t];
    const SlotDesc& sd = slots[tl.slot];
    SlotState* st = states + tl.slot;
    int skip = 0, k = 0, measure = 0, xbuf = 0;
    if (lane == 0) {
      skip = *((volatile int*)&st->done);
      k = *((volatile int*)&st->iters) + 1;
      measure = ((k % sd.K) == 0) || (k >= sd.max_iters);
      xbuf = *((volatile int*)&st->xbuf);
      if (!skip && measure && !ph.last) {  // the host plan must end chunks at measured iterations
        st->error = 1;
        st->done = 1;
        skip = 1;
      }
      if (!skip && !dbg_tile(sd, st, tl.row0 - 1, tl.row0 + tl.nrows + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1))
        skip = 1;
    }
    skip = __shfl_sync(0xffffffffu, skip, 0);
    if (skip) continue;
    k = __shfl_sync(0xffffffffu, k, 0);
    measure = __shfl_sync(0xffffffffu, measure, 0);
    xbuf = __shfl_sync(0xffffffffu, xbuf, 0);

    const int pitch = sd.pitch, n = sd.n;
    double* X = (double*)sd.x[xbuf][colour];
    const double* O = (const double*)sd.x[xbuf][colour ^ 1];
    const double* G = (const double*)sd.g[colour];
    const int q0 = tl.col0 + lane * kVec;
    const int i0 = tl.row0, i1 = tl.row0 + tl.nrows;
    unsigned long long dm;
    if (measure) {
      dm = fast_walk<UNIT_BETA, HAS_G, true>(stages, O, X, G, pitch, n, colour, q0, i0, i1, lane, ph);
      dm = warp_max64(dm);
      if (lane == 0 && dm) atomicMax(&st->dmax_bits, dm);
    } else {
      dm = fast_walk<UNIT_BETA, HAS_G, false>(stages, O, X, G, pitch, n, colour, q0, i0, i1, lane, ph);
    }
    fast_ring(sd, X, colour, tl, q0, lane, ph.nscale);
    if (colour == 1) {
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        if (prev == (unsigned)sd.sweep_tiles - 1u) {
          __threadfence();
          finalize_plain(sd, st, k, measure);
        }
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------------------------------------
// a whole chunk of FP64 phases in one launch
// ------------------------------------------------------------------------------------------------
//
// The per-phase launches above pay a grid start and a drain per colour phase
// (about 8 % of a 4096^2 phase).  k_fast_chain runs the 2L phases of a chunk
// in one cooperative launch (all warps resident): each warp walks its strip
// phase after phase, and before phase p it waits until the strips above,
// below, left and right of it -- the only ones whose cells its stencil reads
// or whose readers it could overwrite -- have finished phase p-1.  A strip
// publishes its progress with a release store after fencing its writes; every
// lane of a waiting warp reads the counters with acquire loads.  Every wait
// is bounded: past kChainSpins polls the warp records an error in the slot
// state, marks it done and returns (the host reports SOR_ERR_INTERNAL).

constexpr int kChainSpins = 1 << 21;  // polls of about 0.1 us each: far above any phase

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until every listed neighbour has completed `target` phases; false on
// timeout.  Lanes 0..3 poll one neighbour each; afterwards every lane takes
// its own acquire of all of them, so its later loads see their writes.
__device__ __forceinline__ bool chain_wait(const unsigned* progress, const int (&nb)[4], unsigned target, int lane) {
  bool ok = true;
  const int mine = lane == 0 ? nb[0] : lane == 1 ? nb[1] : lane == 2 ? nb[2] : lane == 3 ? nb[3] : -1;
  if (mine >= 0) {
    int spins = 0;
    while (ld_acquire_u32(progress + mine) < target) {
      if (++spins > kChainSpins) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
  }
  ok = __all_sync(0xffffffffu, ok);
  if (ok) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (nb[k] >= 0) (void)ld_acquire_u32(progress + nb[k]);
  }
  return ok;
}

template <bool HAS_G>
__global__ void __launch_bounds__(kThreads, 3) k_fast_chain(const SlotDesc* __restrict__ slots, SlotState* states,
                                                            const Tile* __restrict__ strips, int nstrips, int ct,
                                                            const FastPhase* __restrict__ phases, int nphases,
                                                            unsigned* progress) {
  extern __shared__ __align__(16) unsigned char fast_smem[];
  const int lane = threadIdx.x & 31;
  FastStage<HAS_G>* stages = reinterpret_cast<FastStage<HAS_G>*>(fast_smem) + (threadIdx.x >> 5) * kFastStages;
  const int t = blockIdx.x * kWarpsY + (threadIdx.x >> 5);
  if (t >= nstrips) return;  // no strip: nobody waits for this warp
  const Tile tl = strips[t];
  const SlotDesc& sd = slots[tl.slot];
  SlotState* st = states + tl.slot;
  int skip = 0, k0 = 0, xbuf = 0;
  if (lane == 0) {
    skip = *((volatile int*)&st->done);
    k0 = *((volatile int*)&st->iters);
    xbuf = *((volatile int*)&st->xbuf);
    if (!skip && !dbg_tile(sd, st, tl.row0 - 1, tl.row0 + tl.nrows + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1)) {
      st->done = 1;  // the neighbours' bounded waits then end the launch with an error
      skip = 1;
    }
  }
  skip = __shfl_sync(0xffffffffu, skip, 0);
  if (skip) return;  // set only between launches: every warp sees the same value
  k0 = __shfl_sync(0xffffffffu, k0, 0);
  xbuf = __shfl_sync(0xffffffffu, xbuf, 0);
  const int rows = nstrips / ct, r = t / ct, cc = t - r * ct;
  const int nb[4] = {r > 0 ? t - ct : -1, r + 1 < rows ? t + ct : -1, cc > 0 ? t - 1 : -1,
                     cc + 1 < ct ? t + 1 : -1};
  const int pitch = sd.pitch, n = sd.n;
  const int q0 = tl.col0 + lane * kVec;
  const int i0 = tl.row0, i1 = tl.row0 + tl.nrows;
  // every packed column of the strip is interior in rows of both parities:
  // no cell needs the interior mask
  const bool full = tl.col0 + kWarpCols - 1 <= (n >> 1);
  int measure_last = 0;
  for (int p = 0; p < nphases; ++p) {
    const int colour = p & 1;
    const int k = k0 + (p >> 1) + 1;
    const FastPhase ph = phases[p];
    const int measure = ((k % sd.K) == 0) || (k >= sd.max_iters);
    if (measure && !ph.last) {  // the host plan must end chunks at measured iterations
      if (lane == 0) {
        st->error = 1;
        st->done = 1;
      }
      return;
    }
    if (p > 0 && !chain_wait(progress, nb, (unsigned)p, lane)) {
      if (lane == 0) {
        st->error = 1;
        st->done = 1;
      }
      return;
    }
    double* X = (double*)sd.x[xbuf][colour];
    const double* O = (const double*)sd.x[xbuf][colour ^ 1];
    const double* G = (const double*)sd.g[colour];
    const bool unit = ph.beta == 1.0;
    unsigned long long dm = 0;
    if (measure) {
      dm = unit ? fast_walk<true, HAS_G, true>(stages, O, X, G, pitch, n, colour, q0, i0, i1, lane, ph)
                : fast_walk<false, HAS_G, true>(stages, O, X, G, pitch, n, colour, q0, i0, i1, lane, ph);
      dm = warp_max64(dm);
      if (lane == 0 && dm) atomicMax(&st->dmax_bits, dm);
      measure_last = 1;
    } else if (unit && full) {
      (void)fast_walk<true, HAS_G, false, true>(stages, O, X, G, pitch, n, colour, q0, i0, i1, lane, ph);
    } else if (unit) {
      (void)fast_walk<true, HAS_G, false>(stages, O, X, G, pitch, n, colour, q0, i0, i1, lane, ph);
    } else {
      (void)fast_walk<false, HAS_G, false>(stages, O, X, G, pitch, n, colour, q0, i0, i1, lane, ph);
    }
    fast_ring(sd, X, colour, tl, q0, lane, ph.nscale);
    __threadfence();  // this lane's cells are visible before the strip's progress is
    __syncwarp();
    if (lane == 0) st_release_u32(progress + t, (unsigned)(p + 1));
  }
  if (lane == 0) {
    const unsigned prev = atomicAdd(&st->arrive, 1u);
    if (prev == (unsigned)nstrips - 1u) {
      __threadfence();
      finalize_plain(sd, st, k0 + (nphases >> 1), measure_last);
    }
  }
}

int fast_chain_blocks_per_sm() {
  int nb = 0;
  if (cudaFuncSetAttribute(k_fast_chain<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fast_smem_bytes<true>()) != cudaSuccess ||
      cudaFuncSetAttribute(k_fast_chain<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fast_smem_bytes<false>()) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fast_chain<true>, kThreads, fast_smem_bytes<true>()) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_fast_chain(const SlotDesc* slots, SlotState* states, const Tile* strips, int nstrips, int ct,
                              const void* phases, int nphases, unsigned* progress, bool has_g, int grid,
                              cudaStream_t s) {
  if (nstrips <= 0 || nphases <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = has_g ? fast_smem_bytes<true>() : fast_smem_bytes<false>();
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeCooperative;  // every warp resident: the neighbour waits need it
  at.val.cooperative = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  const FastPhase* ph = (const FastPhase*)phases;
  t_launches += 1;
  return has_g ? cudaLaunchKernelEx(&cfg, k_fast_chain<true>, slots, states, strips, nstrips, ct, ph, nphases, progress)
               : cudaLaunchKernelEx(&cfg, k_fast_chain<false>, slots, states, strips, nstrips, ct, ph, nphases,
                                    progress);
}

size_t fast_phase_bytes() { return sizeof(FastPhase); }

void fast_phase_pack(const FastPhaseArgs& a, void* out) {
  FastPhase ph{a.alpha, a.beta, a.gamma, a.dscale, a.nscale, a.last};
  std::memcpy(out, &ph, sizeof(ph));
}

// Saves the unscaled Dirichlet ring cells of both colour arrays of slot 0 into
// d.ring[c] (layout in SlotDesc): rows 0 and N+1 whole, then the column q = 0
// and the east ring column q = ((N + ((r + c) & 1)) >> 1) + 1 of every row r.
__global__ void k_ring_save(const SlotDesc* __restrict__ slots) {
  const SlotDesc& d = slots[0];
  const int n = d.n, pitch = d.pitch, m = n + 2;
  const int c = blockIdx.y;
  const double* X = (const double*)d.x[0][c];
  double* R = (double*)d.ring[c];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * pitch + 2 * m; e += gridDim.x * blockDim.x) {
    double v;
    if (e < pitch) {
      v = X[e];
    } else if (e < 2 * pitch) {
      v = X[(size_t)(n + 1) * pitch + (e - pitch)];
    } else if (e < 2 * pitch + m) {
      const int r = e - 2 * pitch;
      v = X[eidx(r, 0, pitch)];
    } else {
      const int r = e - 2 * pitch - m;
      v = X[eidx(r, ((n + ((r + c) & 1)) >> 1) + 1, pitch)];
    }
    R[e] = v;
  }
}

cudaError_t launch_ring_save(const SlotDesc* slots, cudaStream_t s) {
  t_launches += 1;
  k_ring_save<<<dim3(8, 2), 256, 0, s>>>(slots);
  return cudaGetLastError();
}

int fast_blocks_per_sm() {
  int nb = 0;
  if (cudaFuncSetAttribute(k_sweep_fast<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fast_smem_bytes<true>()) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_fast<true, true>, kThreads,
                                                    fast_smem_bytes<true>()) != cudaSuccess) {
    cudaGetLastError();
    return 4;
  }
  return nb > 0 ? nb : 1;
}

// ------------------------------------------------------------------------------------------------
// residual pass (FP64), both colours per tile
// ------------------------------------------------------------------------------------------------

// FP32 or FP64 value as FP64 (the widening is exact; done on the integer units).
__device__ __forceinline__ double as_f64(float x) { return widen_f32(x); }
__device__ __forceinline__ double as_f64(double x) { return x; }

// Loads 4 consecutive values of a colour array (FP64 or FP32) as FP64.
template <typename T>
__device__ __forceinline__ void load_u4(const T* X, size_t e, double (&v)[4]) {
  T t[4];
  load4(X + e, t);
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = as_f64(t[k]);
}

// Defect correction, first half of a correction step: u += (double)d over the
// interior of every pending refine slot (d from buffer dbuf of x, or the
// slot's own SlotDesc::dbuf when dbuf is kDbufPerSlot), in place.
// Elementwise, so the residual pass that follows reads corrected values
// without recomputing them for each of a cell's four neighbours.
__global__ void __launch_bounds__(kThreads) k_correct(const SlotDesc* __restrict__ slots, SlotState* states,
                                                      const Tile* __restrict__ tiles, int ntiles, int dbuf) {
  __shared__ int ctl[2];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const SlotDesc& sd = slots[tl.slot];
    SlotState* st = states + tl.slot;
    if (threadIdx.x == 0) {
      ctl[0] = *((volatile int*)&st->done) || *((volatile int*)&st->checked_iter) < 0;  // nothing pending
      ctl[1] = *((volatile int*)&st->ubuf);
      if (!dbg_tile(sd, st, tl.row0, tl.row0 + tl.nrows, tl.col0, tl.col0 + kWarpCols)) ctl[0] = 1;
    }
    __syncthreads();
    const int skip = ctl[0], ubuf = ctl[1];
    __syncthreads();
    if (skip) continue;
    const int pitch = sd.pitch, n = sd.n;
    const int q0 = tl.col0 + lane * kVec;
    const int rows_per_warp = (tl.nrows + kWarpsY - 1) / kWarpsY;
    const int i0 = tl.row0 + wy * rows_per_warp;
    const int i1 = min(i0 + rows_per_warp, tl.row0 + tl.nrows);
    for (int i = i0; i < i1; ++i) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int qlim = (n + ((i + c) & 1)) >> 1;
        if (q0 > qlim) continue;
        double* U = sd.u[ubuf][c] + eidx(i, q0, pitch);
        const float* D = (const float*)sd.x[dbuf < 0 ? sd.dbuf : dbuf][c] + eidx(i, q0, pitch);
        double u[4];
        float d[4];
        load4(U, u);
        load4(D, d);
#pragma unroll
        for (int v = 0; v < 4; ++v) u[v] = __dadd_rn(u[v], widen_f32(d[v]));
        if (q0 + 3 <= qlim) {
          store4(U, u);
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (q0 + v <= qlim) U[v] = u[v];
        }
      }
    }
  }
}

// Residual of this lane's 4 cells of one row with row parity S (fixed at
// compile time, so W / E are plain register choices):
//   r~ = (g + ((N + S) + (W + E))) - 4u,
// 4u and the rounding of r~ to FP32 being exact bit operations on the integer
// units (the FP64 rate bounds this pass).  Without a source (HAS_G false)
// g + x with g = +0 is x itself except that -0 becomes +0, which is done on
// the integer units too: 4 FP64 additions per cell instead of 5, the same
// bits.  Refine role: r~ (FP32) is written to R (this lane's first cell).
// Returns max |r~| over the interior cells.
template <int ROLE, int S, bool HAS_G>
__device__ __forceinline__ unsigned long long resid_cells(const double (&own)[4], const double (&nm)[4],
                                                          const double (&nc)[4], const double (&np)[4],
                                                          const double (&gv)[4], double left, double right, int q0,
                                                          int n, float* R) {
  double Wv[4], Ev[4];
  if (S == 0) {
    Wv[0] = nc[0]; Wv[1] = nc[1]; Wv[2] = nc[2]; Wv[3] = nc[3];
    Ev[0] = nc[1]; Ev[1] = nc[2]; Ev[2] = nc[3]; Ev[3] = right;
  } else {
    Wv[0] = left; Wv[1] = nc[0]; Wv[2] = nc[1]; Wv[3] = nc[2];
    Ev[0] = nc[0]; Ev[1] = nc[1]; Ev[2] = nc[2]; Ev[3] = nc[3];
  }
  const int qlim = (n + S) >> 1;
  unsigned long long rm = 0;
  float rv[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double nb = __dadd_rn(__dadd_rn(nm[v], np[v]), __dadd_rn(Wv[v], Ev[v]));
    double gnb;
    if (HAS_G) {
      gnb = __dadd_rn(gv[v], nb);
    } else {
      const unsigned long long b = (unsigned long long)__double_as_longlong(nb);
      gnb = __longlong_as_double((long long)(b == 0x8000000000000000ull ? 0ull : b));  // +0 + nb
    }
    const double r = __dsub_rn(gnb, times4(own[v]));
    const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
    const bool in = (q0 + v) <= qlim;
    if (in) rm = umax64(rm, abs_bits(r));
    if (ROLE == kResidRefine) rv[v] = in ? narrow_f64(__longlong_as_double((long long)rb)) : 0.0f;
  }
  if (ROLE == kResidRefine) {
    if ((q0 + 3) <= qlim) {
      store4(R, rv);
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if ((q0 + v) <= qlim) R[v] = rv[v];
    }
  }
  return rm;
}

// Both colours of row i (the own colour c0 = 0 has parity S0 = i & 1, c0 = 1
// the other), so that each colour's neighbour arrangement is fixed at
// compile time: as a runtime branch the compiler evaluated both
// arrangements' W + E, one more FP64 addition per cell.
template <typename T, int ROLE, int S0, bool HAS_G>
__device__ __forceinline__ unsigned long long resid_row(const T* X0, const T* X1, const double* G0, const double* G1,
                                                        float* R0, float* R1, int i, int q0, int pitch, int n,
                                                        int lane) {
  unsigned long long rm = 0;
#pragma unroll
  for (int c0 = 0; c0 < 2; ++c0) {
    const T* Xs = c0 ? X1 : X0;  // own colour
    const T* Xo = c0 ? X0 : X1;  // other colour
    double own[4], nm[4], nc[4], np[4], gv[4];
    load_u4(Xs, eidx(i, q0, pitch), own);
    load_u4(Xo, eidx(i - 1, q0, pitch), nm);
    load_u4(Xo, eidx(i, q0, pitch), nc);
    load_u4(Xo, eidx(i + 1, q0, pitch), np);
    if (HAS_G) {
      load4((c0 ? G1 : G0) + eidx(i, q0, pitch), gv);
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) gv[v] = 0.0;
    }
    double left = __shfl_up_sync(0xffffffffu, nc[3], 1);
    double right = __shfl_down_sync(0xffffffffu, nc[0], 1);
    if (lane == 0) left = as_f64(Xo[eidx(i, q0 - 1, pitch)]);
    if (lane == 31) right = as_f64(Xo[eidx(i, q0 + kVec, pitch)]);
    float* R = (ROLE == kResidRefine) ? (c0 ? R1 : R0) + eidx(i, q0, pitch) : nullptr;
    if (c0 == 0)
      rm = umax64(rm, resid_cells<ROLE, S0, HAS_G>(own, nm, nc, np, gv, left, right, q0, n, R));
    else
      rm = umax64(rm, resid_cells<ROLE, 1 - S0, HAS_G>(own, nm, nc, np, gv, left, right, q0, n, R));
  }
  return rm;
}

// Rows [i0, i1) of one warp, in pairs of an even and an odd row.
template <typename T, int ROLE, bool HAS_G>
__device__ __forceinline__ unsigned long long resid_rows(const T* X0, const T* X1, const double* G0, const double* G1,
                                                         float* R0, float* R1, int i0, int i1, int q0, int pitch,
                                                         int n, int lane) {
  unsigned long long rm = 0;
  int i = i0;
  if (i < i1 && (i & 1)) {
    rm = umax64(rm, resid_row<T, ROLE, 1, HAS_G>(X0, X1, G0, G1, R0, R1, i, q0, pitch, n, lane));
    ++i;
  }
  for (; i + 1 < i1; i += 2) {  // an even row, then an odd one
    rm = umax64(rm, resid_row<T, ROLE, 0, HAS_G>(X0, X1, G0, G1, R0, R1, i, q0, pitch, n, lane));
    rm = umax64(rm, resid_row<T, ROLE, 1, HAS_G>(X0, X1, G0, G1, R0, R1, i + 1, q0, pitch, n, lane));
  }
  if (i < i1) rm = umax64(rm, resid_row<T, ROLE, 0, HAS_G>(X0, X1, G0, G1, R0, R1, i, q0, pitch, n, lane));
  return rm;
}

// ROLE kResidFinal / kResidCheck: plain slots, iterate x[xbuf] (type T).
// ROLE kResidRefine: refine slots; residual of u[ubuf] (already corrected by
// k_correct), r~ rounded to FP32 into g[c]; counts the correction.
template <typename T, int ROLE>
__global__ void __launch_bounds__(kThreads) k_resid(const SlotDesc* __restrict__ slots, SlotState* states,
                                                    const Tile* __restrict__ tiles, int ntiles, int dbuf) {
  __shared__ unsigned long long red[kWarpsY];
  __shared__ TileCtl ctl;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const SlotDesc& sd = slots[tl.slot];
    SlotState* st = states + tl.slot;
    if (threadIdx.x == 0) {
      TileCtl c;
      const int done = *((volatile int*)&st->done);
      const int it = *((volatile int*)&st->iters);
      c.k = it;
      c.measure = 0;
      if (ROLE == kResidFinal) {
        c.skip = 0;
      } else if (ROLE == kResidCheck) {
        const int conv = *((volatile int*)&st->converged);
        c.skip = conv || it == 0 || (it % sd.K) != 0 || it == *((volatile int*)&st->checked_iter);
      } else {
        c.skip = done;
        c.measure = *((volatile int*)&st->checked_iter) >= 0;  // a correction is pending after the first pass
      }
      c.xbuf = (ROLE == kResidRefine) ? *((volatile int*)&st->ubuf) : *((volatile int*)&st->xbuf);
      if (!dbg_tile(sd, st, tl.row0 - 1, tl.row0 + tl.nrows + 1, tl.col0 - 1, tl.col0 + kWarpCols + 1)) c.skip = 1;
      ctl = c;
    }
    __syncthreads();
    const TileCtl c = ctl;
    __syncthreads();
    if (c.skip) continue;

    const int pitch = sd.pitch, n = sd.n;
    const T* X0;
    const T* X1;
    if (ROLE == kResidRefine) {
      X0 = (const T*)sd.u[c.xbuf][0];
      X1 = (const T*)sd.u[c.xbuf][1];
    } else {
      X0 = (const T*)sd.x[c.xbuf][0];
      X1 = (const T*)sd.x[c.xbuf][1];
    }
    const double* G0 = sd.g64[0];
    const double* G1 = sd.g64[1];
    float* R0 = (ROLE == kResidRefine) ? (float*)sd.g[0] : nullptr;
    float* R1 = (ROLE == kResidRefine) ? (float*)sd.g[1] : nullptr;

    const int q0 = tl.col0 + lane * kVec;
    const int rows_per_warp = (tl.nrows + kWarpsY - 1) / kWarpsY;
    const int i0 = tl.row0 + wy * rows_per_warp;
    const int i1 = min(i0 + rows_per_warp, tl.row0 + tl.nrows);
    // the source term is a compile-time choice per tile (slots of a batch differ)
    const unsigned long long rm = G0 ? resid_rows<T, ROLE, true>(X0, X1, G0, G1, R0, R1, i0, i1, q0, pitch, n, lane)
                                     : resid_rows<T, ROLE, false>(X0, X1, G0, G1, R0, R1, i0, i1, q0, pitch, n, lane);
    block_max_to(rm, &st->rmax_bits, red);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(&st->arrive_res, 1u);
      if (prev == (unsigned)sd.resid_tiles - 1u) {
        __threadfence();
        st->arrive_res = 0;
        const double rmax = bits_to_double(atomicExch(&st->rmax_bits, 0ull));
        const double bmax = bits_to_double(*((volatile unsigned long long*)&st->bmax_bits));
        const double rho = bmax > 0.0 ? __ddiv_rn(rmax, bmax) : rmax;
        st->last_rho = rho;
        if (ROLE == kResidCheck) {
          st->checked_iter = c.k;
          if (rho < sd.tol) {
            st->converged = 1;
            st->done = 1;
          } else if (rho < st->best_rho) {
            st->best_rho = rho;
            st->stall_run = 0;
          } else if (rho < 4.0 * st->best_rho) {  // a plateau near the smallest residual so far
            st->stall_run += 1;
            if (sd.stall > 0 && st->stall_run >= sd.stall) st->done = 1;  // the floor: tol is out of reach
          } else {
            st->stall_run = 0;  // far above it: still the early growth, not a plateau
          }
        } else if (ROLE == kResidRefine) {
          if (c.measure) {  // the correction k_correct applied counts now
            st->outer += 1;
            st->iters += sd.inner;
          }
          st->checked_iter = st->iters;
          if (rho < sd.tol) {
            st->converged = 1;
            st->done = 1;
          } else if (st->iters + sd.inner > sd.max_iters) {
            st->done = 1;
          } else if (rho < st->best_rho) {
            st->best_rho = rho;
            st->stall_run = 0;
          } else if (rho < 4.0 * st->best_rho) {
            st->stall_run += 1;
            if (sd.stall > 0 && st->stall_run >= sd.stall) st->done = 1;
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
// launch wrappers (host)
// ------------------------------------------------------------------------------------------------

static dim3 pack_grid(int n) {
  const int qw = (n + 1) / 2 + 2;
  return dim3((qw + kThreads - 1) / kThreads, n + 2);
}

cudaError_t launch_pack(const PackArgs& a, cudaStream_t s) {
  const dim3 grid = pack_grid(a.n);
  t_launches += 1;
  if (a.fp32) {
    k_pack<float><<<grid, kThreads, 0, s>>>(a.u0, a.f, a.n, a.pitch, a.h2, (float*)a.x[0][0], (float*)a.x[0][1],
                                            (float*)a.x[1][0], (float*)a.x[1][1], (float*)a.g[0], (float*)a.g[1],
                                            a.g64[0], a.g64[1], a.u[0][0], a.u[0][1], a.u[1][0], a.u[1][1],
                                            a.state);
  } else {
    k_pack<double><<<grid, kThreads, 0, s>>>(a.u0, a.f, a.n, a.pitch, a.h2, (double*)a.x[0][0],
                                             (double*)a.x[0][1], (double*)a.x[1][0], (double*)a.x[1][1],
                                             (double*)a.g[0], (double*)a.g[1], a.g64[0], a.g64[1], a.u[0][0],
                                             a.u[0][1], a.u[1][0], a.u[1][1], a.state);
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack(const void* c0, const void* c1, bool fp32, int n, int pitch, double* out,
                          cudaStream_t s) {
  const dim3 grid = pack_grid(n);
  t_launches += 1;
  if (fp32)
    k_unpack<float><<<grid, kThreads, 0, s>>>((const float*)c0, (const float*)c1, n, pitch, out);
  else
    k_unpack<double><<<grid, kThreads, 0, s>>>((const double*)c0, (const double*)c1, n, pitch, out);
  return cudaGetLastError();
}

cudaError_t launch_sweep(SweepKind kind, const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles,
                         int grid, int colour, int sweep, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  t_launches += 1;
  switch (kind) {
    case kSweepPlain64:
      k_sweep<double, 0><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, colour, sweep);
      break;
    case kSweepPlain32:
      k_sweep<float, 0><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, colour, sweep);
      break;
    case kSweepInner32:
      k_sweep<float, 1><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, colour, sweep);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep_fast64(const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles, int grid,
                                int colour, const FastPhaseArgs& a, bool has_g, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const int need = (ntiles + kWarpsY - 1) / kWarpsY;  // one warp per strip
  if (grid <= 0 || grid > need) grid = need;
  FastPhase ph{a.alpha, a.beta, a.gamma, a.dscale, a.nscale, a.last};
  const bool unit = a.beta == 1.0;
  static bool attr_set = false;  // benign race: setting the attributes twice is harmless
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_fast<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fast_smem_bytes<false>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_sweep_fast<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fast_smem_bytes<false>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_sweep_fast<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fast_smem_bytes<true>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_sweep_fast<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fast_smem_bytes<true>());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const size_t sm0 = fast_smem_bytes<false>(), sm1 = fast_smem_bytes<true>();
  t_launches += 1;
  if (unit && !has_g)
    k_sweep_fast<true, false><<<grid, kThreads, sm0, s>>>(slots, states, tiles, ntiles, colour, ph);
  else if (unit && has_g)
    k_sweep_fast<true, true><<<grid, kThreads, sm1, s>>>(slots, states, tiles, ntiles, colour, ph);
  else if (!has_g)
    k_sweep_fast<false, false><<<grid, kThreads, sm0, s>>>(slots, states, tiles, ntiles, colour, ph);
  else
    k_sweep_fast<false, true><<<grid, kThreads, sm1, s>>>(slots, states, tiles, ntiles, colour, ph);
  return cudaGetLastError();
}

cudaError_t launch_resid(ResidKind kind, const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles,
                         int grid, int dbuf, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  t_launches += kind == kResidRefine64 ? 2 : 1;
  if (kind == kResidRefine64Fixed) kind = kResidRefine64;  // the sweeps applied the correction
  else if (kind == kResidRefine64) {  // u += d first (nothing when no correction is pending)
    k_correct<<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, dbuf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  switch (kind) {
    case kResidFinal64:
      k_resid<double, kResidFinal><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, dbuf);
      break;
    case kResidFinal32:
      k_resid<float, kResidFinal><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, dbuf);
      break;
    case kResidCheck64:
      k_resid<double, kResidCheck><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, dbuf);
      break;
    case kResidCheck32:
      k_resid<float, kResidCheck><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, dbuf);
      break;
    case kResidRefine64:
      k_resid<double, kResidRefine><<<grid, kThreads, 0, s>>>(slots, states, tiles, ntiles, dbuf);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// fused FP32 sweeps: the two kernel families behind one interface
// ------------------------------------------------------------------------------------------------

bool fused_depth_supported(int kind, int T) {
  return kind == kFusedWave ? wave_depth_supported(T) : tile_depth_supported(T);
}

int fused_out_cols(int kind, int T) { return kind == kFusedWave ? wave_out_cols(T) : tile_out_cols(T); }

int fused_out_rows(int kind, int n, int T, int sm_count, int seg) {
  if (kind != kFusedWave) return tile_out_rows();
  if (seg > 0) return seg < n ? seg : n;
  return wave_seg_rows(n, T, sm_count);
}

cudaError_t fused_prepare(int kind, int T) { return kind == kFusedWave ? wave_prepare(T) : tile_prepare(T); }

bool fused_corrects(int kind) { return kind != kFusedWave; }

cudaError_t launch_fused(int kind, bool inner, int T, const SlotDesc* slots, SlotState* states, const Tile* tiles,
                         int ntiles, int grid, int nt, int src, int sweep0, cudaStream_t s, bool correct) {
  if (correct && !fused_corrects(kind)) return cudaErrorInvalidValue;
  return kind == kFusedWave ? launch_sweep_wave(inner, T, slots, states, tiles, ntiles, grid, nt, src, sweep0, s)
                            : launch_sweep_tile(inner, T, slots, states, tiles, ntiles, grid, nt, src, sweep0, s,
                                                correct);
}

}  // namespace sorgb
