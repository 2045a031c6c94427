// FP32 colour phases fused over T iterations per shared-memory tile pass
// (temporal blocking of Algorithm 1's red and black phases, Section 3.1):
// the tile family of the fused sweeps.  The wavefront family (sor_wf.cu)
// computes the same iterations bit for bit; which one runs is chosen per
// solve (by grid size, or by the autotuner), since the two trade shared-
// memory traffic against halo recomputation differently: this one is the
// faster of the two while a plate's FP32 state stays in L2.
#include <cuda_runtime.h>

#include "sor_bits.cuh"
#include "sor_devfn.cuh"
#include "sor_device.cuh"
#include "sor_kernels.h"

namespace sorgb {

constexpr int kTbRows = 64;      // output rows of a tile
constexpr int kTbThreads = 256;  // threads of a tile

// ------------------------------------------------------------------------------------------------
// FP32 colour phases fused over several iterations per tile (temporal blocking)
// ------------------------------------------------------------------------------------------------
//
// A tile of kTbRows output rows and OQ = 128 - 2*HQ output packed columns of
// both colours is staged in shared memory together with a halo of HR = 2T
// rows and HQ >= T+1 packed columns (a cell's value after t red-black
// iterations depends on cells at most 2t rows and t packed columns away), so
// every staged row is exactly 128 packed columns: one float4 per lane of a
// warp.  T iterations -- red phase, black phase, each the exact update of
// k_sweep -- then run on the staged copy: each warp walks a segment of rows
// keeping the neighbour colour's rows i-1, i in registers, W/E neighbours come
// by shuffles, and a cell update costs two shared-memory loads and one store.
// After each phase the cells next to the staged border are stale, the stale
// band growing inward by at most one row and one packed column per phase; the
// centre tile stays exact and is written to the other buffer of the
// ping-pong pair, so neighbouring tiles keep reading the previous iterate.
// HBM traffic per cell: one read and one write per T iterations plus the
// halo re-reads, most of which L2 serves.

template <int T>
struct TbGeom {
  static constexpr int HR = 2 * T;                              // halo rows
  static constexpr int HQ = T <= 3 ? 4 : (T <= 7 ? 8 : 12);     // halo packed columns (multiple of 4, >= T+1)
  static constexpr int C = 128;                                 // staged packed columns
  static constexpr int OQ = C - 2 * HQ;                         // output packed columns
  static constexpr int R = kTbRows + 2 * HR;                    // staged rows
  static constexpr size_t smem = 2ull * R * C * sizeof(float);
};

__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gsrc, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 16 : 0;  // src-size 0 fills the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(valid ? gsrc : nullptr), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Right-hand-side values of this lane's 4 cells of one row, read from global
// memory rows before their use (the right-hand side is read-only for the
// launch and each lane uses only the values it loads, so they go straight to
// registers).  Nothing is loaded for rows past the phase's rows or lanes
// without interior cells of that row parity; g then keeps stale values, which
// only masked cells (whose result is discarded) or no row at all ever use.
__device__ __forceinline__ void tb_g_load(float (&g)[4], const float* gp, bool ok) {
  if (ok) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(gp));
    g[0] = v.x; g[1] = v.y; g[2] = v.z; g[3] = v.w;
  }
}

// One row r of a phase on the staged tile.  om / oc / op: the neighbour
// colour's staged rows r-1, r, r+1 (this lane's 4 columns, in registers);
// S = (i + colour) & 1 for the global row i, fixed at compile time, which
// decides which single neighbour value comes from the next lane (S == 0: the
// east one of the last cell; S == 1: the west one of the first cell).  gv:
// the row's right-hand side (HAS_G).  m: this lane's interior cells (unused
// when FULL); out_row / outc: the cells counted by the max|change| of a
// measured phase.  Exact operation order of the oracle.
template <bool LASTM, bool FULL, bool HAS_G, int S>
__device__ __forceinline__ void tb_row(const float (&om)[4], const float (&oc)[4], const float (&op)[4],
                                       float* __restrict__ own_p, const float (&gv)[4], unsigned m,
                                       bool out_row, unsigned outc, float a, float b, unsigned& dm32) {
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
  float own[4];
  load4(own_p, own);
  // Cells of staged columns 0 and C-1 see a wrong W or E (no staged
  // neighbour); like every cell near the staged border they are stale, and
  // the stale band never reaches the output tile.
  float nv[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float sum = radd(radd(om[v], op[v]), radd(W[v], E[v]));
    if (HAS_G) sum = radd(sum, gv[v]);
    const float nu = radd(rmul(a, own[v]), rmul(b, sum));
    const bool in = FULL || ((m >> v) & 1u);
    nv[v] = in ? nu : own[v];
    if (LASTM && out_row && in && ((outc >> v) & 1u)) dm32 = max(dm32, abs_bits32(radd(nu, -own[v])));
  }
  store4(own_p, nv);
}

// Per-phase constants of one warp's rows.
struct TbRows {
  float* Sc;        // own colour, staged
  const float* So;  // neighbour colour, staged
  const float* Gc;  // right-hand side of the own colour at this lane's first cell of row r0 (HAS_G)
  int qf, pitch, lane, r0, out_lo, out_hi;
  unsigned in0, in1, outc;
  bool gok0, gok1;  // this lane has interior cells in rows of parity 0 / 1
  float a, b;
};

// Row r (parity S) with right-hand side gv, after which gv takes row
// r + AHEAD's (a row of the same parity), from gp_next.
template <int C, bool LASTM, bool FULL, bool HAS_G, int S, int AHEAD = 8>
__device__ __forceinline__ void tb_row_at(const TbRows& R, int r, int r1, const float (&om)[4], const float (&oc)[4],
                                          const float (&op)[4], float (&gv)[4], const float* gp_next,
                                          unsigned& dm32) {
  const bool out_row = LASTM && r >= R.out_lo && r < R.out_hi;
  tb_row<LASTM, FULL, HAS_G, S>(om, oc, op, R.Sc + r * C + 4 * R.lane, gv, S ? R.in1 : R.in0, out_row, R.outc, R.a,
                                R.b, dm32);
  if (HAS_G) tb_g_load(gv, gp_next, r + AHEAD < r1 && (S ? R.gok1 : R.gok0));
}

// Rows [R.r0, r1) of the staged tile, the first with parity S0, without a
// right-hand side.  Bodies of four rows cycle four register rows in place
// (rows r-1 .. r+4 pass through X, Y, P, Q and leave X, Y holding r+3, r+4),
// so no row values are moved.
template <int C, bool LASTM, bool FULL, int S0>
__device__ __forceinline__ void tb_rows_plain(const TbRows& R, int r1, unsigned& dm32) {
  const float* So = R.So + 4 * R.lane;
  int r = R.r0;
  float X[4], Y[4], P[4], Q[4], G[4];  // G: unused right-hand side
  load4(So + (r - 1) * C, X);
  load4(So + r * C, Y);
  for (; r + 4 <= r1; r += 4) {
    load4(So + (r + 1) * C, P);
    tb_row_at<C, LASTM, FULL, false, S0>(R, r, r1, X, Y, P, G, nullptr, dm32);
    load4(So + (r + 2) * C, Q);
    tb_row_at<C, LASTM, FULL, false, 1 - S0>(R, r + 1, r1, Y, P, Q, G, nullptr, dm32);
    load4(So + (r + 3) * C, X);
    tb_row_at<C, LASTM, FULL, false, S0>(R, r + 2, r1, P, Q, X, G, nullptr, dm32);
    load4(So + (r + 4) * C, Y);
    tb_row_at<C, LASTM, FULL, false, 1 - S0>(R, r + 3, r1, Q, X, Y, G, nullptr, dm32);
  }
  if (r < r1) {
    load4(So + (r + 1) * C, P);
    tb_row_at<C, LASTM, FULL, false, S0>(R, r, r1, X, Y, P, G, nullptr, dm32);
    if (r + 1 < r1) {
      load4(So + (r + 2) * C, Q);
      tb_row_at<C, LASTM, FULL, false, 1 - S0>(R, r + 1, r1, Y, P, Q, G, nullptr, dm32);
      if (r + 2 < r1) {
        load4(So + (r + 3) * C, X);
        tb_row_at<C, LASTM, FULL, false, S0>(R, r + 2, r1, P, Q, X, G, nullptr, dm32);
      }
    }
  }
}

// The same with a right-hand side: bodies of eight rows (two turns of the
// four register rows), G[j] holding the right-hand side of row r + j and
// refilled with row r + j + 8 as soon as it has been used, so each load is
// issued eight rows before its use.
template <int C, bool LASTM, bool FULL, int S0>
__device__ __forceinline__ void tb_rows_g(const TbRows& R, int r1, unsigned& dm32) {
  const float* So = R.So + 4 * R.lane;
  int r = R.r0;
  float X[4], Y[4], P[4], Q[4];
  float G[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int v = 0; v < 4; ++v) G[j][v] = 0.0f;  // once per phase: a load that is skipped leaves them
  const ptrdiff_t gs = R.pitch;
  const float* gp = R.Gc;  // right-hand side of row r
  const bool ok0 = S0 ? R.gok1 : R.gok0;  // rows of the parity of row r0 / of the other parity
  const bool ok1 = S0 ? R.gok0 : R.gok1;
  load4(So + (r - 1) * C, X);
  load4(So + r * C, Y);
#pragma unroll
  for (int j = 0; j < 8; ++j) tb_g_load(G[j], gp + j * gs, r + j < r1 && ((j & 1) ? ok1 : ok0));
  for (; r + 8 <= r1; r += 8, gp += 8 * gs) {
    load4(So + (r + 1) * C, P);
    tb_row_at<C, LASTM, FULL, true, S0>(R, r, r1, X, Y, P, G[0], gp + 8 * gs, dm32);
    load4(So + (r + 2) * C, Q);
    tb_row_at<C, LASTM, FULL, true, 1 - S0>(R, r + 1, r1, Y, P, Q, G[1], gp + 9 * gs, dm32);
    load4(So + (r + 3) * C, X);
    tb_row_at<C, LASTM, FULL, true, S0>(R, r + 2, r1, P, Q, X, G[2], gp + 10 * gs, dm32);
    load4(So + (r + 4) * C, Y);
    tb_row_at<C, LASTM, FULL, true, 1 - S0>(R, r + 3, r1, Q, X, Y, G[3], gp + 11 * gs, dm32);
    load4(So + (r + 5) * C, P);
    tb_row_at<C, LASTM, FULL, true, S0>(R, r + 4, r1, X, Y, P, G[4], gp + 12 * gs, dm32);
    load4(So + (r + 6) * C, Q);
    tb_row_at<C, LASTM, FULL, true, 1 - S0>(R, r + 5, r1, Y, P, Q, G[5], gp + 13 * gs, dm32);
    load4(So + (r + 7) * C, X);
    tb_row_at<C, LASTM, FULL, true, S0>(R, r + 6, r1, P, Q, X, G[6], gp + 14 * gs, dm32);
    load4(So + (r + 8) * C, Y);
    tb_row_at<C, LASTM, FULL, true, 1 - S0>(R, r + 7, r1, Q, X, Y, G[7], gp + 15 * gs, dm32);
  }
  // at most seven rows left, their right-hand sides in G[0] .. G[6]; nothing further is loaded
  if (r < r1) {
    load4(So + (r + 1) * C, P);
    tb_row_at<C, LASTM, FULL, true, S0>(R, r, r1, X, Y, P, G[0], gp, dm32);
    if (r + 1 < r1) {
      load4(So + (r + 2) * C, Q);
      tb_row_at<C, LASTM, FULL, true, 1 - S0>(R, r + 1, r1, Y, P, Q, G[1], gp, dm32);
      if (r + 2 < r1) {
        load4(So + (r + 3) * C, X);
        tb_row_at<C, LASTM, FULL, true, S0>(R, r + 2, r1, P, Q, X, G[2], gp, dm32);
        if (r + 3 < r1) {
          load4(So + (r + 4) * C, Y);
          tb_row_at<C, LASTM, FULL, true, 1 - S0>(R, r + 3, r1, Q, X, Y, G[3], gp, dm32);
          if (r + 4 < r1) {
            load4(So + (r + 5) * C, P);
            tb_row_at<C, LASTM, FULL, true, S0>(R, r + 4, r1, X, Y, P, G[4], gp, dm32);
            if (r + 5 < r1) {
              load4(So + (r + 6) * C, Q);
              tb_row_at<C, LASTM, FULL, true, 1 - S0>(R, r + 5, r1, Y, P, Q, G[5], gp, dm32);
              if (r + 6 < r1) {
                load4(So + (r + 7) * C, X);
                tb_row_at<C, LASTM, FULL, true, S0>(R, r + 6, r1, P, Q, X, G[6], gp, dm32);
              }
            }
          }
        }
      }
    }
  }
}

template <int C, bool LASTM, bool FULL, bool HAS_G, int S0>
__device__ __forceinline__ void tb_rows(const TbRows& R, int r1, unsigned& dm32) {
  if (HAS_G)
    tb_rows_g<C, LASTM, FULL, S0>(R, r1, dm32);
  else
    tb_rows_plain<C, LASTM, FULL, S0>(R, r1, dm32);
}

// One colour phase on the staged tile: rows [r0, r1) of the staged arrays for
// this warp, clipped to global interior rows.  LASTM: this phase belongs to a
// measured iteration, track max |change| over the tile's output cells.
// FULL: every staged column of the tile is an interior packed column of both
// colours (no ring or padding cell among them), so no cell needs masking.
template <int T, bool LASTM, bool FULL, bool HAS_G>
__device__ __forceinline__ void tb_phase(float* __restrict__ Sc, const float* __restrict__ So,
                                         const float* __restrict__ Gc, int colour, int base_r, int base_q, int r0,
                                         int r1, int n, int pitch, int out_rows, int lane, float a, float b,
                                         unsigned& dm32) {
  using Gm = TbGeom<T>;
  r0 = max(r0, 1 - base_r);  // global rows 1 .. n only
  r1 = min(r1, n + 1 - base_r);
  if (r0 >= r1) return;
  TbRows R;
  R.Sc = Sc;
  R.So = So;
  R.qf = base_q + 4 * lane;
  R.Gc = HAS_G ? Gc + (ptrdiff_t)(base_r + r0) * pitch + R.qf + kOff : nullptr;
  R.pitch = pitch;
  R.lane = lane;
  R.r0 = r0;
  R.out_lo = Gm::HR;
  R.out_hi = Gm::HR + out_rows;
  R.a = a;
  R.b = b;
  // this lane's interior cells for row parity 0 / 1 (bit v: packed column qf + v)
  // and, for the measured phase, its cells inside the output columns
  R.in0 = 0xF;
  R.in1 = 0xF;
  R.outc = 0;
  if (!FULL) {
    R.in0 = 0;
    R.in1 = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int q = R.qf + v;
      R.in0 |= (unsigned)(q >= 1 && q <= (n >> 1)) << v;
      R.in1 |= (unsigned)(q >= 1 && q <= ((n + 1) >> 1)) << v;
    }
  }
  R.gok0 = R.in0 != 0;
  R.gok1 = R.in1 != 0;
  if (LASTM) {
    const int col = 4 * lane;
#pragma unroll
    for (int v = 0; v < 4; ++v) R.outc |= (unsigned)(col + v >= Gm::HQ && col + v < Gm::HQ + Gm::OQ) << v;
  }
  if (((base_r + r0 + colour) & 1) == 0)
    tb_rows<Gm::C, LASTM, FULL, HAS_G, 0>(R, r1, dm32);
  else
    tb_rows<Gm::C, LASTM, FULL, HAS_G, 1>(R, r1, dm32);
}

// MODE 0: plain FP32 iterations on x (rhs g optional), source buffer from the
//         slot state; the last iteration of the launch may be a measured one.
// MODE 1: inner sweeps of defect correction on d with rhs r~; `src` is the
//         buffer holding d (the first launch of a correction, sweep0 == 0,
//         starts from d = 0 and reads nothing).  corr: the launch that ends
//         a slot's inner sweeps adds its final d to u (u += (double)d, the
//         rounding of k_correct) instead of storing d, so no correction pass
//         runs before the next residual.
template <int T, int MODE>
__global__ void __launch_bounds__(kTbThreads, 2) k_sweep_tb(const SlotDesc* __restrict__ slots, SlotState* states,
                                                            const Tile* __restrict__ tiles, int ntiles, int nt_req,
                                                            int src_param, int sweep0, int corr) {
  using Gm = TbGeom<T>;
  constexpr int kWarps = kTbThreads / 32;
  extern __shared__ __align__(16) float tb_smem[];
  float* const S0 = tb_smem;
  float* const S1 = tb_smem + Gm::R * Gm::C;
  __shared__ unsigned long long red[kWarps];
  __shared__ int ctl[7];  // skip, nt, k_end, measure, src, correct u here, u buffer
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const SlotDesc& sd = slots[tl.slot];
    SlotState* st = states + tl.slot;
    if (threadIdx.x == 0) {
      int skip = *((volatile int*)&st->done);
      int nt = 0, k_end = 0, measure = 0, src = 0;
      if (MODE == 0) {
        const int k0 = *((volatile int*)&st->iters);
        nt = min(nt_req, sd.max_iters - k0);
        k_end = k0 + nt;
        measure = (k_end % sd.K) == 0 || k_end >= sd.max_iters;
        src = *((volatile int*)&st->xbuf);
        for (int j = k0 + 1; j < k_end && !skip; ++j)  // the host plan ends launches at measured iterations
          if ((j % sd.K) == 0) {
            st->error = 1;
            st->done = 1;
            skip = 1;
          }
        if (nt <= 0) skip = 1;
      } else {
        nt = min(nt_req, sd.inner - sweep0);
        if (nt <= 0) skip = 1;
        src = src_param;
        ctl[5] = corr && sweep0 + nt >= sd.inner;  // this slot's inner sweeps end in this launch
        ctl[6] = *((volatile int*)&st->ubuf);
      }
      // the output rows and columns of the tile lie inside the slot's arrays
      if (!skip && !dbg_tile(sd, st, tl.row0, tl.row0 + tl.nrows, tl.col0, tl.col0 + Gm::OQ)) skip = 1;
      ctl[0] = skip; ctl[1] = nt; ctl[2] = k_end; ctl[3] = measure; ctl[4] = src;
    }
    __syncthreads();
    const int skip = ctl[0], nt = ctl[1], k_end = ctl[2], measure = ctl[3], src = ctl[4];
    const int fix_u = MODE == 1 ? ctl[5] : 0, ubuf = MODE == 1 ? ctl[6] : 0;
    __syncthreads();
    if (skip) continue;

    const int pitch = sd.pitch, n = sd.n;
    const int base_r = tl.row0 - Gm::HR;
    const int base_q = tl.col0 - Gm::HQ;
    const int base_e = base_q + kOff;  // element index of staged column 0 (a multiple of 4)
    const bool zero_start = (MODE == 1) && sweep0 == 0;
    // stage both colours: warp per row, lane per float4; rows outside the
    // array and columns outside the row read as 0
    for (int row = warp; row < 2 * Gm::R; row += kWarps) {
      const int c = row >= Gm::R;
      const int r = row - c * Gm::R;
      const int i = base_r + r;
      const int e = base_e + 4 * lane;
      const bool valid = !zero_start && i >= 0 && i <= n + 1 && e >= 0 && e + 4 <= pitch;
      const float* gp = valid ? (const float*)sd.x[src][c] + (size_t)i * pitch + e : nullptr;
      cp_async16((c ? S1 : S0) + r * Gm::C + 4 * lane, gp, valid);
    }
    cp_async_wait_all();
    __syncthreads();

    const float a = sd.a32, b = sd.b32;
    unsigned dm32 = 0;
    const bool full = base_q >= 1 && base_q + Gm::C - 1 <= (n >> 1);
    for (int it = 0; it < nt; ++it) {
      const bool lastm = (MODE == 0) && measure && it == nt - 1;
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        // Phase p = 2it + c + 1 of 2nt: only rows within 2nt - p of the output
        // rows can still reach them, so the updated band shrinks by one row
        // at each end per phase (it starts at staged rows 1 .. R-2 when nt = T).
        const int reach = 2 * nt - (2 * it + c + 1);
        const int lo = Gm::HR - reach, hi = Gm::HR + tl.nrows + reach;
        const int seg = (hi - lo + kWarps - 1) / kWarps;
        const int r0 = lo + warp * seg;
        const int r1 = min(r0 + seg, hi);
        float* Sc = c ? S1 : S0;
        const float* So = c ? S0 : S1;
        const float* Gc = (const float*)sd.g[c];
#define TB_PHASE(LM, FL, HG) \
  tb_phase<T, LM, FL, HG>(Sc, So, Gc, c, base_r, base_q, r0, r1, n, pitch, tl.nrows, lane, a, b, dm32)
        if (Gc) {
          if (full) {
            if (lastm) TB_PHASE(true, true, true); else TB_PHASE(false, true, true);
          } else {
            if (lastm) TB_PHASE(true, false, true); else TB_PHASE(false, false, true);
          }
        } else {
          if (full) {
            if (lastm) TB_PHASE(true, true, false); else TB_PHASE(false, true, false);
          } else {
            if (lastm) TB_PHASE(true, false, false); else TB_PHASE(false, false, false);
          }
        }
#undef TB_PHASE
        __syncthreads();
      }
    }
    // the correction ending a slot's inner sweeps: u += (double)d over the
    // centre tile, the u vectors of kTbFixRows rows requested together before
    // any is used (a row at a time, each thread waited for every load)
    if (MODE == 1 && fix_u) {
      constexpr int kTbFixRows = 2;
      for (int row0 = warp; row0 < 2 * kTbRows; row0 += kWarps * kTbFixRows) {
        double u4[kTbFixRows][4];
        float v4[kTbFixRows][4];
        double* Ud[kTbFixRows];
        int cnt[kTbFixRows];  // interior cells of the vector: 4, 1 .. 3 at the row's end, 0 = none
#pragma unroll
        for (int j = 0; j < kTbFixRows; ++j) {
          cnt[j] = 0;
          Ud[j] = nullptr;
          const int row = row0 + j * kWarps;
          const int c = row >= kTbRows;
          const int r = row - c * kTbRows;
          const int col = 4 * lane;
          if (row >= 2 * kTbRows || r >= tl.nrows || col < Gm::HQ || col >= Gm::HQ + Gm::OQ) continue;
          const int i = tl.row0 + r;
          const int qlim = (n + ((i + c) & 1)) >> 1;
          const int qf = base_q + col;
          if (qf > qlim) continue;
          cnt[j] = min(4, qlim - qf + 1);
          load4((c ? S1 : S0) + (Gm::HR + r) * Gm::C + col, v4[j]);
          Ud[j] = sd.u[ubuf][c] + (size_t)i * pitch + qf + kOff;
          if (cnt[j] == 4) {
            load4(Ud[j], u4[j]);
          } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) u4[j][v] = v < cnt[j] ? Ud[j][v] : 0.0;
          }
        }
#pragma unroll
        for (int j = 0; j < kTbFixRows; ++j) {
          if (cnt[j] == 0) continue;
#pragma unroll
          for (int v = 0; v < 4; ++v) u4[j][v] = __dadd_rn(u4[j][v], widen_f32(v4[j][v]));
          if (cnt[j] == 4) {
            store4(Ud[j], u4[j]);
          } else {
#pragma unroll
            for (int v = 0; v < 4; ++v)
              if (v < cnt[j]) Ud[j][v] = u4[j][v];
          }
        }
      }
    } else {
      // write the centre tile to the other buffer: warp per row, lane per float4
      const int dst = src ^ 1;
      for (int row = warp; row < 2 * kTbRows; row += kWarps) {
        const int c = row >= kTbRows;
        const int r = row - c * kTbRows;
        if (r >= tl.nrows) continue;
        const int col = 4 * lane;
        if (col < Gm::HQ || col >= Gm::HQ + Gm::OQ) continue;
        const int i = tl.row0 + r;
        const int s = (i + c) & 1;
        const int qlim = (n + s) >> 1;
        const int qf = base_q + col;
        if (qf > qlim) continue;
        float v4[4];
        load4((c ? S1 : S0) + (Gm::HR + r) * Gm::C + col, v4);
        float* Xd = (float*)sd.x[dst][c] + (size_t)i * pitch + qf + kOff;
        if (qf + 3 <= qlim) {
          store4(Xd, v4);
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (qf + v <= qlim) Xd[v] = v4[v];
        }
      }
    }
    if (MODE == 0) {
      if (measure) {
        unsigned long long dm = warp_max64(abs_bits_of(__uint_as_float(dm32)));
        if (lane == 0) red[warp] = dm;
        __syncthreads();
        if (threadIdx.x == 0) {
          unsigned long long m = 0;
          for (int k = 0; k < kWarps; ++k) m = umax64(m, red[k]);
          if (m) atomicMax(&st->dmax_bits, m);
        }
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        if (prev == (unsigned)sd.sweep_tiles - 1u) {
          __threadfence();
          st->xbuf = src ^ 1;
          finalize_plain(sd, st, k_end, measure);
        }
      }
    }
    __syncthreads();  // the next tile reuses the staged arrays
  }
}

int tile_out_cols(int T) {
  switch (T) {
    case 2: return TbGeom<2>::OQ;
    case 3: return TbGeom<3>::OQ;
    case 4: return TbGeom<4>::OQ;
    case 6: return TbGeom<6>::OQ;
    case 8: return TbGeom<8>::OQ;
    default: return kWarpCols;
  }
}


template <int T, int MODE>
static cudaError_t launch_tile_t(const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles, int grid,
                               int nt, int src, int sweep0, int corr, cudaStream_t s) {
  static bool attr_set = false;  // benign race: setting the attribute twice is harmless
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_tb<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TbGeom<T>::smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  count_kernel_launches(1);
  k_sweep_tb<T, MODE><<<grid, kTbThreads, TbGeom<T>::smem, s>>>(slots, states, tiles, ntiles, nt, src, sweep0, corr);
  return cudaGetLastError();
}

bool tile_depth_supported(int T) { return T == 2 || T == 3 || T == 4 || T == 6 || T == 8; }

cudaError_t launch_sweep_tile(bool inner, int T, const SlotDesc* slots, SlotState* states, const Tile* tiles,
                            int ntiles, int grid, int nt, int src, int sweep0, cudaStream_t s, bool correct) {
  if (ntiles <= 0) return cudaSuccess;
  if (nt < 1 || nt > T) return cudaErrorInvalidValue;
  const int corr = inner && correct ? 1 : 0;
  switch (T) {
    case 2: return inner ? launch_tile_t<2, 1>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s)
                         : launch_tile_t<2, 0>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s);
    case 3: return inner ? launch_tile_t<3, 1>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s)
                         : launch_tile_t<3, 0>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s);
    case 4: return inner ? launch_tile_t<4, 1>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s)
                         : launch_tile_t<4, 0>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s);
    case 6: return inner ? launch_tile_t<6, 1>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s)
                         : launch_tile_t<6, 0>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s);
    case 8: return inner ? launch_tile_t<8, 1>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s)
                         : launch_tile_t<8, 0>(slots, states, tiles, ntiles, grid, nt, src, sweep0, corr, s);
    default: return cudaErrorInvalidValue;
  }
}


int tile_out_rows() { return kTbRows; }

// Opts the kernels of depth T into their shared memory (call outside graph capture).
cudaError_t tile_prepare(int T) {
  cudaError_t e = cudaSuccess;
#define TILE_PREP(TT)                                                                                        \
  if (T == TT) {                                                                                             \
    e = cudaFuncSetAttribute(k_sweep_tb<TT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                             (int)TbGeom<TT>::smem);                                                         \
    if (e == cudaSuccess)                                                                                    \
      e = cudaFuncSetAttribute(k_sweep_tb<TT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                               (int)TbGeom<TT>::smem);                                                       \
  }
  TILE_PREP(2) TILE_PREP(3) TILE_PREP(4) TILE_PREP(6) TILE_PREP(8)
#undef TILE_PREP
  return e;
}

}  // namespace sorgb
