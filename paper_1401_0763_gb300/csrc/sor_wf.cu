// FP32 colour phases fused over T iterations as a register wavefront
// (temporal blocking of Algorithm 1's red and black phases, Section 3.1).
//
// One warp owns a strip of 128 packed columns (4 per lane) and a segment of
// output rows, and streams down the rows once.  At step s it stages row s + 1
// of both colours (asynchronous copies into a per-warp ring in shared memory,
// fetched kWfAhead rows ahead) and then runs all 2T colour phases, phase p on
// row s - p + 1: phase 1 is the red phase of the first iteration, phase 2 its
// black phase, and so on.  Phase p needs the other colour after phase p - 1 on
// rows r - 1, r, r + 1 (the last of them produced by phase p - 1 in this very
// step) and its own colour after phase p - 2 on row r; each phase level keeps
// the last three rows it produced in registers, so a cell update reads no
// memory at all: N and S from registers, W and E from registers plus one
// shuffle per row, the old value from registers.  Every phase of a step
// works on a row of parity (row + colour) & 1 = s & 1, so unrolling six steps
// (the rotation of three rows times the two parities) fixes every register
// index and every shuffle direction at compile time.
//
// Each update is the exact one of the oracle,
//   U <- (1-w)*U + (w/4)*( ((U_N + U_S) + (U_W + U_E)) + g ),
// every product and sum rounded on its own, and the updates of one colour
// are independent (Section 3.1), so the result equals the phase-by-phase
// iteration bit for bit.  Cells near the strip's side edges lack a neighbour
// and go stale, the stale band growing by at most half a packed column per
// phase; HQ >= T + 1 halo columns on each side keep it out of the 128 - 2 HQ
// output columns.  A segment's rows need no halo tile: the 2T - p rows above
// and below that phase p must still update are computed on the way in and
// out of the segment.  The iterate is read from one buffer of a ping-pong
// pair and the output written to the other, so neighbouring strips keep
// reading the previous iterate.
#include <cuda_runtime.h>

#include "sor_devfn.cuh"
#include "sor_device.cuh"
#include "sor_kernels.h"

namespace sorgb {

constexpr int kWfThreads = 128;
constexpr int kWfWarps = kWfThreads / 32;
constexpr int kWfRing = 6;   // staged rows per warp: the unrolled period, so every slot index is a constant
constexpr int kWfAhead = 4;  // rows fetched ahead of the newest row in use (kWfRing - 2)

template <int T>
struct WfGeom {
  static constexpr int HQ = T <= 3 ? 4 : 8;  // halo packed columns of a tile table built for depth T
                                             // (a multiple of 4, >= T + 1; a launch of fewer iterations
                                             // may use a table built for a larger depth)
  static constexpr int OQ = 128 - 2 * HQ;    // output packed columns of a strip
  static constexpr int P = 2 * T;            // phases of a launch
  // resident blocks of 4 warps per SM: the registers of the 2T + 1 phase
  // levels (3 rows of 4 cells each) set how many warps fit
  static constexpr int kMinBlocks = T <= 2 ? 4 : (T <= 4 ? 3 : 2);
};

// Shared memory of a block: per warp, kWfRing rows x 2 colours x 128 floats.
constexpr size_t kWfSmem = (size_t)kWfWarps * kWfRing * 2 * 128 * sizeof(float);

__device__ __forceinline__ void wf_cp_async16(float* smem_dst, const float* gsrc, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int nbytes = valid ? 16 : 0;  // src-size 0 fills the 16 bytes with zeros and reads nothing
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(valid ? gsrc : nullptr),
               "r"(nbytes)
               : "memory");
}

template <int N>
__device__ __forceinline__ void wf_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// New values of this lane's 4 cells of one row: om / oc / op the other
// colour's rows r - 1, r, r + 1, own the cell's previous values, gv its right
// side.  S (the row parity) decides which single neighbour comes from the
// adjacent lane: S == 0: the east one of the last cell, S == 1: the west one of
// the first.  m: cells to update (bit v: packed column qf + v); the others
// keep their value.  Lane 0's west and lane 31's east neighbour are wrong:
// those cells are inside the stale halo.
template <int S, bool HAS_G, bool FAST>
__device__ __forceinline__ void wf_cells(const float (&om)[4], const float (&oc)[4], const float (&op)[4],
                                         const float (&own)[4], const float (&gv)[4], unsigned m, float a, float b,
                                         float (&nv)[4]) {
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
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float sum = radd(radd(om[v], op[v]), radd(W[v], E[v]));
    if (HAS_G) sum = radd(sum, gv[v]);
    const float nu = radd(rmul(a, own[v]), rmul(b, sum));
    nv[v] = (FAST || ((m >> v) & 1u)) ? nu : own[v];
  }
}

// Stores the cells of this lane's 4 whose bit is set in m, without a branch:
// one 16-byte store when all four are set, else one 4-byte store per set bit
// (only lanes at a ring or padding column have some but not all set).
__device__ __forceinline__ void wf_store_row(float* dst, const float (&v)[4], unsigned m) {
  asm volatile(
      "{\n"
      " .reg .pred pf, p0, p1, p2, p3;\n"
      " .reg .b32 t;\n"
      " setp.eq.u32 pf, %5, 15;\n"
      " @pf st.global.v4.f32 [%0], {%1, %2, %3, %4};\n"
      " selp.b32 t, 0, %5, pf;\n"
      " and.b32 t, t, 1;\n setp.ne.u32 p0, t, 0;\n"
      " selp.b32 t, 0, %5, pf;\n"
      " and.b32 t, t, 2;\n setp.ne.u32 p1, t, 0;\n"
      " selp.b32 t, 0, %5, pf;\n"
      " and.b32 t, t, 4;\n setp.ne.u32 p2, t, 0;\n"
      " selp.b32 t, 0, %5, pf;\n"
      " and.b32 t, t, 8;\n setp.ne.u32 p3, t, 0;\n"
      " @p0 st.global.f32 [%0], %1;\n"
      " @p1 st.global.f32 [%0+4], %2;\n"
      " @p2 st.global.f32 [%0+8], %3;\n"
      " @p3 st.global.f32 [%0+12], %4;\n"
      "}\n" ::"l"(dst),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "r"(m)
      : "memory");
}

// Everything a warp needs about its current tile.
struct WfTile {
  float* ring;                   // this warp's staging ring
  const float* x0;               // source iterate, red / black
  const float* x1;
  float* y0;                     // destination iterate, red / black
  float* y1;
  const float* g0;               // right side, red / black (HAS_G)
  const float* g1;
  int n, pitch, e, lane;
  int a, a_end;                  // output rows [a, a_end)
  int nt2;                       // phases that update (2 x iterations of this launch)
  int meas_lo;                   // first measured phase (> 2T: none)
  bool zero;                     // the iterate starts at 0 (first sweeps of a correction)
  bool gok;                      // this lane's 4 columns lie inside the row (right-side loads)
  bool fetch_ok;                 // ... and the iterate is read (not a zero start)
  unsigned in0, in1;             // interior cells for row parity 0 / 1
  unsigned out0, out1;           // interior cells inside the output columns, parity 0 / 1
  float a32, b32;
};

// Running addresses of a tile: the next row to stage and the two rows the
// current step finishes (advanced by one row per step).
struct WfRun {
  const float* fx0;  // row frow of the source iterate, this lane's columns: red / black
  const float* fx1;
  int frow;
  float* py0;        // red row s - 2T + 2 of the destination
  float* py1;        // black row s - 2T + 1 of the destination
};

// Stage row w.frow of both colours into ring slot SL as one commit group
// (rows outside the array, columns outside the row and zero starts read as 0),
// then advance to the next row.
template <int SL>
__device__ __forceinline__ void wf_fetch(const WfTile& t, WfRun& w) {
  const bool valid = t.fetch_ok && w.frow >= 0 && w.frow <= t.n + 1;
  wf_cp_async16(t.ring + (SL * 2 + 0) * 128 + 4 * t.lane, w.fx0, valid);
  wf_cp_async16(t.ring + (SL * 2 + 1) * 128 + 4 * t.lane, w.fx1, valid);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  w.fx0 += t.pitch;
  w.fx1 += t.pitch;
  ++w.frow;
}

// Step s of the wavefront, K = s mod 6: stage row s + 1 + kWfAhead, take the
// black row s + 1 and the red row s from the ring, run phases 1 .. 2T on rows
// s .. s - 2T + 1, store the two finished rows.  lv[q][slot]: rows produced
// by phase q (q = 0: the black input rows), slot = producing step mod 3; the
// ring slot of row r is r mod 6.
// FAST tiles (all 128 staged columns interior, every row any phase computes
// inside 1 .. n, all T iterations run) update every cell; the others compute
// each phase on its whole row and keep, per cell, the cells that must not
// change (a phase past the slot's iterations, a ring or outside row, a row
// above those the output needs, a ring or padding column).  Either way no
// branch surrounds a shuffle, so the shuffles and loads of later phases can
// be issued early.
template <int T, bool HAS_G, bool FAST, int K>
__device__ __forceinline__ void wf_step(const WfTile& t, WfRun& w, float (&lv)[2 * T + 1][3][4], int s,
                                        unsigned& dm32) {
  constexpr int S = K & 1;        // parity (row + colour) & 1 of every phase of this step
  constexpr int c0 = K % 3;       // slot of the rows produced at this step
  constexpr int c1 = (K + 2) % 3; // ... at the previous step
  constexpr int c2 = (K + 1) % 3; // ... two steps ago
  wf_fetch<(K + 1 + kWfAhead) % kWfRing>(t, w);
  wf_wait<kWfAhead>();  // row s + 1 has arrived
  load4(t.ring + (((K + 1) % kWfRing) * 2 + 1) * 128 + 4 * t.lane, lv[0][c0]);
  float r0[4];
  load4(t.ring + ((K % kWfRing) * 2 + 0) * 128 + 4 * t.lane, r0);
  const unsigned m = S ? t.in1 : t.in0;
  const unsigned mo = S ? t.out1 : t.out0;
#pragma unroll
  for (int p = 1; p <= 2 * T; ++p) {
    const int r = s - p + 1;
    float own[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) own[v] = p == 1 ? r0[v] : lv[p >= 2 ? p - 2 : 0][c2][v];
    unsigned mp = 0xFu;
    if (!FAST) mp = (p <= t.nt2 && r >= max(1, t.a - (2 * T - p)) && r <= t.n) ? m : 0u;
    float gv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (HAS_G && (FAST || (t.gok && r >= 1 && r <= t.n))) {
      const float* gp = ((p & 1) ? t.g0 : t.g1) + (ptrdiff_t)r * t.pitch + t.e;
      const float4 g4 = __ldg(reinterpret_cast<const float4*>(gp));
      gv[0] = g4.x; gv[1] = g4.y; gv[2] = g4.z; gv[3] = g4.w;
    }
    wf_cells<S, HAS_G, FAST>(lv[p - 1][c2], lv[p - 1][c1], lv[p - 1][c0], own, gv, mp, t.a32, t.b32, lv[p][c0]);
    // max |change| of the measured iteration (FAST: its two phases are the last two)
    if ((!FAST || p >= 2 * T - 1) && p >= t.meas_lo && r >= t.a && r < t.a_end) {
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if ((mo >> v) & 1u) dm32 = max(dm32, abs_bits32(radd(lv[p][c0][v], -own[v])));
    }
  }
  const int rr = s - 2 * T + 2;  // red row finished by phase 2T - 1
  const int rb = s - 2 * T + 1;  // black row finished by phase 2T
  wf_store_row(w.py0, lv[2 * T - 1][c0], (rr >= t.a && rr < t.a_end) ? mo : 0u);
  wf_store_row(w.py1, lv[2 * T][c0], (rb >= t.a && rb < t.a_end) ? mo : 0u);
  w.py0 += t.pitch;
  w.py1 += t.pitch;
}

// Prologue for a tile whose first step has s0 mod 6 == K0: stage rows
// s0 - 1 .. s0 + kWfAhead (ring slots (s0 - 1) mod 6 ..) and load the black
// rows s0 - 1 and s0, produced "two steps" and "one step" before the first.
template <int T, int K0>
__device__ __forceinline__ void wf_prologue(const WfTile& t, WfRun& w, float (&lv)[2 * T + 1][3][4]) {
  wf_fetch<(K0 + 5) % kWfRing>(t, w);
  wf_fetch<(K0 + 0) % kWfRing>(t, w);
  wf_fetch<(K0 + 1) % kWfRing>(t, w);
  wf_fetch<(K0 + 2) % kWfRing>(t, w);
  wf_fetch<(K0 + 3) % kWfRing>(t, w);
  wf_fetch<(K0 + 4) % kWfRing>(t, w);
  wf_wait<kWfAhead>();  // rows s0 - 1 and s0 have arrived
  load4(t.ring + (((K0 + 5) % kWfRing) * 2 + 1) * 128 + 4 * t.lane, lv[0][(K0 + 1) % 3]);
  load4(t.ring + ((K0 % kWfRing) * 2 + 1) * 128 + 4 * t.lane, lv[0][(K0 + 2) % 3]);
}

// The whole tile: steps s0 .. s_last, entered at the unrolled step that
// matches s0 mod 6.
template <int T, bool HAS_G, bool FAST>
__device__ __forceinline__ void wf_tile(const WfTile& t, unsigned& dm32) {
  float lv[2 * T + 1][3][4];
#pragma unroll
  for (int q = 0; q <= 2 * T; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int v = 0; v < 4; ++v) lv[q][k][v] = 0.0f;
  const int s0 = t.a - 2 * T + 1;          // first row phase 1 must update
  const int s_last = t.a_end + 2 * T - 2;  // phase 2T finishes row a_end - 1 there
  const int K0 = ((s0 % kWfRing) + kWfRing) % kWfRing;
  WfRun w;
  w.frow = s0 - 1;
  w.fx0 = t.x0 + (ptrdiff_t)(s0 - 1) * t.pitch + t.e;
  w.fx1 = t.x1 + (ptrdiff_t)(s0 - 1) * t.pitch + t.e;
  w.py0 = t.y0 + (ptrdiff_t)(s0 - 2 * T + 2) * t.pitch + t.e;
  w.py1 = t.y1 + (ptrdiff_t)(s0 - 2 * T + 1) * t.pitch + t.e;
  switch (K0) {
    case 0: wf_prologue<T, 0>(t, w, lv); break;
    case 1: wf_prologue<T, 1>(t, w, lv); break;
    case 2: wf_prologue<T, 2>(t, w, lv); break;
    case 3: wf_prologue<T, 3>(t, w, lv); break;
    case 4: wf_prologue<T, 4>(t, w, lv); break;
    default: wf_prologue<T, 5>(t, w, lv); break;
  }
  int s = s0;
  switch (K0) {
    case 0:
      do {
        wf_step<T, HAS_G, FAST, 0>(t, w, lv, s, dm32);
        if (++s > s_last) break;
        case 1:
        wf_step<T, HAS_G, FAST, 1>(t, w, lv, s, dm32);
        if (++s > s_last) break;
        case 2:
        wf_step<T, HAS_G, FAST, 2>(t, w, lv, s, dm32);
        if (++s > s_last) break;
        case 3:
        wf_step<T, HAS_G, FAST, 3>(t, w, lv, s, dm32);
        if (++s > s_last) break;
        case 4:
        wf_step<T, HAS_G, FAST, 4>(t, w, lv, s, dm32);
        if (++s > s_last) break;
        default:
        wf_step<T, HAS_G, FAST, 5>(t, w, lv, s, dm32);
        ++s;
      } while (s <= s_last);
  }
  wf_wait<0>();  // the rows fetched past the segment land before the ring is reused
}

// MODE 0: plain FP32 iterations on x (right side g optional), source buffer
//         from the slot state; the last iteration of the launch may be a
//         measured one (max |change| over the output cells).
// MODE 1: inner sweeps of defect correction on d with right side r~; `src`
//         is the buffer holding d (the first launch of a correction,
//         sweep0 == 0, starts from d = 0 and reads nothing).
// One warp per tile of the tile table (a segment of output rows of one
// strip); the tiles of one slot in a launch partition its interior.  T is the
// number of iterations of the launch; the table may have been built for a
// larger depth: hq is its halo (staged columns 0 .. 127 start hq columns left
// of a tile's first output column, 128 - 2 hq output columns), hq >= T + 1.
template <int T, int MODE>
__global__ void __launch_bounds__(kWfThreads, WfGeom<T>::kMinBlocks)
    k_sweep_wf(const SlotDesc* __restrict__ slots, SlotState* states, const Tile* __restrict__ tiles, int ntiles,
               int nt_req, int src_param, int sweep0, int hq) {
  extern __shared__ __align__(16) float wf_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* const ring = wf_smem + (size_t)warp * kWfRing * 2 * 128;
  for (int ti = blockIdx.x * kWfWarps + warp; ti < ntiles; ti += gridDim.x * kWfWarps) {
    const Tile tl = tiles[ti];
    const SlotDesc& sd = slots[tl.slot];
    SlotState* st = states + tl.slot;
    int skip = 0, nt = 0, k_end = 0, measure = 0, src = 0;
    if (lane == 0) {
      skip = *((volatile int*)&st->done);
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
      } else {
        nt = min(nt_req, sd.inner - sweep0);
        src = src_param;
      }
      if (nt <= 0) skip = 1;
      // the output rows and columns of the tile lie inside the slot's arrays
      if (!skip && !dbg_tile(sd, st, tl.row0, tl.row0 + tl.nrows, tl.col0, tl.col0 + 128 - 2 * hq)) skip = 1;
    }
    skip = __shfl_sync(0xffffffffu, skip, 0);
    if (skip) continue;
    nt = __shfl_sync(0xffffffffu, nt, 0);
    k_end = __shfl_sync(0xffffffffu, k_end, 0);
    measure = __shfl_sync(0xffffffffu, measure, 0);
    src = __shfl_sync(0xffffffffu, src, 0);

    WfTile t;
    const int n = sd.n, pitch = sd.pitch;
    const int q0 = tl.col0 - hq;  // first staged packed column (q0 + kOff is a multiple of 4)
    t.ring = ring;
    t.n = n;
    t.pitch = pitch;
    t.lane = lane;
    t.e = q0 + kOff + 4 * lane;
    t.x0 = (const float*)sd.x[src][0];
    t.x1 = (const float*)sd.x[src][1];
    t.y0 = (float*)sd.x[src ^ 1][0];
    t.y1 = (float*)sd.x[src ^ 1][1];
    t.g0 = (const float*)sd.g[0];
    t.g1 = (const float*)sd.g[1];
    t.a = tl.row0;
    t.a_end = tl.row0 + tl.nrows;
    t.nt2 = 2 * nt;
    t.meas_lo = (MODE == 0 && measure) ? 2 * nt - 1 : (1 << 20);
    t.zero = (MODE == 1) && sweep0 == 0;
    t.gok = t.e >= 0 && t.e + 4 <= pitch;
    t.fetch_ok = t.gok && !t.zero;
    t.in0 = t.in1 = t.out0 = t.out1 = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int q = q0 + 4 * lane + v;
      const unsigned i0 = (unsigned)(q >= 1 && q <= (n >> 1));
      const unsigned i1 = (unsigned)(q >= 1 && q <= ((n + 1) >> 1));
      const unsigned oc = (unsigned)(q >= tl.col0 && q < tl.col0 + 128 - 2 * hq);
      t.in0 |= i0 << v;
      t.in1 |= i1 << v;
      t.out0 |= (i0 & oc) << v;
      t.out1 |= (i1 & oc) << v;
    }
    t.a32 = sd.a32;
    t.b32 = sd.b32;
    // FAST: all 128 staged columns interior for both row parities, every row a
    // phase computes (s0 - 2T + 1 .. s_last, see wf_tile) inside 1 .. n, and
    // all T iterations run for this slot
    const bool fast = q0 >= 1 && q0 + 127 <= (n >> 1) && t.a - 4 * T + 2 >= 1 && t.a_end + 2 * T - 2 <= n && nt == T;
    unsigned dm32 = 0;
    if (t.g0 || MODE == 1) {
      if (fast) wf_tile<T, true, true>(t, dm32); else wf_tile<T, true, false>(t, dm32);
    } else {
      if (fast) wf_tile<T, false, true>(t, dm32); else wf_tile<T, false, false>(t, dm32);
    }

    if (MODE == 0) {
      if (measure) {
        const unsigned dmw = __reduce_max_sync(0xffffffffu, dm32);
        if (lane == 0 && dmw) atomicMax(&st->dmax_bits, abs_bits_of(__uint_as_float(dmw)));
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        if (prev == (unsigned)sd.sweep_tiles - 1u) {
          __threadfence();
          st->xbuf = src ^ 1;
          finalize_plain(sd, st, k_end, measure);
        }
      }
    }
  }
}

template <int T, int MODE>
static cudaError_t launch_wf_t(const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles, int grid,
                               int nt, int src, int sweep0, int hq, cudaStream_t s) {
  static bool attr_set = false;  // benign race: setting the attribute twice is harmless
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_sweep_wf<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWfSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int blocks = (ntiles + kWfWarps - 1) / kWfWarps;
  if (grid <= 0 || grid > blocks) grid = blocks;
  count_kernel_launches(1);
  k_sweep_wf<T, MODE><<<grid, kWfThreads, kWfSmem, s>>>(slots, states, tiles, ntiles, nt, src, sweep0, hq);
  return cudaGetLastError();
}

bool wave_depth_supported(int T) { return T >= 2 && T <= 5; }

int wave_out_cols(int T) { return 128 - 2 * (T <= 3 ? WfGeom<3>::HQ : WfGeom<5>::HQ); }

int wave_warps_per_sm(int T) {
  return kWfWarps * (T <= 2 ? WfGeom<2>::kMinBlocks : (T <= 4 ? WfGeom<4>::kMinBlocks : WfGeom<5>::kMinBlocks));
}

// Output rows per tile of one plate solved alone: about one tile per
// resident warp of the GPU (strips x segments ~ SMs x warps per SM), at
// least 16 rows (a segment recomputes 2T - 1 rows of phases above and below
// it) and at most 256.
int wave_seg_rows(int n, int T, int sm_count) {
  const int qmax = (n + 1) / 2;
  const int strips = (qmax + wave_out_cols(T) - 1) / wave_out_cols(T);
  const long long warps = (long long)(sm_count > 0 ? sm_count : 1) * wave_warps_per_sm(T);
  long long seg = ((long long)n * strips + warps - 1) / warps;
  if (seg < 16) seg = 16;
  if (seg > 256) seg = 256;
  if (seg > n) seg = n;
  return (int)seg;
}

// Opts every kernel a launch of a depth-T table may use (1 .. T iterations)
// into its shared memory.
cudaError_t wave_prepare(int T) {
  cudaError_t e = cudaSuccess;
#define WF_PREP(TT)                                                                                        \
  if (e == cudaSuccess && TT <= T)                                                                         \
    e = cudaFuncSetAttribute(k_sweep_wf<TT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWfSmem);  \
  if (e == cudaSuccess && TT <= T)                                                                         \
    e = cudaFuncSetAttribute(k_sweep_wf<TT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWfSmem);
  WF_PREP(1) WF_PREP(2) WF_PREP(3) WF_PREP(4) WF_PREP(5)
#undef WF_PREP
  return e;
}

// A launch of nt <= T iterations over a tile table built for depth T runs the
// kernel compiled for nt iterations with the table's halo.
cudaError_t launch_sweep_wave(bool inner, int T, const SlotDesc* slots, SlotState* states, const Tile* tiles,
                              int ntiles, int grid, int nt, int src, int sweep0, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (!wave_depth_supported(T) || nt < 1 || nt > T) return cudaErrorInvalidValue;
  const int hq = (128 - wave_out_cols(T)) / 2;
  switch (nt) {
#define WF_CASE(TT)                                                                                          \
  case TT:                                                                                                   \
    return inner ? launch_wf_t<TT, 1>(slots, states, tiles, ntiles, grid, nt, src, sweep0, hq, s)             \
                 : launch_wf_t<TT, 0>(slots, states, tiles, ntiles, grid, nt, src, sweep0, hq, s);
    WF_CASE(1) WF_CASE(2) WF_CASE(3) WF_CASE(4) WF_CASE(5)
#undef WF_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sorgb
