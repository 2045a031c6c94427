// Whole solves of small plates on a cooperative grid spanning many SMs.
//
// Algorithm 1 runs to the end inside one launch: each block owns a band of
// rows of both colour arrays in shared memory (plus a ghost row above and
// below), updates its band in the red phase, publishes the two edge rows it
// changed to the slot's global arrays, waits at a grid-wide barrier (the
// phase barrier of Section 3.2), reads its neighbours' edge rows into its
// ghost rows, and does the same for the black phase.  On tested iterations
// every block adds its largest |change| to a grid-wide maximum (Section 2.1)
// before the second barrier, and all blocks take the same stop decision from
// it after the barrier (Section 3.3).  A thread-block cluster (sor_cluster.cu)
// does the same within 16 SMs with hardware barriers, and is then bound by
// their FP64 rate; spreading a small plate over many SMs makes the phases
// short and leaves the barriers as the cost.
//
// The update is the exact-order form of k_sweep (every product and sum
// rounded on its own), so results equal the oracle bit for bit.  The
// barrier's waits are bounded: a block that waits too long records an error
// in the slot state and leaves, and so do the others after their own waits
// run out; the launch is cooperative, so every block is resident and a wait
// can only run out if a block stopped.
#include <cuda_runtime.h>

#include <algorithm>

#include "sor_devfn.cuh"
#include "sor_kernels.h"

namespace sorgb {

constexpr int kGridThreads = 256;
constexpr int kGridWarps = kGridThreads / 32;
constexpr int kGridSpins = 1 << 22;  // barrier polls of about 50 ns: far above any phase

// Grid-wide state of one launch (zeroed before it).
struct GridSync {
  unsigned count;                   // arrivals at the current barrier
  unsigned gen;                     // barriers passed
  unsigned long long dmax_bits[2];  // max |change| of the current tested iteration, alternating by parity
};

__device__ __forceinline__ unsigned grid_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier with a bounded wait; false on every thread of the block when
// this block's wait ran out.  Writes before it are visible after it.
__device__ __forceinline__ bool grid_barrier(GridSync* gs, unsigned& gen, unsigned nblocks) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned g = gen;
    if (atomicAdd(&gs->count, 1u) == nblocks - 1u) {
      atomicExch(&gs->count, 0u);  // nobody arrives at the next barrier before the release below
      __threadfence();
      atomicExch(&gs->gen, g + 1u);
    } else {
      int spins = 0;
      while (grid_ld_acquire(&gs->gen) == g) {
        if (++spins > kGridSpins) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    gen = g + 1u;
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Loads `count` elements of a global row that another block wrote before the
// last barrier, bypassing this SM's L1 (which may hold an older copy).
template <typename T>
__device__ __forceinline__ void grid_load_row(T* dst, const T* src, int count) {
  for (int e = threadIdx.x; e < count; e += blockDim.x) dst[e] = __ldcg(src + e);
}

template <typename T>
__global__ void __launch_bounds__(kGridThreads) k_grid_solve(const SlotDesc* __restrict__ slots, SlotState* states,
                                                             int slot, GridSync* gs) {
  extern __shared__ __align__(16) unsigned char gsm[];
  __shared__ unsigned long long wmax[kGridWarps];
  const SlotDesc& sd = slots[slot];
  SlotState* st = states + slot;
  const unsigned B = gridDim.x;
  const int n = sd.n, pitch = sd.pitch, m = n + 2;
  const int R = (m + (int)B - 1) / (int)B;  // rows per band
  const int rlo = min(m, (int)blockIdx.x * R), rhi = min(m, rlo + R);
  const int nr = rhi - rlo;
  // local row lr holds grid row rlo - 1 + lr: lr = 0 and lr = nr + 1 are the ghosts
  T* const S0 = (T*)gsm;
  T* const S1 = (T*)gsm + (size_t)(R + 2) * pitch;
  const int xbuf = st->xbuf;
  T* const X0 = (T*)sd.x[xbuf][0];
  T* const X1 = (T*)sd.x[xbuf][1];
  const bool ok_geom = dbg_range((long long)(rlo - 1 < 0 ? 0 : rlo - 1) * pitch,
                                 (long long)(rhi + 1 > m ? m : rhi + 1) * pitch, (long long)m * pitch, st);
  for (int idx = threadIdx.x; ok_geom && idx < 2 * (nr + 2) * pitch; idx += blockDim.x) {
    const int c = idx / ((nr + 2) * pitch);
    const int e = idx - c * (nr + 2) * pitch;
    const int r = rlo - 1 + e / pitch;
    if (r >= 0 && r < m) (c ? S1 : S0)[e] = (c ? X1 : X0)[(long long)(rlo - 1) * pitch + e];
  }
  __syncthreads();

  const T a = sizeof(T) == 4 ? (T)sd.a32 : (T)sd.a64;
  const T b = sizeof(T) == 4 ? (T)sd.b32 : (T)sd.b64;
  const int r_first = max(rlo, 1), r_last = min(rhi, n + 1);  // interior rows of the band
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned gen = 0;
  int k = st->iters, converged = 0, failed = ok_geom ? 0 : 1;
  double last_dmax = st->last_dmax;

  while (!failed && k < sd.max_iters) {
    ++k;
    const bool measure = (k % sd.K) == 0 || k >= sd.max_iters;
    unsigned long long dm = 0;
    unsigned dm32 = 0;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      T* Sc = c ? S1 : S0;
      const T* So = c ? S0 : S1;
      const T* Gc = (const T*)sd.g[c];
      for (int row = r_first + warp; row < r_last; row += kGridWarps) {
        const int s = (row + c) & 1;
        const int qlim = (n + s) >> 1;
        const size_t lb = (size_t)(row - rlo + 1) * pitch + kOff;
        for (int q = 1 + lane; q <= qlim; q += 32) {
          const size_t le = lb + q;
          const T own = Sc[le];
          T sum = radd(radd(So[le - pitch], So[le + pitch]), radd(So[le - s], So[le - s + 1]));
          if (Gc) sum = radd(sum, Gc[(size_t)row * pitch + q + kOff]);
          const T nu = radd(rmul(a, own), rmul(b, sum));
          Sc[le] = nu;
          if (measure) {
            if (sizeof(T) == 4)
              dm32 = max(dm32, abs_bits32((float)radd(nu, -own)));
            else
              dm = umax64(dm, abs_bits((double)radd(nu, -own)));
          }
        }
      }
      __syncthreads();
      // publish the band's first and last rows of colour c (interior rows only)
      T* Xc = c ? X1 : X0;
      if (nr > 0 && rlo >= 1 && rlo <= n)
        for (int e = threadIdx.x; e < pitch; e += blockDim.x) Xc[(size_t)rlo * pitch + e] = Sc[(size_t)pitch + e];
      if (nr > 1 && rhi - 1 >= 1 && rhi - 1 <= n)
        for (int e = threadIdx.x; e < pitch; e += blockDim.x)
          Xc[(size_t)(rhi - 1) * pitch + e] = Sc[(size_t)nr * pitch + e];
      if (c == 1 && measure) {  // this block's largest change of the iteration into the grid-wide maximum
        if (sizeof(T) == 4) dm = abs_bits_of(__uint_as_float(dm32));
        dm = warp_max64(dm);
        if (lane == 0) wmax[warp] = dm;
        __syncthreads();
        if (threadIdx.x == 0) {
          unsigned long long mm = 0;
          for (int w = 0; w < kGridWarps; ++w) mm = umax64(mm, wmax[w]);
          if (mm) atomicMax(&gs->dmax_bits[k & 1], mm);
        }
      }
      if (!grid_barrier(gs, gen, B)) {
        failed = 1;
        break;
      }
      if (c == 0 && blockIdx.x == 0 && threadIdx.x == 0)
        gs->dmax_bits[(k + 1) & 1] = 0;  // every block read it last iteration, before this barrier
      // the neighbours' edge rows of colour c into this band's ghost rows
      if (rlo - 1 >= 1 && rlo - 1 <= n) grid_load_row(Sc, Xc + (size_t)(rlo - 1) * pitch, pitch);
      if (rhi <= n) grid_load_row(Sc + (size_t)(nr + 1) * pitch, Xc + (size_t)rhi * pitch, pitch);
      __syncthreads();
    }
    if (failed) break;
    if (measure) {
      last_dmax = bits_to_double(__ldcg(&gs->dmax_bits[k & 1]));
      if (sd.stop == kStopDelta && (k % sd.K) == 0 && last_dmax < sd.tol) {
        converged = 1;
        break;
      }
    }
  }
  // write the band back (its interior rows; the ring never changes)
  for (int idx = threadIdx.x; idx < 2 * nr * pitch; idx += blockDim.x) {
    const int c = idx / (nr * pitch);
    const int e = idx - c * nr * pitch;
    const int r = rlo + e / pitch;
    if (r >= 1 && r <= n) (c ? X1 : X0)[(size_t)rlo * pitch + e] = (c ? S1 : S0)[(size_t)pitch + e];
  }
  if (threadIdx.x == 0) {
    if (failed) {  // any block that gave up (the others then give up at their next barrier)
      atomicExch(&st->error, ok_geom ? 1 : kErrBounds);
      st->done = 1;
    } else if (blockIdx.x == 0) {
      st->iters = k;
      st->converged = converged;
      st->done = 1;
      st->last_dmax = last_dmax;
    }
  }
}

// Blocks of the grid for an n x n plate: bands of at least 4 rows, at most
// the blocks that can be resident at once.
template <typename T>
static int grid_blocks(int n, int sm_count, size_t* smem_out, int pitch) {
  static int per_sm = -1;
  const int m = n + 2;
  int B = std::max(1, m / 4);
  const int R = (m + B - 1) / B;
  const size_t smem = 2ull * (R + 2) * pitch * sizeof(T);
  if (per_sm < 0) {
    if (cudaFuncSetAttribute(k_grid_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_solve<T>, kGridThreads, 96 * 1024) !=
            cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
  }
  *smem_out = smem;
  if (per_sm <= 0 || smem > 96 * 1024) return 0;
  return std::min(B, sm_count * per_sm);
}

bool grid_solve_fits(bool fp32, int n, int pitch, int sm_count) {
  size_t smem = 0;
  const int B = fp32 ? grid_blocks<float>(n, sm_count, &smem, pitch) : grid_blocks<double>(n, sm_count, &smem, pitch);
  if (B <= 0) return false;
  // the bands must cover the plate with the blocks that can be resident
  const int m = n + 2;
  const int R = (m + B - 1) / B;
  return 2ull * (R + 2) * pitch * (fp32 ? 4 : 8) <= 96 * 1024;
}

size_t grid_sync_bytes() { return sizeof(GridSync); }

cudaError_t launch_grid_solve(bool fp32, int n, int pitch, int sm_count, const SlotDesc* slots, SlotState* states,
                              int slot, void* sync, cudaStream_t s) {
  size_t smem = 0;
  const int B = fp32 ? grid_blocks<float>(n, sm_count, &smem, pitch) : grid_blocks<double>(n, sm_count, &smem, pitch);
  if (B <= 0) return cudaErrorInvalidValue;
  const int m = n + 2;
  const int R = (m + B - 1) / B;
  smem = 2ull * (R + 2) * pitch * (fp32 ? 4 : 8);
  if (smem > 96 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(GridSync), s);
  if (e != cudaSuccess) return e;
  GridSync* gs = (GridSync*)sync;
  void* args[] = {(void*)&slots, (void*)&states, (void*)&slot, (void*)&gs};
  count_kernel_launches(1);
  return fp32 ? cudaLaunchCooperativeKernel((const void*)k_grid_solve<float>, dim3(B), dim3(kGridThreads), args,
                                            smem, s)
              : cudaLaunchCooperativeKernel((const void*)k_grid_solve<double>, dim3(B), dim3(kGridThreads), args,
                                            smem, s);
}


// ------------------------------------------------------------------------------------------------
// The same solves without grid barriers
// ------------------------------------------------------------------------------------------------
//
// k_grid_flow computes exactly the iterations of k_grid_solve (same bands,
// same exact-order update) with both barriers of an iteration replaced:
// * Edge rows travel as tagged words.  Each value of a band's first and last
//   interior rows is stored together with the number of the phase that
//   produced it in one 64-bit word (an FP64 value as two words, high and low
//   half), so a neighbour that reads a word carrying the phase it expects
//   holds that phase's value, with no fence or flag in between.  A band reads
//   its neighbours' words of phase p before it publishes phase p + 1, and
//   writes its own words of phase p + 2 only after reading its neighbours'
//   phase p + 1, so no word is overwritten before it has been read.
// * The stop test (Section 2.1) runs behind the sweeps.  At the end of each
//   tested iteration every band keeps a copy of its rows and posts its
//   largest |change| as tagged words; one more block, the arbiter, collects
//   the posts of each tested iteration in order and posts the decision (stop
//   or go on) with the grid-wide maximum.  A band runs on while decisions are
//   pending, at most kFlowDepth tested iterations ahead of the last decision
//   it has read; when a decision says stop, every band returns to its copy of
//   that iteration.  Iteration count, stop iteration, last max|change| and
//   solution are those of Algorithm 1 exactly.
// * Every wait is bounded and also watches an abort word: a block whose wait
//   runs out sets it and marks its edge words with kTagDone, which ends every
//   wait on them, so the others stop in turn and the solve reports an error.
//   A band that stops normally marks its edge words the same way, so a
//   neighbour that has run ahead never waits for it; that neighbour only
//   computes iterations it will discard.
//
// Sync buffer (8-byte words, zeroed before the launch): [0, 16) abort word;
// xch: per band, colour and edge (top / bottom) the qmax values of packed
// columns 1 .. qmax; post: per ring slot and band, its largest |change| as
// two tagged words; dec: per ring slot the decision, as three tagged words
// (stop / converged flags, then the maximum's high and low halves).

constexpr int kFlowDepth = 4;                // tested iterations a band may run ahead of the decisions it has read
constexpr int kFlowRing = 8;                 // slots of the post and decision rings (> kFlowDepth)
constexpr unsigned kTagDone = 0xFFFFFFFFu;   // edge words of a band that has stopped: ends every wait on them
constexpr long long kGridFlowSpins = 1ll << 22;  // polls of a wait for a neighbour's phase or for a decision
constexpr int kFlowThreads = 256;

__device__ __forceinline__ unsigned long long flow_ld(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void flow_st(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long flow_word(unsigned tag, unsigned payload) {
  return ((unsigned long long)tag << 32) | payload;
}
__device__ __forceinline__ bool flow_tag_ok(unsigned long long w, unsigned tag) {
  const unsigned t = (unsigned)(w >> 32);
  return t == tag || t == kTagDone;
}

// One value as tagged words: FP32 in one word, FP64 as its high and low halves.
template <typename T>
struct FlowVal;
template <>
struct FlowVal<float> {
  static constexpr int W = 1;
  __device__ static void put(unsigned long long* p, unsigned tag, float v) {
    flow_st(p, flow_word(tag, __float_as_uint(v)));
  }
  __device__ static bool get(const unsigned long long* p, unsigned tag, float& v) {
    const unsigned long long w = flow_ld(p);
    if (!flow_tag_ok(w, tag)) return false;
    v = __uint_as_float((unsigned)w);
    return true;
  }
};
template <>
struct FlowVal<double> {
  static constexpr int W = 2;
  __device__ static void put(unsigned long long* p, unsigned tag, double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    flow_st(p, flow_word(tag, (unsigned)(b >> 32)));
    flow_st(p + 1, flow_word(tag, (unsigned)b));
  }
  __device__ static bool get(const unsigned long long* p, unsigned tag, double& v) {
    const unsigned long long w0 = flow_ld(p), w1 = flow_ld(p + 1);
    if (!flow_tag_ok(w0, tag) || !flow_tag_ok(w1, tag)) return false;
    v = __longlong_as_double((long long)((w0 << 32) | (w1 & 0xffffffffull)));
    return true;
  }
};

// Word offsets of the sync buffer's parts for B bands of a plate with qmax
// packed columns and W words per value.
struct FlowLayout {
  size_t xch, post, dec, words;
  __host__ __device__ static FlowLayout make(int B, int qmax, int W) {
    FlowLayout f;
    f.xch = 16;
    f.post = f.xch + (size_t)B * 4 * qmax * W;
    f.dec = f.post + (size_t)kFlowRing * B * 2;
    f.words = f.dec + (size_t)kFlowRing * 3;
    return f;
  }
};

// Interior rows [lo, hi) of band b (rows per band R) of an n x n plate.
__host__ __device__ __forceinline__ void flow_band(int b, int R, int n, int& lo, int& hi) {
  lo = b * R > 1 ? b * R : 1;
  hi = b * R + R < n + 1 ? b * R + R : n + 1;
}

__device__ __forceinline__ unsigned flow_ld32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// First tested iteration after it0 is number 0: iteration (it0 / K + 1 + j) K,
// or the last iteration if that is smaller.
__device__ __forceinline__ long long flow_tested_iter(long long j, int it0, int K, int max_iters) {
  const long long k = ((long long)it0 / K + 1 + j) * K;
  return k < max_iters ? k : (long long)max_iters;
}

// The arbiter block: for each tested iteration in order, waits for every
// band's post, takes the grid-wide largest |change| and posts the decision
// of Algorithm 1's stop test (stop at a tested iteration whose max|change|
// is below the tolerance, or at the iteration cap).
__device__ void flow_arbiter(const SlotDesc& sd, int it0, int B, int R, unsigned long long* sync,
                             const FlowLayout& L) {
  __shared__ unsigned long long red[kFlowThreads / 32];
  __shared__ int go;
  unsigned* const abort_w = (unsigned*)sync;
  const int n = sd.n, K = sd.K, max_iters = sd.max_iters;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long kprev = it0;
  for (long long j = 0;; ++j) {
    const long long kj = flow_tested_iter(j, it0, K, max_iters);
    const long long limit = kGridFlowSpins + (kj - kprev) * 4096;  // the posts come K iterations after the last ones
    kprev = kj;
    const unsigned tag = (unsigned)(j + 1);
    unsigned long long m = 0;
    int ok = 1;
    for (int b = threadIdx.x; b < B && ok; b += blockDim.x) {
      int lo, hi;
      flow_band(b, R, n, lo, hi);
      if (lo >= hi) continue;  // a band of ring rows only posts nothing
      const unsigned long long* p = sync + L.post + ((size_t)(j % kFlowRing) * B + b) * 2;
      long long spins = 0;
      unsigned long long w0 = 0, w1 = 0;
      while (true) {
        w0 = flow_ld(p);
        w1 = flow_ld(p + 1);
        if ((unsigned)(w0 >> 32) == tag && (unsigned)(w1 >> 32) == tag) break;
        if (++spins > limit || ((spins & 63) == 0 && flow_ld32(abort_w))) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      if (ok) m = umax64(m, (w0 << 32) | (w1 & 0xffffffffull));
    }
    m = warp_max64(m);
    if (lane == 0) red[warp] = m;
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) atomicExch(abort_w, 1u);
      return;
    }
    if (threadIdx.x == 0) {
      unsigned long long mm = 0;
      for (int w = 0; w < kFlowThreads / 32; ++w) mm = umax64(mm, red[w]);
      const bool conv = (kj % K) == 0 && sd.stop == kStopDelta && bits_to_double(mm) < sd.tol;
      const bool stop = conv || kj >= max_iters;
      unsigned long long* d = sync + L.dec + (size_t)(j % kFlowRing) * 3;
      flow_st(d, flow_word(tag, (stop ? 1u : 0u) | (conv ? 2u : 0u)));
      flow_st(d + 1, flow_word(tag, (unsigned)(mm >> 32)));
      flow_st(d + 2, flow_word(tag, (unsigned)mm));
      go = !stop;
    }
    __syncthreads();
    if (!go) return;
  }
}

// Bands of R rows (the last block of the grid is the arbiter).  Shared
// memory: both colours of the band with a ghost row above and below
// ((R + 2) rows each, local row lr = grid row rlo - 1 + lr), then
// kFlowDepth copies of the band's interior rows of both colours.
template <typename T>
__global__ void __launch_bounds__(kFlowThreads) k_grid_flow(const SlotDesc* __restrict__ slots, SlotState* states,
                                                            int slot, int R, unsigned long long* sync) {
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ unsigned long long wmax[kFlowThreads / 32];
  __shared__ int ctl[3];  // decision read by thread 0: stop slot (-1: none yet), failed, converged
  __shared__ unsigned long long ctl_m;
  const SlotDesc& sd = slots[slot];
  SlotState* st = states + slot;
  const int B = (int)gridDim.x - 1;
  const int n = sd.n, pitch = sd.pitch, m = n + 2, qmax = (n + 1) >> 1;
  constexpr int W = FlowVal<T>::W;
  const FlowLayout L = FlowLayout::make(B, qmax, W);
  unsigned* const abort_w = (unsigned*)sync;
  const int it0 = st->iters;
  if (it0 >= sd.max_iters) return;  // nothing to do (never launched so)
  if ((int)blockIdx.x == B) {
    flow_arbiter(sd, it0, B, R, sync, L);
    return;
  }
  const int b = blockIdx.x;
  const int rlo = min(m, b * R), rhi = min(m, rlo + R), nr = rhi - rlo;
  int r_first, r_last;  // interior rows of the band
  flow_band(b, R, n, r_first, r_last);
  if (r_first >= r_last) return;  // ring rows only: no work, and no band waits for it
  const int nri = r_last - r_first;
  const bool up = r_first - 1 >= 1;  // the band above owns interior row r_first - 1
  const bool down = r_last <= n;     // the band below owns interior row r_last
  T* const S0 = (T*)fsm;
  T* const S1 = S0 + (size_t)(R + 2) * pitch;
  T* const snap = S1 + (size_t)(R + 2) * pitch;  // [kFlowDepth][2][R][pitch]
  const int xbuf = st->xbuf;
  T* const X0 = (T*)sd.x[xbuf][0];
  T* const X1 = (T*)sd.x[xbuf][1];
  unsigned long long* const xch = sync + L.xch;
  auto xslot = [&](int bb, int c, int ed) -> unsigned long long* {
    return xch + (((size_t)bb * 2 + c) * 2 + ed) * (size_t)qmax * W;
  };
  const bool ok_geom = dbg_range((long long)(rlo - 1 < 0 ? 0 : rlo - 1) * pitch,
                                 (long long)(rhi + 1 > m ? m : rhi + 1) * pitch, (long long)m * pitch, st);
  for (int idx = threadIdx.x; ok_geom && idx < 2 * (nr + 2) * pitch; idx += blockDim.x) {
    const int c = idx / ((nr + 2) * pitch);
    const int e = idx - c * (nr + 2) * pitch;
    const int r = rlo - 1 + e / pitch;
    if (r >= 0 && r < m) (c ? S1 : S0)[e] = (c ? X1 : X0)[(long long)(rlo - 1) * pitch + e];
  }
  __syncthreads();

  const T a = sizeof(T) == 4 ? (T)sd.a32 : (T)sd.a64;
  const T bw = sizeof(T) == 4 ? (T)sd.b32 : (T)sd.b64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int k = it0;
  unsigned ph = 0;     // phases computed (the tag of their edge words)
  int jn = 0, jd = 0;  // tested iterations posted / decisions read
  int stop_j = -1, failed = ok_geom ? 0 : 1;
  // thread 0: the words of decision jd as loaded at the previous iteration
  unsigned long long pf0 = 0, pf1 = 0, pf2 = 0;

  while (!failed) {
    // ---- decisions read so far: consume those that have arrived, in order;
    // wait only when kFlowDepth are pending or the iteration cap is reached
    if (threadIdx.x == 0) {
      int stopped = -1, fail = 0, conv = 0;
      unsigned long long mstop = 0;
      while (jd < jn) {
        const bool must = (jn - jd >= kFlowDepth) || k >= sd.max_iters;
        const unsigned tag = (unsigned)(jd + 1);
        const unsigned long long* d = sync + L.dec + (size_t)(jd % kFlowRing) * 3;
        long long spins = 0;
        // pf*: the words of slot jd as loaded one iteration ago (or cleared)
        while (!((unsigned)(pf0 >> 32) == tag && (unsigned)(pf1 >> 32) == tag && (unsigned)(pf2 >> 32) == tag)) {
          if (!must) break;
          if (++spins > kGridFlowSpins || ((spins & 63) == 0 && flow_ld32(abort_w))) {
            fail = 1;
            atomicExch(abort_w, 1u);
            break;
          }
          if (spins > 1) __nanosleep(64);
          pf0 = flow_ld(d);
          pf1 = flow_ld(d + 1);
          pf2 = flow_ld(d + 2);
        }
        if (fail || !((unsigned)(pf0 >> 32) == tag && (unsigned)(pf1 >> 32) == tag && (unsigned)(pf2 >> 32) == tag))
          break;
        if ((unsigned)pf0 & 1u) {
          stopped = jd;
          conv = ((unsigned)pf0 >> 1) & 1u;
          mstop = (pf1 << 32) | (pf2 & 0xffffffffull);
          break;
        }
        ++jd;
        pf0 = pf1 = pf2 = 0;  // not loaded for the next slot yet
      }
      if (stopped < 0 && !fail && jd < jn) {  // load the oldest pending decision for the next iteration
        const unsigned long long* d = sync + L.dec + (size_t)(jd % kFlowRing) * 3;
        pf0 = flow_ld(d);
        pf1 = flow_ld(d + 1);
        pf2 = flow_ld(d + 2);
      }
      ctl[0] = stopped;
      ctl[1] = fail;
      ctl[2] = conv;
      ctl_m = mstop;
    }
    __syncthreads();
    stop_j = ctl[0];
    failed = ctl[1];
    if (stop_j >= 0 || failed) break;

    // ---- iteration k + 1: red phase, black phase
    ++k;
    const bool tested = (k % sd.K) == 0 || k >= sd.max_iters;
    unsigned long long dm = 0;
    unsigned dm32 = 0;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      ++ph;
      T* Sc = c ? S1 : S0;
      T* So = c ? S0 : S1;
      const T* Gc = (const T*)sd.g[c];
      if (ph > 1) {  // the neighbours' rows of the other colour from phase ph - 1 into the ghost rows
        const int oc = 1 - c;
        int ok = 1;
        for (int e = threadIdx.x; e < 2 * qmax && ok; e += blockDim.x) {
          const int ed = e >= qmax;  // 0: ghost row above (the upper band's last row), 1: below
          if (ed ? !down : !up) continue;
          const int q = 1 + e - ed * qmax;
          const int row = ed ? r_last : r_first - 1;
          if (q > ((n + ((row + oc) & 1)) >> 1)) continue;
          const unsigned long long* p = xslot(ed ? b + 1 : b - 1, oc, ed ? 0 : 1) + (size_t)(q - 1) * W;
          T v;
          long long spins = 0;
          while (!FlowVal<T>::get(p, ph - 1, v)) {
            if (++spins > kGridFlowSpins || ((spins & 63) == 0 && flow_ld32(abort_w))) {
              ok = 0;
              atomicExch(abort_w, 1u);
              break;
            }
            __nanosleep(32);
          }
          if (ok) So[(size_t)(row - rlo + 1) * pitch + q + kOff] = v;
        }
        if (__syncthreads_or(!ok)) {
          failed = 1;
          break;
        }
      }
      for (int e = threadIdx.x; e < nri * qmax; e += blockDim.x) {
        const int row = r_first + e / qmax;
        const int q = 1 + e % qmax;
        const int s = (row + c) & 1;
        if (q > ((n + s) >> 1)) continue;
        const size_t le = (size_t)(row - rlo + 1) * pitch + kOff + q;
        const T own = Sc[le];
        T sum = radd(radd(So[le - pitch], So[le + pitch]), radd(So[le - s], So[le - s + 1]));
        if (Gc) sum = radd(sum, Gc[(size_t)row * pitch + q + kOff]);
        const T nu = radd(rmul(a, own), rmul(bw, sum));
        Sc[le] = nu;
        if (tested) {
          if (sizeof(T) == 4)
            dm32 = max(dm32, abs_bits32((float)radd(nu, -own)));
          else
            dm = umax64(dm, abs_bits((double)radd(nu, -own)));
        }
      }
      __syncthreads();
      // this phase's values of the band's first and last interior rows, for the bands above and below
      for (int e = threadIdx.x; e < 2 * qmax; e += blockDim.x) {
        const int ed = e >= qmax;  // 0: first row (read by the band above), 1: last row (by the band below)
        if (ed ? !down : !up) continue;
        const int q = 1 + e - ed * qmax;
        const int row = ed ? r_last - 1 : r_first;
        if (q > ((n + ((row + c) & 1)) >> 1)) continue;
        FlowVal<T>::put(xslot(b, c, ed) + (size_t)(q - 1) * W, ph, Sc[(size_t)(row - rlo + 1) * pitch + q + kOff]);
      }
    }
    if (failed) break;
    if (tested) {  // copy of the band after iteration k, and its largest |change|
      T* sn = snap + (size_t)(jn % kFlowDepth) * 2 * R * pitch;
      for (int idx = threadIdx.x; idx < 2 * nri * pitch; idx += blockDim.x) {
        const int c = idx / (nri * pitch);
        const int e = idx - c * nri * pitch;
        sn[(size_t)c * R * pitch + e] = (c ? S1 : S0)[(size_t)(r_first - rlo + 1) * pitch + e];
      }
      if (sizeof(T) == 4) dm = abs_bits_of(__uint_as_float(dm32));
      dm = warp_max64(dm);
      if (lane == 0) wmax[warp] = dm;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long mm = 0;
        for (int w = 0; w < kFlowThreads / 32; ++w) mm = umax64(mm, wmax[w]);
        unsigned long long* pp = sync + L.post + ((size_t)(jn % kFlowRing) * B + b) * 2;
        flow_st(pp, flow_word((unsigned)(jn + 1), (unsigned)(mm >> 32)));
        flow_st(pp + 1, flow_word((unsigned)(jn + 1), (unsigned)mm));
      }
      ++jn;
    }
  }
  // the solution: the band's copy of the stop iteration
  if (!failed && stop_j >= 0) {
    const T* sn = snap + (size_t)(stop_j % kFlowDepth) * 2 * R * pitch;
    for (int idx = threadIdx.x; idx < 2 * nri * pitch; idx += blockDim.x) {
      const int c = idx / (nri * pitch);
      const int e = idx - c * nri * pitch;
      (c ? X1 : X0)[(size_t)r_first * pitch + e] = sn[(size_t)c * R * pitch + e];
    }
  }
  // end every wait on this band's edge words
  for (int e = threadIdx.x; e < 4 * qmax * W; e += blockDim.x) flow_st(xslot(b, 0, 0) + e, flow_word(kTagDone, 0u));
  if (threadIdx.x == 0) {
    if (failed) {
      atomicExch(abort_w, 1u);
      atomicExch(&st->error, ok_geom ? 1 : kErrBounds);
      st->done = 1;
    } else if (r_first == 1) {
      st->iters = (int)flow_tested_iter(stop_j, it0, sd.K, sd.max_iters);
      st->converged = ctl[2];
      st->last_dmax = bits_to_double(ctl_m);
      st->done = 1;
    }
  }
}

// Rows per band and bands of k_grid_flow for an n x n plate: bands of at
// least two rows, at most one block per SM with the arbiter's; 0 if the
// plate does not fit (then *smem_out is meaningless).
template <typename T>
static int flow_geometry(int n, int pitch, int sm_count, int* R_out, size_t* smem_out) {
  static int per_sm = -1;
  constexpr int kSmemCap = 200 * 1024;
  if (per_sm < 0) {
    if (cudaFuncSetAttribute(k_grid_flow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_flow<T>, kFlowThreads, kSmemCap) !=
            cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
  }
  if (per_sm <= 0 || sm_count < 2) return 0;
  const int m = n + 2;
  const int R = std::max(2, (m + sm_count - 2) / (sm_count - 1));
  const int B = (m + R - 1) / R;
  const size_t smem = (2ull * (R + 2) + 2ull * kFlowDepth * R) * pitch * sizeof(T);
  if (smem > (size_t)kSmemCap || B + 1 > sm_count * per_sm) return 0;
  *R_out = R;
  *smem_out = smem;
  return B;
}

bool grid_flow_fits(bool fp32, int n, int pitch, int sm_count) {
  int R = 0;
  size_t smem = 0;
  return (fp32 ? flow_geometry<float>(n, pitch, sm_count, &R, &smem)
               : flow_geometry<double>(n, pitch, sm_count, &R, &smem)) > 0;
}

size_t grid_flow_sync_bytes(bool fp32, int n, int pitch, int sm_count) {
  int R = 0;
  size_t smem = 0;
  const int B = fp32 ? flow_geometry<float>(n, pitch, sm_count, &R, &smem)
                     : flow_geometry<double>(n, pitch, sm_count, &R, &smem);
  if (B <= 0) return 0;
  return FlowLayout::make(B, (n + 1) / 2, fp32 ? 1 : 2).words * sizeof(unsigned long long);
}

cudaError_t launch_grid_flow(bool fp32, int n, int pitch, int sm_count, const SlotDesc* slots, SlotState* states,
                             int slot, void* sync, size_t sync_bytes, cudaStream_t s) {
  int R = 0;
  size_t smem = 0;
  const int B = fp32 ? flow_geometry<float>(n, pitch, sm_count, &R, &smem)
                     : flow_geometry<double>(n, pitch, sm_count, &R, &smem);
  if (B <= 0) return cudaErrorInvalidValue;
  const size_t need = FlowLayout::make(B, (n + 1) / 2, fp32 ? 1 : 2).words * sizeof(unsigned long long);
  if (sync_bytes < need) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(sync, 0, need, s);
  if (e != cudaSuccess) return e;
  unsigned long long* sy = (unsigned long long*)sync;
  void* args[] = {(void*)&slots, (void*)&states, (void*)&slot, (void*)&R, (void*)&sy};
  count_kernel_launches(1);
  return fp32 ? cudaLaunchCooperativeKernel((const void*)k_grid_flow<float>, dim3(B + 1), dim3(kFlowThreads), args,
                                            smem, s)
              : cudaLaunchCooperativeKernel((const void*)k_grid_flow<double>, dim3(B + 1), dim3(kFlowThreads), args,
                                            smem, s);
}

}  // namespace sorgb
