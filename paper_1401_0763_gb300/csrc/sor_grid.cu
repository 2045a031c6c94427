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

}  // namespace sorgb
