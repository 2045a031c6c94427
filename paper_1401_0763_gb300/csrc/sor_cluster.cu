// Whole solves of small grids inside one thread-block cluster.
//
// A grid of up to a few hundred cells per side fits in the distributed shared
// memory of a cluster of 8 or 16 CTAs (one band of rows of both colour
// arrays per CTA).  The kernel then runs Algorithm 1 to the end by itself:
// each iteration is the red phase over every CTA's rows, a cluster barrier,
// the black phase, a cluster barrier (the phase barrier of Section 3.2 as a
// hardware barrier).  Every CTA also keeps ghost copies of the row just above
// and just below its band; after a phase it pushes the two edge rows it
// updated into its neighbours' ghost rows (distributed shared memory stores),
// so the update loop itself reads only local shared memory.  On tested
// iterations every CTA publishes its max |change| (or its largest scaled
// residual), all of them read the cluster-wide maximum after the barrier and
// take the same stop decision.  One launch replaces 2 launches per iteration,
// which dominate the time of a small grid.  The update is the exact-order
// form of k_sweep (every product and sum rounded on its own), so results match
// the unfused exact path and the CPU oracle bit for bit.
#include <cooperative_groups.h>

#include "sor_devfn.cuh"
#include "sor_kernels.h"

namespace cg = cooperative_groups;

namespace sorgb {

constexpr int kClusterThreads = 512;
constexpr int kClusterWarps = kClusterThreads / 32;

// Shared-memory rows per colour of one CTA: its band of R rows plus a ghost
// row on each side.
__host__ __device__ __forceinline__ int cluster_band_rows(int m, int C) { return (m + C - 1) / C; }

template <typename T>
__global__ void __launch_bounds__(kClusterThreads) k_cluster_solve(const SlotDesc* __restrict__ slots,
                                                                   SlotState* states, int slot) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char csm[];
  __shared__ unsigned long long wmax[kClusterWarps];
  __shared__ unsigned long long pub[2];  // this CTA's max |change| and max |r~| of the current test
  const SlotDesc& sd = slots[slot];
  SlotState* st = states + slot;
  const int n = sd.n, pitch = sd.pitch, m = n + 2;
  const int R = cluster_band_rows(m, C);
  const int rlo = min(m, rank * R), rhi = min(m, rlo + R);
  const int nr = rhi - rlo;  // rows of the band (0 for CTAs past the grid)
  // local row lr holds grid row rlo - 1 + lr: lr = 0 and lr = nr + 1 are the ghosts
  T* const S0 = (T*)csm;
  T* const S1 = (T*)csm + (size_t)(R + 2) * pitch;
  const int xbuf = st->xbuf;

  // stage the band and both ghost rows of both colours
  for (int idx = threadIdx.x; idx < 2 * (nr + 2) * pitch; idx += blockDim.x) {
    const int c = idx / ((nr + 2) * pitch);
    const int e = idx - c * (nr + 2) * pitch;
    const int lr = e / pitch;
    const int r = rlo - 1 + lr;
    if (r >= 0 && r < m) (c ? S1 : S0)[e] = ((const T*)sd.x[xbuf][c])[(size_t)(rlo - 1) * pitch + e];
  }
  cluster.sync();

  const T a = sizeof(T) == 4 ? (T)sd.a32 : (T)sd.a64;
  const T b = sizeof(T) == 4 ? (T)sd.b32 : (T)sd.b64;
  const int r_first = max(rlo, 1), r_last = min(rhi, n + 1);  // interior rows of the band: [r_first, r_last)
  const double bmax = bits_to_double(st->bmax_bits);
  int k = st->iters, converged = 0, run = st->stall_run;
  double best_rho = st->best_rho, last_dmax = st->last_dmax, last_rho = st->last_rho;
  int checked = st->checked_iter;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  auto cluster_max = [&](unsigned long long v, int which) -> unsigned long long {
    v = warp_max64(v);
    if (lane == 0) wmax[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long mm = 0;
      for (int w = 0; w < kClusterWarps; ++w) mm = umax64(mm, wmax[w]);
      pub[which] = mm;
    }
    cluster.sync();
    unsigned long long all = 0;
    for (int r = 0; r < C; ++r) all = umax64(all, *cluster.map_shared_rank(&pub[which], r));
    return all;
  };

  // after phase c: copy the band's first / last row of colour c into the
  // ghost rows of the CTAs above / below (interior rows only: the ring never
  // changes and was staged into the ghosts at the start)
  auto push_edges = [&](T* Sc) {
    __syncthreads();
    if (nr > 0) {
      if (rank > 0 && rlo >= 1 && rlo <= n) {
        // the band above ends at row rlo - 1: its ghost row below is local row R + 1
        T* dst = cluster.map_shared_rank(Sc, rank - 1) + (size_t)(R + 1) * pitch;
        const T* src = Sc + (size_t)1 * pitch;
        for (int e = threadIdx.x; e < pitch; e += blockDim.x) dst[e] = src[e];
      }
      if (rank + 1 < C && rhi < m && rhi - 1 >= 1 && rhi - 1 <= n) {
        T* dst = cluster.map_shared_rank(Sc, rank + 1);  // its ghost row above is local row 0
        const T* src = Sc + (size_t)nr * pitch;
        for (int e = threadIdx.x; e < pitch; e += blockDim.x) dst[e] = src[e];
      }
    }
  };

  while (k < sd.max_iters) {
    ++k;
    const bool measure = (k % sd.K) == 0 || k >= sd.max_iters;
    unsigned long long dm = 0;
    unsigned dm32 = 0;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      T* Sc = c ? S1 : S0;
      const T* So = c ? S0 : S1;
      const T* Gc = (const T*)sd.g[c];
      for (int row = r_first + warp; row < r_last; row += kClusterWarps) {
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
      push_edges(Sc);
      cluster.sync();
    }
    if (measure) {
      if (sizeof(T) == 4) dm = abs_bits_of(__uint_as_float(dm32));
      last_dmax = bits_to_double(cluster_max(dm, 0));
      if (sd.stop == kStopDelta && (k % sd.K) == 0 && last_dmax < sd.tol) {
        converged = 1;
        break;
      }
    }
    if (sd.stop == kStopResid && (k % sd.K) == 0) {
      // scaled residual r~ = (g + ((N+S)+(W+E))) - 4u in FP64 over this CTA's cells of both colours
      unsigned long long rm = 0;
      for (int c = 0; c < 2; ++c) {
        const double* G64 = sd.g64[c];
        const T* Sc = c ? S1 : S0;
        const T* So = c ? S0 : S1;
        for (int row = r_first + warp; row < r_last; row += kClusterWarps) {
          const int s = (row + c) & 1;
          const int qlim = (n + s) >> 1;
          const size_t lb = (size_t)(row - rlo + 1) * pitch + kOff;
          for (int q = 1 + lane; q <= qlim; q += 32) {
            const size_t le = lb + q;
            const double nb = __dadd_rn(__dadd_rn((double)So[le - pitch], (double)So[le + pitch]),
                                        __dadd_rn((double)So[le - s], (double)So[le - s + 1]));
            const double g = G64 ? G64[(size_t)row * pitch + q + kOff] : 0.0;
            const double r = __dadd_rn(__dadd_rn(g, nb), -__dmul_rn(4.0, (double)Sc[le]));
            rm = umax64(rm, abs_bits(r));
          }
        }
      }
      const double rmax = bits_to_double(cluster_max(rm, 1));
      const double rho = bmax > 0.0 ? __ddiv_rn(rmax, bmax) : rmax;
      last_rho = rho;
      checked = k;
      if (rho < sd.tol) {
        converged = 1;
        break;
      }
      if (rho < best_rho) {
        best_rho = rho;
        run = 0;
      } else if (rho < 4.0 * best_rho) {
        run += 1;
        if (sd.stall > 0 && run >= sd.stall) break;
      } else {
        run = 0;
      }
    }
  }
  // write the band back and record the outcome (every CTA took the same decisions)
  for (int idx = threadIdx.x; idx < 2 * nr * pitch; idx += blockDim.x) {
    const int c = idx / (nr * pitch);
    const int e = idx - c * nr * pitch;
    ((T*)sd.x[xbuf][c])[(size_t)rlo * pitch + e] = (c ? S1 : S0)[(size_t)pitch + e];
  }
  if (rank == 0 && threadIdx.x == 0) {
    st->iters = k;
    st->converged = converged;
    st->done = 1;
    st->last_dmax = last_dmax;
    st->last_rho = last_rho;
    st->checked_iter = checked;
    st->stall_run = run;
    st->best_rho = best_rho;
  }
  cluster.sync();  // no CTA leaves while others may still read its shared memory
}

template <typename T>
static cudaError_t cluster_config(int n, int pitch, int* csize, size_t* smem) {
  static int cached = -1;  // cluster size the device accepts for this kernel
  if (cached < 0) {
    cudaError_t e = cudaFuncSetAttribute(k_cluster_solve<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cluster_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = 200 * 1024;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 16;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int cs = 0;
    e = cudaOccupancyMaxPotentialClusterSize(&cs, k_cluster_solve<T>, &cfg);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cs = 8;
    }
    cached = cs >= 16 ? 16 : 8;
  }
  *csize = cached;
  const int R = cluster_band_rows(n + 2, cached);
  *smem = 2ull * (R + 2) * pitch * sizeof(T);
  return cudaSuccess;
}

bool cluster_solve_fits(bool fp32, int n, int pitch) {
  int cs = 0;
  size_t smem = 0;
  const cudaError_t e = fp32 ? cluster_config<float>(n, pitch, &cs, &smem) : cluster_config<double>(n, pitch, &cs, &smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return smem <= 200 * 1024;
}

cudaError_t launch_cluster_solve(bool fp32, int n, int pitch, const SlotDesc* slots, SlotState* states, int slot,
                                 cudaStream_t s) {
  int cs = 0;
  size_t smem = 0;
  cudaError_t e = fp32 ? cluster_config<float>(n, pitch, &cs, &smem) : cluster_config<double>(n, pitch, &cs, &smem);
  if (e != cudaSuccess) return e;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = cs;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  count_kernel_launches(1);
  return fp32 ? cudaLaunchKernelEx(&cfg, k_cluster_solve<float>, slots, states, slot)
              : cudaLaunchKernelEx(&cfg, k_cluster_solve<double>, slots, states, slot);
}

}  // namespace sorgb
