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
#include <cmath>
#include <cstring>
#include <map>
#include <sstream>
#include <utility>
#include <vector>

#include "sor_devfn.cuh"
#include "sor_runtime.h"

namespace sorgb {
namespace {

__device__ __forceinline__ size_t e3(int k, int i, int q, int m, int pitch) {
  return ((size_t)k * (size_t)m + (size_t)i) * (size_t)pitch + (size_t)(q + kOff);
}

// Solve description in device memory (constant while the solve runs).
struct Desc3 {
  void* x[2];            // colour arrays (FP64 or FP32)
  const void* g[2];      // h^2 f in the sweep type, or null
  const double* g64[2];  // h^2 f in FP64 for the residual, or null
  int n, m, pitch, K, max_iters, stop, tiles;
  float a32, b32;        // (float)(1 - w), (float)(w / 6)
  double a64, b64;       // 1 - w, w / 6
  double tol;
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
  unsigned long long bb = 0;
  if (q < qw) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int j = 2 * q - 1 + t;
      if (j < 0 || j >= m) continue;
      const int c = (i + j + k) & 1;
      const size_t nat = ((size_t)k * m + i) * m + j;
      const size_t e = e3(k, i, q, m, pitch);
      (c ? x1 : x0)[e] = (T)u0[nat];
      const bool interior = i >= 1 && i <= n && j >= 1 && j <= n && k >= 1 && k <= n;
      double gc = 0.0;
      if (interior && f) gc = __dmul_rn(h2, f[((size_t)(k - 1) * n + (i - 1)) * n + (j - 1)]);
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

// Rows [i0, i1) of plane k for one warp, one colour phase, exact order.
template <typename T, bool MEASURE, bool HAS_G>
__device__ __forceinline__ unsigned long long sweep3_rows(T* __restrict__ X, const T* __restrict__ O,
                                                          const T* __restrict__ G, T a, T b, int pitch, int m, int n,
                                                          int colour, int k, int q0, int i0, int i1, int lane) {
  unsigned long long dm = 0;
  unsigned dm32 = 0;
  if (i0 >= i1) return 0;
  T om[4], oc[4], op[4];
  load4(O + e3(k, i0 - 1, q0, m, pitch), om);
  load4(O + e3(k, i0, q0, m, pitch), oc);
  for (int i = i0; i < i1; ++i) {
    T own[4], dn[4], up[4], gv[4];
    load4(O + e3(k, i + 1, q0, m, pitch), op);
    load4(X + e3(k, i, q0, m, pitch), own);
    load4(O + e3(k - 1, i, q0, m, pitch), dn);
    load4(O + e3(k + 1, i, q0, m, pitch), up);
    if (HAS_G) load4(G + e3(k, i, q0, m, pitch), gv);
    T left = __shfl_up_sync(0xffffffffu, oc[3], 1);
    T right = __shfl_down_sync(0xffffffffu, oc[0], 1);
    if (lane == 0) left = O[e3(k, i, q0 - 1, m, pitch)];
    if (lane == 31) right = O[e3(k, i, q0 + kVec, m, pitch)];
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
      T sum = radd(radd(radd(om[v], op[v]), radd(W[v], E[v])), radd(dn[v], up[v]));
      if (HAS_G) sum = radd(sum, gv[v]);
      const T nu = radd(rmul(a, own[v]), rmul(b, sum));
      const bool in = (q0 + v) <= qlim;
      // cells past the interior keep their value (the whole vector is written back)
      nv[v] = in ? nu : own[v];
      if (MEASURE && in) {
        if (sizeof(T) == 4)
          dm32 = max(dm32, abs_bits32((float)radd(nu, -own[v])));
        else
          dm = umax64(dm, abs_bits((double)radd(nu, -own[v])));
      }
    }
    store4(X + e3(k, i, q0, m, pitch), nv);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      om[v] = oc[v];
      oc[v] = op[v];
    }
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

// One colour phase over tiles (plane, rows, 128 packed columns); a tile's
// rows are split among the block's warps.  The last tile to finish the black
// phase closes the iteration.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_sweep3d(const Desc3* __restrict__ dp, SlotState* st,
                                                      const Tile* __restrict__ tiles, int ntiles, int colour) {
  __shared__ unsigned long long red[kWarpsY];
  __shared__ int ctl[3];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const Desc3& d = *dp;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    if (threadIdx.x == 0) {
      const int kk = *((volatile int*)&st->iters) + 1;
      ctl[0] = *((volatile int*)&st->done);
      ctl[1] = kk;
      ctl[2] = ((kk % d.K) == 0) || (kk >= d.max_iters);
    }
    __syncthreads();
    const int skip = ctl[0], kk = ctl[1], measure = ctl[2];
    __syncthreads();
    if (skip) continue;
    T* X = (T*)d.x[colour];
    const T* O = (const T*)d.x[colour ^ 1];
    const T* G = (const T*)d.g[colour];
    const T a = sizeof(T) == 4 ? (T)d.a32 : (T)d.a64;
    const T b = sizeof(T) == 4 ? (T)d.b32 : (T)d.b64;
    const int k = tl.row0 / d.m, ib = tl.row0 - k * d.m;
    const int q0 = tl.col0 + lane * kVec;
    const int rpw = (tl.nrows + kWarpsY - 1) / kWarpsY;
    const int i0 = ib + wy * rpw;
    const int i1 = min(i0 + rpw, ib + tl.nrows);
    unsigned long long dm = 0;
    // the source term is a compile-time choice: as a runtime test the compiler
    // issues its addition speculatively, one more FP64 operation per cell
    if (measure)
      dm = G ? sweep3_rows<T, true, true>(X, O, G, a, b, d.pitch, d.m, d.n, colour, k, q0, i0, i1, lane)
             : sweep3_rows<T, true, false>(X, O, G, a, b, d.pitch, d.m, d.n, colour, k, q0, i0, i1, lane);
    else if (G)
      (void)sweep3_rows<T, false, true>(X, O, G, a, b, d.pitch, d.m, d.n, colour, k, q0, i0, i1, lane);
    else
      (void)sweep3_rows<T, false, false>(X, O, G, a, b, d.pitch, d.m, d.n, colour, k, q0, i0, i1, lane);
    if (measure) block_max_to(dm, &st->dmax_bits, red);
    if (colour == 1) {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&st->arrive, 1u);
        if (prev == (unsigned)d.tiles - 1u) {
          __threadfence();
          finalize3(d, st, kk, measure);
        }
      }
      __syncthreads();
    }
  }
}

// Scaled residual over tiles, both colours, in FP64.  CHECK: the residual
// stop of Algorithm 1's test on iterations that are multiples of K (decided
// by the last tile); otherwise only rho of the current iterate is recorded.
template <typename T, bool CHECK>
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
      if (CHECK)
        skip = *((volatile int*)&st->converged) || it == 0 || (it % d.K) != 0 ||
               it == *((volatile int*)&st->checked_iter);
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
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const double nb =
              __dadd_rn(__dadd_rn(__dadd_rn((double)nm[v], (double)np[v]), __dadd_rn((double)W[v], (double)E[v])),
                        __dadd_rn((double)dn[v], (double)up[v]));
          const double r = __dadd_rn(__dadd_rn(gv[v], nb), -__dmul_rn(6.0, (double)own[v]));
          if ((q0 + v) <= qlim) rm = umax64(rm, abs_bits(r));
        }
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
        if (CHECK) {
          st->checked_iter = it;
          if (rho < d.tol) {
            st->done = 1;
            st->converged = 1;
          }
        }
      }
    }
    __syncthreads();
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

template <typename T>
sor_status run3d(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out, sor_result* res) {
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

  // tiles: plane k, rows of 32, columns of 128 packed cells
  std::vector<Tile> tiles;
  for (int k = 1; k <= n; ++k)
    for (int r = 0; r < L.row_tiles(); ++r)
      for (int t = 0; t < L.col_tiles(); ++t)
        tiles.push_back(Tile{0, k * m + 1 + r * kTileRows, 1 + t * kWarpCols, std::min(kTileRows, n - r * kTileRows)});
  const int nt = (int)tiles.size();

  size_t bytes = 2 * elems * sizeof(T) + sizeof(Desc3) + sizeof(SlotState) + sizeof(Tile) * nt + 1024;
  if (has_f) bytes += 2 * elems * sizeof(T) + (sizeof(T) == 4 ? 2 * elems * sizeof(double) : 0);
  const bool stage_u = !in_dev || !out_dev;
  if (stage_u) bytes += ncube * sizeof(double);
  if (has_f && !f_dev) bytes += nf * sizeof(double);
  Buffers3 B;
  B.c = c;
  sor_status rs = ctx_reserve(c, bytes, false, 0.0);
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
  double* d_u = stage_u ? (double*)B.get(ncube * sizeof(double)) : nullptr;
  double* d_f = (has_f && !f_dev) ? (double*)B.get(nf * sizeof(double)) : nullptr;
  if (!x[0] || !x[1] || (has_f && (!g[0] || !g[1] || !g64[0] || !g64[1])) || !d_desc || !d_state || !d_tiles ||
      (stage_u && !d_u) || (has_f && !f_dev && !d_f)) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  cudaStream_t s = c->stream;

  Desc3 d;
  std::memset(&d, 0, sizeof(d));
  d.x[0] = x[0];
  d.x[1] = x[1];
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

  // one chunk of L iterations starting after iteration `first`: two phases per
  // iteration and, for the residual stop, the test after multiples of K
  auto enqueue = [&](int first, int Lc) -> sor_status {
    for (int it = 1; it <= Lc; ++it) {
      k_sweep3d<T><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt, 0);
      k_sweep3d<T><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt, 1);
      if (stop == kStopResid && (first + it) % d.K == 0)
        k_resid3d<T, true><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
    }
    SOR3_CK(c, cudaGetLastError());
    return SOR_OK;
  };
  const int chunk = c->opt_chunk.load() > 0 ? c->opt_chunk.load() : 64;
  const bool use_graphs = c->opt_graphs.load() != 0;
  SOR3_CK(c, cudaEventRecord(ev0, s));
  long long planned = 0;
  bool finished = st.done != 0;
  while (!finished && planned < p->max_iters) {
    const int Lc = (int)std::min<long long>(chunk, p->max_iters - planned);
    if (use_graphs) {
      const std::pair<int, int> key(Lc, stop == kStopResid ? (int)(planned % d.K) : 0);
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
  k_resid3d<T, false><<<grid, kThreads, 0, s>>>(d_desc, d_state, d_tiles, nt);
  SOR3_CK(c, cudaGetLastError());
  double* out_dst = out_dev ? u_out : d_u;
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

}  // namespace

sor_status solve3d_blocking(Ctx* c, const sor_params* p, const double* u0, const double* f, double* u_out,
                            sor_result* res) {
  if (!p || !u0 || !u_out) {
    c->set_error("params, u0 and u_out must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  std::ostringstream why;
  if (p->n < 1 || p->n > kMax3dN) why << "n must be in [1, " << kMax3dN << "]";
  else if (p->precision != SOR_FP64 && p->precision != SOR_FP32) why << "3D solves run in FP64 or FP32";
  else if (p->stop != SOR_STOP_MAXDELTA && p->stop != SOR_STOP_RESID_REL) why << "unknown stop rule";
  else if (p->max_iters < 0 || p->check_every < 1) why << "max_iters >= 0 and check_every >= 1 required";
  else if (p->flags & ~SOR_FLAG_EXACT_ORDER) why << "unknown flags";
  else if (p->stall_window != 0) why << "stall_window is not supported on 3D grids";
  else if (std::isnan(p->tol) || std::isnan(p->omega)) why << "tol and omega must not be NaN";
  else if (p->omega > 0.0 && !(p->omega < 2.0)) why << "omega must be in (0, 2)";
  if (!why.str().empty()) {
    c->set_error(why.str());
    return SOR_ERR_INVALID_ARG;
  }
  return p->precision == SOR_FP64 ? run3d<double>(c, p, u0, f, u_out, res) : run3d<float>(c, p, u0, f, u_out, res);
}

}  // namespace sorgb
