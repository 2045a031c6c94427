// Device helpers shared by the kernel translation units: operations rounded
// one at a time (no contraction), vector loads / stores of 4 consecutive
// packed cells, and order-preserving bit patterns for max reductions.
#pragma once
#include <cuda_runtime.h>

#include "sor_device.cuh"

namespace sorgb {

__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  double2 a = reinterpret_cast<const double2*>(p)[0];
  double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// |x| as the bit pattern of a non-negative double: unsigned order == numeric
// order, and any NaN compares above +inf, so a NaN is never lost by max.
// The sign is cleared by an integer AND on the high word in inline PTX:
// written as a mask of the 64-bit pattern, the compiler turned it into an
// FP64 absolute value, one more instruction on the FP64 pipe per call.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
  asm("and.b32 %0, %0, 0x7fffffff;" : "+r"(hi));
  return ((unsigned long long)hi << 32) | lo;
}
// The same for a float: FP32 kernels keep their max|change| as float bits
// (integer max, no FP64 instruction) and widen once per thread.
__device__ __forceinline__ unsigned abs_bits32(float x) { return __float_as_uint(x) & 0x7fffffffu; }
__device__ __forceinline__ unsigned long long abs_bits_of(float x) { return abs_bits((double)x); }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }

// Block-wide max of v into *dst (atomic).  All threads of the block call it.
__device__ __forceinline__ void block_max_to(unsigned long long v, unsigned long long* dst,
                                             unsigned long long* smem /* [kWarpsY] */) {
  v = warp_max64(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) smem[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = smem[0];
#pragma unroll
    for (int k = 1; k < kWarpsY; ++k) m = umax64(m, smem[k]);
    if (m) atomicMax(dst, m);
  }
  __syncthreads();
}

// Plain-mode bookkeeping after the black phase of iteration k (Algorithm 1):
// count the iteration, test the change on check iterations, stop at the cap.
__device__ __forceinline__ void finalize_plain(const SlotDesc& sd, SlotState* st, int k, int measure) {
  st->arrive = 0;
  st->iters = k;
  if (measure) {
    const double mk = bits_to_double(atomicExch(&st->dmax_bits, 0ull));
    st->last_dmax = mk;
    if (sd.stop == kStopDelta && (k % sd.K) == 0 && mk < sd.tol) {
      st->done = 1;
      st->converged = 1;
    }
  }
  if (k >= sd.max_iters) st->done = 1;
}

// Device-side index checks of the debug build (SOR_DEBUG_BOUNDS): the range
// [lo, hi) must lie inside [0, limit); when it does not, the slot's error
// word records kErrBounds (the solve then returns SOR_ERR_INTERNAL) and the
// caller skips the access.  Release builds compile every check to `true`.
__device__ __forceinline__ bool dbg_range(long long lo, long long hi, long long limit, SlotState* st) {
#ifdef SOR_DEBUG_BOUNDS
  if (lo >= 0 && lo <= hi && hi <= limit) return true;
  if (st) atomicExch(&st->error, kErrBounds);
  return false;
#else
  (void)lo;
  (void)hi;
  (void)limit;
  (void)st;
  return true;
#endif
}

// Debug check of a tile that touches rows [r0, r1) and packed columns
// [q0, q1) of the colour arrays of slot sd (element offset q + kOff in a row).
__device__ __forceinline__ bool dbg_tile(const SlotDesc& sd, SlotState* st, int r0, int r1, int q0, int q1) {
  return dbg_range(r0, r1, (long long)sd.n + 2, st) &&
         dbg_range((long long)q0 + kOff, (long long)q1 + kOff, (long long)sd.pitch, st);
}

__device__ __forceinline__ size_t eidx(int i, int q, int pitch) { return (size_t)i * pitch + q + kOff; }

// Data-flow scheduling of a chunk of colour phases (the cube and 9-point
// kernels): per-strip progress counters published with release stores after
// fenced writes and read with acquire loads.
constexpr int kFlowSpins = 1 << 21;  // polls of about 0.1 us each: far above any phase

__device__ __forceinline__ unsigned flow_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void flow_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Lanes 0..NB-1 poll one counter each (-1 = none) until it reaches `target`;
// false on timeout (bounded: `limit` polls).  Afterwards every lane takes
// its own acquire of all of them, so its later loads see their writes.
template <int NB>
__device__ __forceinline__ bool flow_wait(const unsigned* progress, const int (&nb)[NB], unsigned target, int lane,
                                          int limit = kFlowSpins) {
  bool ok = true;
  int mine = -1;
#pragma unroll
  for (int k = 0; k < NB; ++k)
    if (lane == k) mine = nb[k];
  if (mine >= 0) {
    int spins = 0;
    while (flow_ld_acquire(progress + mine) < target) {
      if (++spins > limit) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
  }
  ok = __all_sync(0xffffffffu, ok);
  if (ok) {
#pragma unroll
    for (int k = 0; k < NB; ++k)
      if (nb[k] >= 0) (void)flow_ld_acquire(progress + nb[k]);
  }
  return ok;
}

}  // namespace sorgb
