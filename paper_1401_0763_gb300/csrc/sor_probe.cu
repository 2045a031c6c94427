// FP64 pipe-rate probe: the measured peak that the FP64 colour phases are
// reported against.
//
// On GB300 the FP64 default phases are bound by the rate at which the SMs
// execute FP64 instructions, not by HBM; the nominal rate (2 FP64 lanes per
// clock per SM) is what the hardware promises, this probe is what it does.
// Every thread of a full-occupancy grid runs kChains independent chains of
// FP64 fused multiply-adds (kind 0) or additions (kind 1), so each SM
// sub-partition always has independent FP64 work to issue; the rate is the
// lane operations of the whole grid divided by the CUDA-event time of the
// launch on the context's stream.  The chains' values stay in [0, 2] and
// every chain's end value is stored, so no work can be dropped.
#include <cuda_runtime.h>

#include <sstream>

#include "sor_devfn.cuh"
#include "sor_runtime.h"

namespace sorgb {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;  // 2048 threads per SM: full occupancy
constexpr int kProbeIters = 1 << 14;  // about 70 ms per launch at the nominal rate

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_rate(int iters, double a, double b, double* out) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x & 7) * 0.125 + (double)k * 0.01;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (KIND == 0)
        x[k] = __fma_rn(x[k], a, b);  // contracts towards b / (1 - a)
      else
        x[k] = __dadd_rn(x[k], (it & 1) ? -b : b);  // oscillates around its start
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s = __dadd_rn(s, x[k]);
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

sor_status diag_fp64_rate(Ctx* c, int kind, double* ops_per_s) {
  if (!ops_per_s || (kind != 0 && kind != 1)) {
    c->set_error("kind must be 0 (FMA) or 1 (addition), ops_per_s non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  const int blocks = c->sm_count * kProbeBlocksPerSm;
  const size_t out_bytes = (size_t)blocks * kProbeThreads * sizeof(double);
  double* out = (double*)ctx_dev_alloc(c, out_bytes);
  if (!out) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  const double a = 0.5, b = 0.5;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, c->stream);
    if (e != cudaSuccess) break;
    if (kind == 0)
      k_fp64_rate<0><<<blocks, kProbeThreads, 0, c->stream>>>(kProbeIters, a, b * 1e-3, out);
    else
      k_fp64_rate<1><<<blocks, kProbeThreads, 0, c->stream>>>(kProbeIters, a, b * 1e-3, out);
    count_kernel_launches(1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ctx_dev_free(c, out);
  if (e != cudaSuccess) {
    std::ostringstream os;
    os << "FP64 rate probe: " << cudaGetErrorString(e);
    c->set_error(os.str());
    cudaGetLastError();
    return SOR_ERR_CUDA;
  }
  const double ops = (double)blocks * kProbeThreads * (double)kProbeIters * kChains;
  *ops_per_s = ms > 0.0f ? ops / (ms * 1e-3) : 0.0;
  return SOR_OK;
}

// One index through the debug build's check, an index below a one-element
// range: the check must refuse it and record kErrBounds.  No memory is
// accessed at that index in any build; release builds compile the check away
// and report that it did not fire.
__global__ void k_dbg_probe(SlotState* st, int* fired) { *fired = dbg_range(-1, 0, 1, st) ? 0 : 1; }

sor_status diag_bounds(Ctx* c, int* fired) {
  if (!fired) {
    c->set_error("fired must be non-NULL");
    return SOR_ERR_INVALID_ARG;
  }
  const size_t bytes = sizeof(SlotState) + 256;
  unsigned char* buf = (unsigned char*)ctx_dev_alloc(c, bytes);
  if (!buf) {
    c->set_error("device allocation failed");
    return SOR_ERR_OOM;
  }
  SlotState* st = (SlotState*)buf;
  int* out = (int*)(buf + sizeof(SlotState) + 128);
  SlotState hs;
  int hf = -1;
  cudaError_t e = cudaMemsetAsync(buf, 0, bytes, c->stream);
  if (e == cudaSuccess) {
    k_dbg_probe<<<1, 1, 0, c->stream>>>(st, out);
    count_kernel_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, out, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  ctx_dev_free(c, buf);
  if (e != cudaSuccess) {
    c->set_error(cudaGetErrorString(e));
    cudaGetLastError();
    return SOR_ERR_CUDA;
  }
  if (hf != 0 && hf != 1) return SOR_ERR_INTERNAL;
  if (hf == 1 && hs.error != kErrBounds) return SOR_ERR_INTERNAL;  // fired but recorded nothing
  *fired = hf;
  return SOR_OK;
}

}  // namespace sorgb
