// diag.cu -- device diagnostics: the FP64 instruction rate this GPU sustains.
//
// The FP64 propagation path is bound by the FP64 pipe (a few FP64 lanes per
// SM): its FFT butterflies, potential matvecs and kinetic phases are chains of
// DFMA, DADD and DMUL with per-thread register operands.  This measures the
// rate at which the device retires such instructions, as the denominator of
// an instruction-rate roofline, next to the unit-count peak.
#include <cuda_runtime.h>

#include "../../include/dso.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// Every thread runs kChains independent chains x <- fma(x, y, z) with x, y
// and z in per-thread registers (the operand pattern of the butterflies).
// The result is written only when it is the impossible value -1 (every chain
// stays positive), so the store never happens but the chains cannot be
// removed; `sink` is one double.
__global__ void dfma_chains_kernel(int iters, double seed, double* sink) {
  double x[kChains], y[kChains], z[kChains];
  const double t = seed * (threadIdx.x + 1);
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    x[k] = t + k;
    y[k] = 0.999999 - 1e-9 * k;
    z[k] = 1e-7 * (k + 1) * t;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], y[k], z[k]);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0) sink[0] = s;
}

}  // namespace

extern "C" dso_status dso_fp64_issue_rate(int device, double* inst_per_s) {
  if (!inst_per_s) return DSO_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return DSO_ECUDA;
  if (device < 0 || device >= ndev) return DSO_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (cudaSetDevice(device) != cudaSuccess) return DSO_ECUDA;
  int nsm = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* sink = nullptr;
  dso_status rc = DSO_OK;
  const int threads = 256, iters = 4096;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, sizeof(double)) != cudaSuccess) {
    rc = DSO_ECUDA;
  } else {
    // 8 CTAs of 8 warps per SM keep every FP64 pipe fed
    const int blocks = 8 * nsm;
    float best = 0.f;
    for (int rep = 0; rep < 4 && rc == DSO_OK; ++rep) {  // the first is warm-up
      cudaEventRecord(e0, st);
      dfma_chains_kernel<<<blocks, threads, 0, st>>>(iters, 1.0 + rep, sink);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = DSO_ECUDA;
        break;
      }
      if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (rc == DSO_OK) {
      const double inst = (double)blocks * threads * (double)iters * kChains;
      *inst_per_s = best > 0.f ? inst / (best * 1e-3) : 0.0;
    }
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
