// pass_launch.cuh -- per-(L, SV) instantiation and launch of axis_pass_kernel.
#pragma once

#include "axis_pass.cuh"
#include "dso_internal.h"

namespace dso {

template <int L, int SV>
cudaError_t launch_one(const PassArgs& a, long long ntiles, cudaStream_t st) {
  static bool attr_set[64] = {};  // the attribute is set once per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const int threads = SV * a.G * (L / 8);
  const size_t smem = (size_t)SV * a.G * L * sizeof(double2);
  if (threads > MaxThreads<L, SV>::value) return cudaErrorInvalidConfiguration;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(axis_pass_kernel<L, SV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  axis_pass_kernel<L, SV><<<(unsigned)ntiles, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int SV>
cudaError_t launch_by_length(int L, const PassArgs& a, long long ntiles, cudaStream_t st) {
  switch (L) {
    case 8: return launch_one<8, SV>(a, ntiles, st);
    case 16: return launch_one<16, SV>(a, ntiles, st);
    case 32: return launch_one<32, SV>(a, ntiles, st);
    case 64: return launch_one<64, SV>(a, ntiles, st);
    case 128: return launch_one<128, SV>(a, ntiles, st);
    case 256: return launch_one<256, SV>(a, ntiles, st);
    case 512: return launch_one<512, SV>(a, ntiles, st);
    case 1024: return launch_one<1024, SV>(a, ntiles, st);
    case 2048:
      if constexpr (SV * 2048 <= 8192) return launch_one<2048, SV>(a, ntiles, st);
      break;
    case 4096:
      if constexpr (SV * 4096 <= 8192) return launch_one<4096, SV>(a, ntiles, st);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace dso
