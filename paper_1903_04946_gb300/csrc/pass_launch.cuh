// pass_launch.cuh -- per-(L, SV) instantiation and launch of axis_pass_kernel.
#pragma once

#include <utility>

#include "axis_pass.cuh"
#include "axis_pass_pq.cuh"
#include "axis_pass_reg.cuh"
#include "axis_pass_tma.cuh"
#include "dso_internal.h"

namespace dso {

// Launch `k` on `st`; with `pdl`, as a programmatic dependent launch, so the
// kernel's CTAs may start while the previous kernel on the stream finishes
// (each axis-pass kernel waits for it with griddepcontrol.wait before its
// first read of the wavefunction).  Inside stream capture this becomes a
// programmatic edge of the CUDA graph.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, bool pdl,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <int L, int SV, typename C>
cudaError_t launch_one_t(const PassArgs& a, long long ntiles, cudaStream_t st) {
  static bool attr_set[64] = {};  // the attribute is set once per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const int threads = SV * a.G * (L / 8);
  const int Wi = 1 << (a.stride_log2 < a.G_log2 ? a.stride_log2 : a.G_log2);  // as make_geom
  const size_t smem = (size_t)SV * a.G * tile_layout(L, (int)sizeof(C), Wi).ls * sizeof(C);
  if (threads > MaxThreads<L, SV>::value || smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(axis_pass_kernel<L, SV, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const cudaError_t e = launch_k(axis_pass_kernel<L, SV, C>, (unsigned)ntiles, threads, smem, st, a.pdl != 0, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int L, int SV>
cudaError_t launch_one(const PassArgs& a, long long ntiles, cudaStream_t st) {
  return a.fp32 ? launch_one_t<L, SV, float2>(a, ntiles, st) : launch_one_t<L, SV, double2>(a, ntiles, st);
}

// Shared memory of the persistent variant: two psi tile buffers and one
// table buffer (S(S+1)/2 potential entries, or one kinetic phase, per point).
inline size_t pq_smem_bytes(int L, int SV, int G) {
  const int np = SV > 1 ? SV * (SV + 1) / 2 : 1;
  return (size_t)(2 * SV + np) * G * L * sizeof(double2);
}

template <int L, int SV>
cudaError_t launch_pq(const PassArgs& a, long long ntiles, unsigned* queue, cudaStream_t st) {
  static bool attr_set[64] = {};
  static int nsm[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const int threads = SV * a.G * (L / 8);
  const size_t smem = pq_smem_bytes(L, SV, a.G);
  if (threads > 256 || smem > 200 * 1024 || !queue) return cudaErrorInvalidConfiguration;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(axis_pass_pq_kernel<L, SV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, axis_pass_pq_kernel<L, SV>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * nsm[dev];
  if (grid > ntiles) grid = ntiles;
  e = launch_k(axis_pass_pq_kernel<L, SV>, (unsigned)grid, threads, smem, st, a.pdl != 0, a, queue);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int L, int SV>
cudaError_t launch_tma(const PassArgs& a, const TmaMaps* maps, long long ntiles, cudaStream_t st) {
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const int threads = SV * a.G * (L / 8);
  const size_t smem = tma_smem_bytes<L, SV>(a.G);
  if (threads > 256 || smem > 220 * 1024 || !maps) return cudaErrorInvalidConfiguration;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(axis_pass_tma_kernel<L, SV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         220 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const cudaError_t e = launch_k(axis_pass_tma_kernel<L, SV>, (unsigned)ntiles, threads, smem, st, a.pdl != 0, a,
                                 *maps);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Persistent TMA variant: a grid of min(ntiles, CTAs per SM x SMs) CTAs
// drains the tile queue.
template <int L, int SV>
cudaError_t launch_tmap(const PassArgs& a, const TmaMaps* maps, long long ntiles, unsigned* queue, cudaStream_t st) {
  static bool attr_set[64] = {};
  static int nsm[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const int threads = SV * a.G * (L / 8);
  const bool has_tab = (SV > 1 && a.U1) || (a.flags & PASS_T);
  if ((SV > 1 && a.U1) && (a.flags & PASS_T)) return cudaErrorInvalidConfiguration;  // 1-D passes
  const size_t smem = tmap_smem_bytes<L, SV>(a.G, has_tab);
  if (threads > 256 || smem > 220 * 1024 || !maps || !queue) return cudaErrorInvalidConfiguration;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(axis_pass_tmap_kernel<L, SV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         220 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, axis_pass_tmap_kernel<L, SV>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (a.ctas_per_sm > 0 && a.ctas_per_sm < per_sm) per_sm = a.ctas_per_sm;
  long long grid = (long long)per_sm * nsm[dev];
  if (grid > ntiles) grid = ntiles;
  e = launch_k(axis_pass_tmap_kernel<L, SV>, (unsigned)grid, threads, smem, st, a.pdl != 0, a, *maps, queue);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Register-resident variant (lines of 32..128 points): reg_lines<L, SV>() line
// positions of SV surfaces per CTA, contiguous lines or lines of one outer row.
template <int L, int SV, typename C>
cudaError_t launch_reg_t(const PassArgs& a, long long ntiles, cudaStream_t st) {
  constexpr bool split_fits = SV >= 3 && reg_fits<L, (SV >= 3 ? SV - 1 : 1), C>();
  if constexpr (!reg_fits<L, SV, C>() && !split_fits) {
    return cudaErrorInvalidConfiguration;
  } else {
    static bool attr_set[2][2][64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const bool contig = a.stride_log2 == 0;
    if (a.G != reg_lines<L, SV>() || (SV == 1 && (a.U1 || a.U2)) || (a.flags & PASS_XTW) ||
        (!contig && a.stride_log2 < a.G_log2))
      return cudaErrorInvalidConfiguration;
    // surface 0 decoupled: a CTA for it and one for the block of the others
    const bool split = split_fits && a.dec0 && a.U1;
    if (!split && !reg_fits<L, SV, C>()) return cudaErrorInvalidConfiguration;
    constexpr int NP = SV * (SV + 1) / 2, NPB = SV * (SV - 1) / 2;
    const int np_staged = split ? NPB : (SV > 1 && a.U1) ? (SV > 2 && a.dec0 ? NP - (SV - 1) : NP) : 0;
    const size_t smem = reg_smem_bytes<L, SV>(contig, sizeof(C) == 8, np_staged);
    const size_t smem_max = reg_smem_bytes<L, SV>(contig, sizeof(C) == 8, SV > 1 ? NP : 0);
    if (smem_max > 227 * 1024) return cudaErrorInvalidConfiguration;
    void (*k)(PassArgs) = nullptr;
    if constexpr (split_fits) {
      if (split)
        k = contig ? axis_pass_reg_split_kernel<L, (SV >= 3 ? SV : 3), true, C>
                   : axis_pass_reg_split_kernel<L, (SV >= 3 ? SV : 3), false, C>;
    }
    if constexpr (reg_fits<L, SV, C>()) {
      if (!split) k = contig ? axis_pass_reg_kernel<L, SV, true, C> : axis_pass_reg_kernel<L, SV, false, C>;
    }
    if (!k) return cudaErrorInvalidConfiguration;
    if (!attr_set[split][contig][dev]) {
      const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
      if (e != cudaSuccess) return e;
      attr_set[split][contig][dev] = true;
    }
    const cudaError_t e =
        launch_k(k, (unsigned)(split ? 2 * ntiles : ntiles), reg_threads<SV>(), smem, st, a.pdl != 0, a);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
}

template <int L, int SV>
cudaError_t launch_variant(int variant, const PassArgs& a, long long ntiles, unsigned* queue, const TmaMaps* maps,
                           cudaStream_t st) {
  if (variant == 4) {  // FP64 and FP32
    if constexpr (L == 32 || L == 64 || L == 128)
      return a.fp32 ? launch_reg_t<L, SV, float2>(a, ntiles, st) : launch_reg_t<L, SV, double2>(a, ntiles, st);
    return cudaErrorInvalidConfiguration;
  }
  if (variant != 0 && a.fp32) return cudaErrorInvalidConfiguration;  // FP64 only
  if (variant != 0 && (a.flags & PASS_TAX)) return cudaErrorInvalidConfiguration;  // grid-sized tables only
  if (variant != 0 && (a.flags & PASS_XTW)) return cudaErrorInvalidConfiguration;  // split axes: tile kernel
  if (variant == 1) {
    if constexpr (SV * L / 8 <= 256) return launch_pq<L, SV>(a, ntiles, queue, st);
    return cudaErrorInvalidConfiguration;
  }
  if (variant == 2) {
    if constexpr (L <= 256 && SV * L / 8 <= 256) return launch_tma<L, SV>(a, maps, ntiles, st);
    return cudaErrorInvalidConfiguration;
  }
  if (variant == 3) {
    if constexpr (L <= 256 && SV * L / 8 <= 256) return launch_tmap<L, SV>(a, maps, ntiles, queue, st);
    return cudaErrorInvalidConfiguration;
  }
  return launch_one<L, SV>(a, ntiles, st);
}

template <int SV>
cudaError_t launch_by_length(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                             const TmaMaps* maps, cudaStream_t st) {
  switch (L) {
    case 8: return launch_variant<8, SV>(variant, a, ntiles, queue, maps, st);
    case 16: return launch_variant<16, SV>(variant, a, ntiles, queue, maps, st);
    case 32: return launch_variant<32, SV>(variant, a, ntiles, queue, maps, st);
    case 64: return launch_variant<64, SV>(variant, a, ntiles, queue, maps, st);
    case 128: return launch_variant<128, SV>(variant, a, ntiles, queue, maps, st);
    case 256: return launch_variant<256, SV>(variant, a, ntiles, queue, maps, st);
    case 512: return launch_variant<512, SV>(variant, a, ntiles, queue, maps, st);
    case 1024: return launch_variant<1024, SV>(variant, a, ntiles, queue, maps, st);
    case 2048:
      if constexpr (SV * 2048 <= 8192) return launch_variant<2048, SV>(variant, a, ntiles, queue, maps, st);
      break;
    case 4096:
      if constexpr (SV * 4096 <= 8192) return launch_variant<4096, SV>(variant, a, ntiles, queue, maps, st);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace dso
