// pass_plane.cu -- instantiation and launch of the plane passes
// (axis_pass_plane.cuh) of the per-axis and the joint kinetic step: planes of
// LA x LB points, LA, LB in {32, 64, 128}.
#include "axis_pass_plane.cuh"
#include "dso_internal.h"

namespace dso {
namespace {

template <int LA, int LB, typename C>
cudaError_t launch_plane_t(const PassArgs& a, long long nplanes, cudaStream_t st) {
  if constexpr (!reg_fits<LA, 1, C>() || !reg_fits<LB, 1, C>()) {
    return cudaErrorInvalidConfiguration;
  } else {
    using PG = PlaneGeom<LA, LB, C>;
    // per-axis phases (PASS_TAX): one exchange; the grid's phase: two
    const bool axes = (a.flags & PASS_TAX) != 0;
    constexpr size_t smem_axes = plane_smem_bytes<LA, LB, C>(), smem_joint = plane_joint_smem_bytes<LA, LB, C>();
    static_assert(smem_axes <= 227 * 1024 && smem_joint <= 227 * 1024, "plane pass shared memory");
    const size_t smem = axes ? smem_axes : smem_joint;
    static bool attr_set[2][64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void (*k)(PassArgs) = axes ? axis_pass_plane_kernel<LA, LB, C> : axis_pass_plane_joint_kernel<LA, LB, C>;
    if (!attr_set[axes][dev]) {
      const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set[axes][dev] = true;
    }
    const long long ctas = nplanes * PG::K;
    if (nplanes < 1 || ctas > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = PG::K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.pdl ? 2 : 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
}

template <int LA, typename C>
cudaError_t launch_plane_b(int LB, const PassArgs& a, long long nplanes, cudaStream_t st) {
  switch (LB) {
    case 32: return launch_plane_t<LA, 32, C>(a, nplanes, st);
    case 64: return launch_plane_t<LA, 64, C>(a, nplanes, st);
    case 128: return launch_plane_t<LA, 128, C>(a, nplanes, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename C>
cudaError_t launch_plane_c(int LA, int LB, const PassArgs& a, long long nplanes, cudaStream_t st) {
  switch (LA) {
    case 32: return launch_plane_b<32, C>(LB, a, nplanes, st);
    case 64: return launch_plane_b<64, C>(LB, a, nplanes, st);
    case 128: return launch_plane_b<128, C>(LB, a, nplanes, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

}  // namespace

bool axis_pass_plane_supported(int LA, int LB, bool fp32) {
  auto ok = [](int L) { return L == 32 || L == 64 || L == 128; };
  if (!ok(LA) || !ok(LB)) return false;
  // a thread's amplitudes of one line fit its registers (reg_fits)
  const int w = fp32 ? 2 : 4;
  return (LA == 128 ? 16 : 8) * w <= 96 && (LB == 128 ? 16 : 8) * w <= 96;
}

cudaError_t launch_axis_pass_plane(int LA, int LB, const PassArgs& a, long long nplanes, cudaStream_t st) {
  const int need = PASS_FWD | PASS_T | PASS_PLANE;  // with or without PASS_TAX
  if ((a.flags & need) != need || (a.flags & (PASS_INV_FIRST | PASS_XTW)) || a.U1 || a.U2 || !a.tau || !a.tw ||
      !a.tw2 || a.stride != LB || !axis_pass_plane_supported(LA, LB, a.fp32 != 0) ||
      nplanes * LA * LB != (long long)a.nbatch * a.S * a.P)
    return cudaErrorInvalidConfiguration;
  return a.fp32 ? launch_plane_c<float2>(LA, LB, a, nplanes, st) : launch_plane_c<double2>(LA, LB, a, nplanes, st);
}

}  // namespace dso
