// pass_sv1.cu -- axis-pass kernels staging 1 surface(s) per tile.
#include "pass_launch.cuh"

namespace dso {
cudaError_t launch_axis_pass_sv1(int L, const PassArgs& a, long long ntiles, cudaStream_t st) {
  return launch_by_length<1>(L, a, ntiles, st);
}
}  // namespace dso
