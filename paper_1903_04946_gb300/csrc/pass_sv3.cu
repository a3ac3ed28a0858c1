// pass_sv3.cu -- axis-pass kernels staging 3 surface(s) per tile.
#include "pass_launch.cuh"

namespace dso {
cudaError_t launch_axis_pass_sv3(int L, const PassArgs& a, long long ntiles, cudaStream_t st) {
  return launch_by_length<3>(L, a, ntiles, st);
}
}  // namespace dso
