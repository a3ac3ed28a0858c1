// pass_sv3.cu -- axis-pass kernels staging 3 surface(s) per tile.
#include "pass_launch.cuh"

namespace dso {
cudaError_t launch_axis_pass_sv3(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                   const TmaMaps* maps, cudaStream_t st) {
  return launch_by_length<3>(L, variant, a, ntiles, queue, maps, st);
}
}  // namespace dso
