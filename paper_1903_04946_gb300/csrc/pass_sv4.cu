// pass_sv4.cu -- axis-pass kernels staging 4 surface(s) per tile.
#include "pass_launch.cuh"

namespace dso {
cudaError_t launch_axis_pass_sv4(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                   const TmaMaps* maps, cudaStream_t st) {
  return launch_by_length<4>(L, variant, a, ntiles, queue, maps, st);
}
}  // namespace dso
