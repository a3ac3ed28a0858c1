// observables.cu -- FP64 reductions for norm, populations and energy.
//
// Sec. II A: norm ||psi||, surface populations ||psi_s||^2 and the energy
// <psi|H|psi>.  With the grid measure dV = prod_d dq_d:
//   pops_s = dV sum_q |psi_s(q)|^2,
//   <V>    = dV sum_q Re sum_{r,c} conj(psi_r) V_rc psi_c,
//   <T>    = dV / P sum_k T(p_k) sum_s |psi~_s(p_k)|^2   (Parseval for the
//            unnormalised forward FFT), T(p) = sum_d p_d^2 / (2 m_d).
// Two launches: per-block partial sums (each block walks a fixed strided set
// of grid points), then one block adds the partials in block order, so the
// result does not depend on scheduling.  The caller applies dV.
#include "dso_internal.h"

namespace dso {

namespace {
constexpr int kBlocks = 608;  // 4 x 152 SMs
constexpr int kThreads = 256;
constexpr int kMaxCols = DSO_OBS_COLS;
}  // namespace

int obs_partial_blocks() { return kBlocks; }

__global__ void obs_partial_kernel(ObsArgs a, double* __restrict__ partials) {
  __shared__ double red[kThreads];
  const int ncol = a.S + 2;  // pops[S], <V>, <T> (unscaled)
  double acc[kMaxCols];
  for (int c = 0; c < kMaxCols; ++c) acc[c] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.P; g += stride) {
    double2 x[4];
    for (int s = 0; s < a.S; ++s) {
      x[s] = a.psi[(size_t)s * a.P + g];
      acc[s] += x[s].x * x[s].x + x[s].y * x[s].y;
    }
    double ev = 0.0;
    int k = 0;
    for (int r = 0; r < a.S; ++r)
      for (int c = r; c < a.S; ++c) {
        const double v = a.V[(size_t)k * a.P + g];
        const double re = x[r].x * x[c].x + x[r].y * x[c].y;  // Re conj(x_r) x_c
        ev += (r == c) ? v * re : 2.0 * v * re;
        ++k;
      }
    acc[a.S] += ev;
    // kinetic weight of this momentum grid point
    long long rem = g;
    double T = 0.0;
    int64_t off = 0;
    int64_t offs[3];
    for (int d = 0; d < a.D; ++d) {
      offs[d] = off;
      off += a.n[d];
    }
    for (int d = a.D - 1; d >= 0; --d) {
      const int64_t kd = rem % a.n[d];
      rem /= a.n[d];
      T += a.Tax[offs[d] + kd];
    }
    double m2 = 0.0;
    for (int s = 0; s < a.S; ++s) {
      const double2 y = a.psik[(size_t)s * a.P + g];
      m2 += y.x * y.x + y.y * y.y;
    }
    acc[a.S + 1] += T * m2;
  }
  for (int c = 0; c < ncol; ++c) {
    red[threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * ncol + c] = red[0];
    __syncthreads();
  }
}

__global__ void obs_final_kernel(const double* __restrict__ partials, int nblocks, int ncol, double* out) {
  const int c = threadIdx.x;
  if (c >= ncol) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * ncol + c];
  out[c] = s;
}

cudaError_t launch_observables(const ObsArgs& a, double* partials, double* out, cudaStream_t st) {
  obs_partial_kernel<<<kBlocks, kThreads, 0, st>>>(a, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  obs_final_kernel<<<1, 32, 0, st>>>(partials, kBlocks, a.S + 2, out);
  return cudaGetLastError();
}

}  // namespace dso
