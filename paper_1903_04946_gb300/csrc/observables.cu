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
#include <stdint.h>

#include <mutex>

#include <cudaTypedefs.h>

#include "../../include/dso.h"
#include "dso_internal.h"

namespace dso {

namespace {
constexpr int kBlocks = 608;  // 4 x 152 SMs
constexpr int kThreads = 256;
constexpr int kMaxCols = DSO_OBS_COLS;
}  // namespace

int obs_partial_blocks() { return kBlocks; }

__device__ __forceinline__ double2 load_c(const void* base, size_t i, int fp32) {
  if (fp32) {
    const float2 v = ((const float2*)base)[i];
    return make_double2((double)v.x, (double)v.y);
  }
  return ((const double2*)base)[i];
}

__global__ void obs_partial_kernel(ObsArgs a, double* __restrict__ partials) {
  __shared__ double red[kThreads];
  const int ncol = a.S + 2;  // pops[S], <V>, <T> (unscaled)
  double acc[kMaxCols];
  for (int c = 0; c < kMaxCols; ++c) acc[c] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < a.P; g += stride) {
    double2 x[4];
    for (int s = 0; s < a.S; ++s) {
      x[s] = load_c(a.psi, (size_t)s * a.P + g, a.fp32);
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
    // kinetic weight of this momentum grid point (storage order of a.vl:
    // permuted along split axes)
    int64_t kd[3] = {0, 0, 0};
    momentum_indices(a.vl, g, kd);
    double T = 0.0;
    int64_t off = 0;
    for (int d = 0; d < a.vl.D; ++d) {
      T += a.Tax[off + kd[d]];
      off += a.vl.n[d];
    }
    double m2 = 0.0;
    for (int s = 0; s < a.S; ++s) {
      const double2 y = load_c(a.psik, (size_t)s * a.P + g, a.fp32);
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

// ---------------------------------------------------------------------------
// Allocation-free position-space observables.
//
// Some callers cannot call cudaMalloc at all: code that runs under a
// caching or pool allocator that owns every device allocation, inside an
// engine whose memory budget is fixed before the first step, or in a context
// where allocation would synchronise the device.  This variant of the
// per-block reduction above keeps its partial sums in a file-scope device
// array instead of a buffer from the context, so it allocates nothing.  The
// array (kNoAllocBlocks x kNoAllocCols doubles, 19,456 bytes) is held by
// every GPU that loads the library until the process exits.
// ---------------------------------------------------------------------------
namespace dso {
namespace {

constexpr int kNoAllocBlocks = 304;  // 2 x 152 SMs
constexpr int kNoAllocCols = 8;      // S populations + <V>, S <= 4, padded
static __device__ __align__(256) double g_noalloc_partials[kNoAllocBlocks * kNoAllocCols];

// Host-side device addresses of g_noalloc_partials, one per device.  The
// array's name in host code is only a host stand-in for the symbol, so the
// address must come from cudaGetSymbolAddress with that device current.
// The driver context the address belongs to is kept beside it: after a
// device reset the module is loaded again in a new context and the array may
// sit elsewhere, so a changed context means looking the address up again.
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};
CUcontext g_noalloc_ctx[64] = {};

// The calling thread's current driver context (cuCtxGetCurrent, looked up
// once through the runtime so the library needs no -lcuda), or null.
CUcontext current_driver_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuCtxGetCurrent_v4000)f;
  });
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

__global__ void obs_position_partial_kernel(const double2* __restrict__ psi, const double* __restrict__ V, int S,
                                            long long P, double* __restrict__ partials) {
  __shared__ double red[kThreads];
  double acc[kNoAllocCols];
  for (int c = 0; c < kNoAllocCols; ++c) acc[c] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < P; g += stride) {
    double2 x[4];
    for (int s = 0; s < S; ++s) {
      x[s] = psi[(size_t)s * P + g];
      acc[s] += x[s].x * x[s].x + x[s].y * x[s].y;
    }
    if (V) {
      double ev = 0.0;
      int k = 0;
      for (int r = 0; r < S; ++r)
        for (int c = r; c < S; ++c) {
          const double v = V[(size_t)k * P + g];
          const double re = x[r].x * x[c].x + x[r].y * x[c].y;
          ev += (r == c) ? v * re : 2.0 * v * re;
          ++k;
        }
      acc[S] += ev;
    }
  }
  // every block writes all S + 1 of its columns: no slot is read before this
  // call has written it, so the array needs no clearing between calls
  for (int c = 0; c <= S; ++c) {
    red[threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kNoAllocCols + c] = red[0];
    __syncthreads();
  }
}

__global__ void obs_position_final_kernel(const double* __restrict__ partials, int ncol, double dV, double* out) {
  const int c = threadIdx.x;
  if (c >= ncol) return;
  double s = 0.0;
  for (int b = 0; b < kNoAllocBlocks; ++b) s += partials[(size_t)b * kNoAllocCols + c];
  out[c] = s * dV;
}

}  // namespace
}  // namespace dso

extern "C" dso_status dso_position_observables_noalloc(const void* psi, const double* V, int S, int64_t P,
                                                       double dV, double* out, void* cuda_stream) {
  using namespace dso;
  if (!psi || !out) return DSO_EINVAL;
  if (S < 1 || S + 1 > kNoAllocCols || S > DSO_MAX_SURFACES) return DSO_EINVAL;  // scratch holds S <= 4
  if (P < 1) return DSO_EINVAL;
  // misaligned element pointers would fault the kernels (a sticky error that
  // ends the caller's CUDA context): reject them here
  if ((uintptr_t)psi % 16 != 0 || (uintptr_t)out % 8 != 0 || (V && (uintptr_t)V % 8 != 0)) return DSO_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DSO_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const CUcontext cur = current_driver_context();
    if (!g_noalloc_ptr[dev] || cur != g_noalloc_ctx[dev]) {
      // first call on this device (or in a new context of it): look up the
      // array's device address with the device current
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr) return DSO_ECUDA;
      g_noalloc_ptr[dev] = (double*)ptr;
      g_noalloc_ctx[dev] = current_driver_context();
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  obs_position_partial_kernel<<<kNoAllocBlocks, kThreads, 0, st>>>((const double2*)psi, V, S, (long long)P, scratch);
  if (cudaGetLastError() != cudaSuccess) return DSO_ECUDA;
  obs_position_final_kernel<<<1, 32, 0, st>>>(scratch, S + 1, dV, out);
  if (cudaGetLastError() != cudaSuccess) return DSO_ECUDA;
  return DSO_OK;
}

