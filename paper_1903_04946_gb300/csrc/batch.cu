// batch.cu -- one persistent launch per composed time step for many jobs
// with uneven grids (the batch slots of include/dso.h).
//
// Every job in a batch has its own grid, surfaces, potential, scheme and time
// step; one composed step of a job is its own sequence of axis passes
// (capi.cu), each a set of independent tiles.  A launch runs one composed
// step of every unfinished job: its work list is the passes of all jobs, cut
// into segments (one pass of one job), ordered by the pass's position in its
// job's step ("round") and then by job, so that a job's pass r comes after
// its pass r - 1.  The items of the list (one tile each) are numbered in that
// order and handed out by one global counter, one to each CTA as it starts;
// a CTA that takes a tile of a job's pass r first waits until every tile of
// that job's pass r - 1 has completed (a counter per segment).  Only running
// CTAs take items, and an item depends only on items with smaller numbers,
// all of which are already held by running (or finished) CTAs; so the lowest
// unfinished item can always proceed and the launch cannot deadlock, whatever
// the order in which the hardware starts its CTAs.  The wait is bounded all
// the same: after kBatchWaitPolls polls it records code 6 and goes on.
//
// Within a launch a pass reads what another SM wrote earlier in the same
// launch, so the tile body (axis_pass_rt.cuh) moves the wavefunction through
// L2 only; the completion counters are released by a device-scope fence and
// acquired with ld.acquire.gpu, and a block barrier passes the acquired data
// on to the CTA's other threads.
#include <cuda_runtime.h>

#include "axis_pass_rt.cuh"
#include "dso_internal.h"

namespace dso {

namespace {

constexpr int kBatchWaitPolls = 1 << 24;  // with a 128 ns back-off: a few seconds

// Resident CTAs per SM the register allocation must allow: 4 (64 registers;
// 144 bytes of spills per thread in FP64, none in FP32).  Measured on the
// 544-job batching mix: 0.657 s per 10 steps with 2 (124 registers, no
// spills), 0.582 s with 3, 0.575 s with 4.
#ifndef DSO_BATCH_MIN_BLOCKS
#define DSO_BATCH_MIN_BLOCKS 4
#endif

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One work item (one tile) per CTA, taken from the ordered counter when the
// CTA starts (not by blockIdx, so that items are taken in order by running
// CTAs only).  A persistent loop over items would let the compiler keep the
// loop-invariant shared-memory addresses of every FFT stage live across
// items: over 250 registers with spills; here the register count is set by
// the occupancy bound below.
template <typename C>
__global__ void __launch_bounds__(kRtThreads, DSO_BATCH_MIN_BLOCKS) batch_worklist_kernel(const BatchSeg* __restrict__ segs, int nseg,
                                                                     const BatchPass* __restrict__ passes,
                                                                     long long total,
                                                                     unsigned long long* __restrict__ head,
                                                                     unsigned* __restrict__ done,
                                                                     int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  __shared__ long long s_item;
  __shared__ int s_seg;
  __shared__ __align__(16) BatchPass s_pass;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const long long item = (long long)atomicAdd(head, 1ull);
    s_item = item;
    if (item < total) {
      // the segment holding the item: the last one starting at or before it
      int lo = 0, hi = nseg - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].item0 <= item) lo = mid; else hi = mid - 1;
      }
      s_seg = lo;
      const int prev = segs[lo].prev;
      if (prev >= 0) {  // every tile of the job's previous pass must be done
        const unsigned need = (unsigned)passes[segs[prev].pass].ntiles;
        int polls = 0;
        while (ld_acquire(&done[prev]) < need) {
          if (++polls > kBatchWaitPolls) {
            atomicExch(err, 6);
            break;
          }
          __nanosleep(128);
        }
      }
    }
  }
  __syncthreads();
  const long long item = s_item;
  if (item >= total) return;
  const BatchSeg sg = segs[s_seg];
  // the pass's arguments into shared memory, read there by every thread
  {
    const int* src = reinterpret_cast<const int*>(&passes[sg.pass]);
    int* dst = reinterpret_cast<int*>(&s_pass);
    for (int w = tid; w < (int)(sizeof(BatchPass) / sizeof(int)); w += kRtThreads) dst[w] = __ldg(&src[w]);
  }
  __syncthreads();
  tile_pass_rt<C>(sm, s_pass.a, s_pass.L, s_pass.log2L, s_pass.SV, item - sg.item0, tid, kRtThreads);
  __syncthreads();  // every store of the tile is issued
  if (tid == 0) {
    __threadfence();  // ... and visible at device scope before the count
    atomicAdd(&done[s_seg], 1u);
  }
}

template <typename C>
cudaError_t launch_t(const BatchSeg* segs, int nseg, const BatchPass* passes, long long total,
                     unsigned long long* head, unsigned* done, int* err, size_t smem, cudaStream_t st) {
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(batch_worklist_kernel<C>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (smem > 96 * 1024) return cudaErrorInvalidConfiguration;
  if (total < 1) return cudaSuccess;
  if (total > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  batch_worklist_kernel<C><<<(unsigned)total, kRtThreads, smem, st>>>(segs, nseg, passes, total, head, done, err);
  return cudaGetLastError();
}

}  // namespace

size_t batch_tile_smem(int L, int SV, int G, int Wi, bool fp32) {
  const int esz = fp32 ? 8 : 16;
  return (size_t)SV * G * tile_layout(L, esz, Wi).ls * esz;
}

int batch_max_tile_amplitudes() { return kRtMaxTile; }

cudaError_t launch_batch_worklist(bool fp32, const BatchSeg* segs, int nseg, const BatchPass* passes, long long total,
                                  unsigned long long* head, unsigned* done, int* err, size_t smem, cudaStream_t st) {
  return fp32 ? launch_t<float2>(segs, nseg, passes, total, head, done, err, smem, st)
              : launch_t<double2>(segs, nseg, passes, total, head, done, err, smem, st);
}

}  // namespace dso
