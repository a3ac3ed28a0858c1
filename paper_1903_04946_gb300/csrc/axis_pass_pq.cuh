// axis_pass_pq.cuh -- persistent, prefetching variant of the axis pass.
//
// Same arithmetic as axis_pass_kernel (axis_pass.cuh): per tile, optional
// inverse FFT, potential matvec(s), forward FFT, kinetic phase + inverse FFT,
// along one axis.  What changes is how tiles reach the FP64 pipe:
//
//  * a grid of a few CTAs per SM takes tiles from a per-launch queue (one
//    atomic per tile), so every SM stays busy until the queue drains and the
//    tail is one tile, not one wave;
//  * while a tile is transformed, the CTA's next tile streams into a second
//    shared-memory buffer with cp.async, and the potential (or kinetic) table
//    entries of the current tile stream in during its first FFT, so the
//    FP64 work never waits on global memory;
//  * for 64-point lines the second-stage twiddles of each thread are fixed and
//    live in registers.
//
// The queue is two counters in device memory, zero before a launch: the CTA
// that finishes last resets them, so consecutive launches on one stream (and
// CUDA-graph replays) reuse them without a memset.
#pragma once

#include "axis_pass.cuh"

namespace dso {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Stage with per-thread twiddles held in registers (used for the last stage
// of 64-point lines, where each thread's k is fixed for the whole launch).
template <int L, bool INV>
__device__ __forceinline__ void stockham8_regtw(double2* sm, int Ls, const double2 (&w)[4], int nslots, int tid,
                                                unsigned wmask) {
  constexpr int Q = L / 8;
  double2 v[8];
  const bool act = tid < nslots;
  const int line = tid / (L / 8);
  const int u = tid % (L / 8);
  double2* ln = sm + (size_t)line * L;
  if (act) {
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = ln[u + r * Q];
  }
  stage_sync<L>(wmask);
  if (act) {
    const int k = u & (Ls - 1);
    dft8_tw<INV>(v, w[0], w[1], w[2], w[3]);
    const int base = (u - k) * 8 + k;
#pragma unroll
    for (int r = 0; r < 8; ++r) ln[base + r * Ls] = v[r];
  }
  stage_sync<L>(wmask);
}

template <int L, bool INV>
__device__ __forceinline__ void fft_lines_pq(double2* sm, const double2* __restrict__ tw, const double2 (&wreg)[4],
                                             int nslots, int tid, int nthr) {
  using PL = Plan<L>;
  const unsigned wmask = warp_lanes_mask(tid, nthr);
  if constexpr (L == 64) {
    stockham_stage<L, 8, INV, 1>(sm, 1, tw, nslots, tid, nthr, wmask, plain_layout(L));
    stockham8_regtw<L, INV>(sm, 8, wreg, nslots, tid, wmask);
  } else {
    stockham_stage<L, PL::first, INV, 1>(sm, 1, tw, nslots, tid, nthr, wmask, plain_layout(L));
    int Ls = PL::first;
#pragma unroll 1
    for (int st = 0; st < PL::n8; ++st) {
      stockham_stage<L, 8, INV, 1>(sm, Ls, tw, nslots, tid, nthr, wmask, plain_layout(L));
      Ls *= 8;
    }
  }
}

struct PqTile {
  TileGeom tg;
  int surf0;
  size_t uoff;  // this job's offset into the potential tables
};

__device__ __forceinline__ PqTile pq_tile(long long tile, int SV, const PassArgs& a) {
  PqTile t;
  const TileJob tj = split_tile(tile, SV, a);
  t.surf0 = tj.surf0;
  t.uoff = (size_t)tj.job * a.u_batch_stride;
  t.tg = make_geom(tj.tile, a);
  return t;
}

// Issue the cp.async copies of `count` complex entries per tile element of
// `src` ([count][P] layout, or [S][P] for psi) into `dst` ([count][G*L]).
template <int L>
__device__ __forceinline__ void pq_issue(double2* dst, const double2* src, int count, long long P, const PqTile& t,
                                         int G, long long stride, int tid, int nthr, const double2* base = nullptr,
                                         long long extent = 0, int* err = nullptr) {
  const int tile_pts = G * L;
#pragma unroll 1
  for (int c = 0; c < count; ++c) {
    const double2* s = src + (size_t)c * P;
    double2* d = dst + (size_t)c * tile_pts;
#pragma unroll 1
    for (int e = tid; e < tile_pts; e += nthr) {
      int g, n;
      tile_elem<L>(e, t.tg, g, n);
#ifdef DSO_DEBUG_BOUNDS
      if (base && !DSO_CHECK_INDEX((long long)(&s[t.tg.addr(g, n, L, stride)] - base), extent, 110, err)) continue;
#endif
      cp_async16(&d[g * L + n], &s[t.tg.addr(g, n, L, stride)]);
    }
  }
}

template <int SV>
__device__ __forceinline__ void pq_potential(double2* sm, const double2* ub, int tile_pts, int tid, int nthr,
                                             int dec0) {
  constexpr int NP = SV * (SV + 1) / 2;
#pragma unroll 1
  for (int e = tid; e < tile_pts; e += nthr) {
    double2 x[SV], y[SV], u[NP];
#pragma unroll
    for (int s = 0; s < SV; ++s) x[s] = sm[(size_t)s * tile_pts + e];
#pragma unroll
    for (int k = 0; k < NP; ++k)
      u[k] = (SV > 2 && dec0 && k >= 1 && k < SV) ? make_double2(0.0, 0.0) : ub[(size_t)k * tile_pts + e];
    matvec_sym<SV>(u, x, y, dec0);
#pragma unroll
    for (int s = 0; s < SV; ++s) sm[(size_t)s * tile_pts + e] = y[s];
  }
}

// Shared memory: psi buffers [2][SV][G*L], then a table buffer
// [max(NP, 1)][G*L] (potential unitary entries, or kinetic phases).
template <int L, int SV>
__global__ void __launch_bounds__(256) axis_pass_pq_kernel(PassArgs a, unsigned* __restrict__ queue) {
  extern __shared__ double2 sm[];
  __shared__ long long s_next;
  constexpr int NP = SV * (SV + 1) / 2;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = a.G;
  const int tile_pts = G * L;
  const int tsize = SV * tile_pts;
  double2* const buf0 = sm;
  double2* tb = sm + 2 * tsize;
  const long long ntiles = (SV == a.S) ? (long long)a.nbatch * (a.lines / G)
                                       : (long long)a.nbatch * a.S * (a.lines / G);
  const int nslots = SV * G * (L / 8);

  // register twiddles for the second stage of 64-point lines
  double2 wreg[4];
  if constexpr (L == 64) {
    const int k = (tid % (L / 8)) & 7;
    load_tw8<L>((const double2*)a.tw, k, wreg[0], wreg[1], wreg[2], wreg[3]);
  }

  __shared__ long long s_first;
  pdl_wait();  // psi and the queue reset are the previous pass's
  pdl_trigger();
  if (tid == 0) s_first = (long long)atomicAdd(&queue[0], 1u);
  __syncthreads();
  long long cur = s_first;
  if (cur < ntiles) {
    const PqTile t = pq_tile(cur, SV, a);
    pq_issue<L>(buf0, (double2*)a.psi + (size_t)t.surf0 * a.P, SV, a.P, t, G, a.stride, tid, nthr,
                (const double2*)a.psi, a.psi_elems, a.err);
  }
  cp_async_commit();
  int b = 0;
  while (cur < ntiles) {
    if (tid == 0) s_next = (long long)atomicAdd(&queue[0], 1u);
    __syncthreads();  // s_next published; buf[b^1] free (its store finished)
    const long long nxt = s_next;
    if (nxt < ntiles) {
      const PqTile t = pq_tile(nxt, SV, a);
      pq_issue<L>(buf0 + (b ^ 1) * tsize, (double2*)a.psi + (size_t)t.surf0 * a.P, SV, a.P, t, G, a.stride, tid,
                  nthr, (const double2*)a.psi, a.psi_elems, a.err);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of the current tile landed
    __syncthreads();

    const PqTile t = pq_tile(cur, SV, a);
    double2* x = buf0 + b * tsize;
    const bool vstep = (SV > 1) && (a.U1 != nullptr);
    // stream the current tile's table entries in behind the first FFT
    if (vstep) {
      pq_issue<L>(tb, (const double2*)a.U1 + t.uoff, NP, a.P, t, G, a.stride, tid, nthr,
                  (const double2*)a.U_base, a.u_elems, a.err);
    } else if (a.flags & PASS_T) {
      pq_issue<L>(tb, (const double2*)a.tau, 1, a.P, t, G, a.stride, tid, nthr, (const double2*)a.tau_base,
                  a.tau_elems, a.err);
    }
    cp_async_commit();

    if (a.flags & PASS_INV_FIRST) fft_lines_pq<L, true>(x, (const double2*)a.tw, wreg, nslots, tid, nthr);
    if (vstep) {
      cp_async_wait<0>();
      __syncthreads();
      // table and psi buffers share the [g][n] order, so pq_potential walks
      // both with one flat index
      pq_potential<SV>(x, tb, tile_pts, tid, nthr, a.dec0);
      __syncthreads();
      if (a.U2) {
        apply_potential<L, SV>(x, (const double2*)a.U2 + t.uoff, t.tg, G, a.stride, a.P, tid, nthr, plain_layout(L),
                               &a);
      }
      if (a.flags & PASS_T) {  // 1-D grids: the kinetic phase follows in this pass
        pq_issue<L>(tb, (const double2*)a.tau, 1, a.P, t, G, a.stride, tid, nthr);
        cp_async_commit();
      }
    }
    if (a.flags & PASS_FWD) fft_lines_pq<L, false>(x, (const double2*)a.tw, wreg, nslots, tid, nthr);
    if (a.flags & PASS_T) {
      cp_async_wait<0>();
      __syncthreads();
#pragma unroll 1
      for (int e = tid; e < tile_pts; e += nthr) {
        const double2 ph = tb[e];
        for (int s = 0; s < SV; ++s) {
          double2* p = &x[(size_t)s * tile_pts + e];
          *p = cmul(*p, ph);
        }
      }
      __syncthreads();
      if (a.tau2) {  // second kinetic phase of a step boundary, from global memory
#pragma unroll 1
        for (int e = tid; e < tile_pts; e += nthr) {
          const int g = e / L, n = e - (e / L) * L;
          double2 ph = __ldg(&((const double2*)a.tau2)[t.tg.addr(g, n, L, a.stride)]);
          ph = cscale(ph, a.tau2_scale);
          for (int s = 0; s < SV; ++s) {
            double2* p = &x[(size_t)s * tile_pts + e];
            *p = cmul(*p, ph);
          }
        }
        __syncthreads();
      }
      fft_lines_pq<L, true>(x, (const double2*)a.tw, wreg, nslots, tid, nthr);
    }
    __syncthreads();
    for (int s = 0; s < SV; ++s) {
      double2* dst = (double2*)a.psi + (size_t)(t.surf0 + s) * a.P;
#pragma unroll 1
      for (int e = tid; e < tile_pts; e += nthr) {
        int g, n;
        tile_elem<L>(e, t.tg, g, n);
        if (DSO_CHECK_INDEX((long long)(t.surf0 + s) * a.P + t.tg.addr(g, n, L, a.stride), a.psi_elems, 111, a.err))
          dst[t.tg.addr(g, n, L, a.stride)] = x[(size_t)s * tile_pts + g * L + n];
      }
    }
    cur = nxt;
    b ^= 1;
  }
  cp_async_wait<0>();
  // the last CTA out resets the queue for the next launch
  if (tid == 0) {
    __threadfence();
    const unsigned done = atomicAdd(&queue[1], 1u);
    if (done == gridDim.x - 1) {
      queue[0] = 0u;
      queue[1] = 0u;
      __threadfence();
    }
  }
}

}  // namespace dso
