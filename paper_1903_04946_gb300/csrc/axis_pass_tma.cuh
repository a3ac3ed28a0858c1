// axis_pass_tma.cuh -- axis pass with TMA tile movement (lines of L <= 256).
//
// Same arithmetic as axis_pass_kernel (axis_pass.cuh).  On this GPU the FP64
// unit is fed through the same L1TEX instruction queue as per-thread global
// loads and stores: with ncu, a pure DFMA loop stalls on "tex_throttle" at
// 99.8 % FP64 pipe use, and the per-thread-load version of this pass spends
// its stalls there with the FP64 pipe only 53-68 % busy.  This variant moves
// every global byte with the Tensor Memory Accelerator instead: one thread
// issues a bulk tensor copy per tile (wavefunction, potential or kinetic
// table) and one bulk copy of the twiddle table, all completing on an
// mbarrier, and the result goes back with one bulk tensor store.  The L1TEX
// queue then carries FP64 work only.
//
// The tile is the 5-D box {2, Wi, L, Go, SV} of the view
// (re/im, inner index i, line position n, outer index o, surface) of psi, so
// shared memory holds it as [s][o][n][i][re,im]: element n of line (s, g),
// g = o*Wi + i, sits at ((s*Go + o)*L + n)*Wi + i.  Tables use the same box
// with the component (or unique-coefficient) index as the last coordinate,
// so one flat index e = (o*L + n)*Wi + i addresses the same grid point in the
// wavefunction block of every surface and in every table component.
#pragma once

#include <cuda.h>

#include "axis_pass.cuh"

namespace dso {

struct TmaMaps {
  CUtensorMap psi;   // box {2, Wi, L, Go, SV}
  CUtensorMap tab;   // potential unitaries (box {2, Wi, L, Go, NP}) or kinetic phases (box {.., 1})
  CUtensorMap tab2;  // kinetic phases when the pass also applies the potential (1-D grids)
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bounded wait on phase `parity`: false if it did not complete within
// `limit` polls.  The waits for tile copies use kWaitPolls; the drain of
// copies still in flight after an error always uses kWaitPolls too, so that
// no CTA leaves while a copy into its shared memory can still land.
constexpr int kWaitPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit = kWaitPolls) {
  const unsigned a = smem_u32(bar);
  for (int it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                             const void* src) {
  asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(map),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One Stockham stage on lines stored with element stride Wi (TMA layout).
template <int L, int R, bool INV>
__device__ __forceinline__ void tma_stage(double2* sm, int Ls, const double2* __restrict__ tws, int G, int Go_unused,
                                          int Wi_log2, int nslots, int tid, unsigned wmask) {
  constexpr int NB = 8 / R;
  constexpr int Q = L / R;
  const int Wi = 1 << Wi_log2;
  double2 v[8];
  const bool act = tid < nslots;
  const int line = tid / (L / 8);
  const int u = tid % (L / 8);
  // line -> (surface s, tile line g = o*Wi + i): base of element 0, stride Wi
  const int s = line / G;
  const int g = line - s * G;
  const int o = g >> Wi_log2, i = g & (Wi - 1);
  double2* ln = sm + ((size_t)(s * (G >> Wi_log2) + o) * L) * Wi + i;
  if (act) {
#pragma unroll
    for (int beta = 0; beta < NB; ++beta) {
      const int j = u * NB + beta;
#pragma unroll
      for (int r = 0; r < R; ++r) v[beta * R + r] = ln[(j + r * Q) << Wi_log2];
    }
  }
  stage_sync<L>(wmask);
  if (act) {
#pragma unroll
    for (int beta = 0; beta < NB; ++beta) {
      const int j = u * NB + beta;
      const int k = j & (Ls - 1);
      double2* x = &v[beta * R];
      if (R == 8 && Ls > 1) {
        double2 w1, w2, w4, w8;
        load_tw8<L, true>(tws, (L / (Ls * 8)) * k, w1, w2, w4, w8);
        dft8_tw<INV>(x, w1, w2, w4, w8);
      } else {
        dftR<R, INV>(x);
      }
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) ln[(base + r * Ls) << Wi_log2] = x[r];
    }
  }
  stage_sync<L>(wmask);
}

template <int L, bool INV>
__device__ __forceinline__ void tma_fft(double2* sm, const double2* tws, int G, int Wi_log2, int nslots, int tid,
                                        int nthr) {
  using PL = Plan<L>;
  const unsigned wmask = warp_lanes_mask(tid, nthr);
  tma_stage<L, PL::first, INV>(sm, 1, tws, G, 0, Wi_log2, nslots, tid, wmask);
  int Ls = PL::first;
#pragma unroll 1
  for (int st = 0; st < PL::n8; ++st) {
    tma_stage<L, 8, INV>(sm, Ls, tws, G, 0, Wi_log2, nslots, tid, wmask);
    Ls *= 8;
  }
}

template <int SV>
__device__ __forceinline__ void tma_potential(double2* x, const double2* ub, int tile_pts, int tid, int nthr,
                                              int dec0) {
  constexpr int NP = SV * (SV + 1) / 2;
  for (int e = tid; e < tile_pts; e += nthr) {
    double2 xs[SV], y[SV], u[NP];
#pragma unroll
    for (int s = 0; s < SV; ++s) xs[s] = x[(size_t)s * tile_pts + e];
#pragma unroll
    for (int k = 0; k < NP; ++k)
      u[k] = (SV > 2 && dec0 && k >= 1 && k < SV) ? make_double2(0.0, 0.0) : ub[(size_t)k * tile_pts + e];
    matvec_sym<SV>(u, xs, y, dec0);
#pragma unroll
    for (int s = 0; s < SV; ++s) x[(size_t)s * tile_pts + e] = y[s];
  }
}

// The second potential unitary of a step boundary (one launch in N_B) is
// read straight from global memory.
template <int L, int SV>
__device__ __forceinline__ void tma_potential_global(double2* x, const double2* __restrict__ U, const PassArgs& a,
                                                     long long o0, long long i0, int Wi_log2, int tile_pts, int tid,
                                                     int nthr, int dec0 = 0) {
  constexpr int NP = SV * (SV + 1) / 2;
  const int Wi = 1 << Wi_log2;
  for (int e = tid; e < tile_pts; e += nthr) {
    const int i = e & (Wi - 1);
    const int n = (e >> Wi_log2) & (L - 1);
    const int o = e >> (Wi_log2 + Plan<L>::log2L);
    const long long gi = (((o0 + o) * L + n) << a.stride_log2) + i0 + i;
    double2 xs[SV], y[SV], u[NP];
#pragma unroll
    for (int s = 0; s < SV; ++s) xs[s] = x[(size_t)s * tile_pts + e];
#pragma unroll
    for (int k = 0; k < NP; ++k)
      u[k] = (SV > 2 && dec0 && k >= 1 && k < SV) ? make_double2(0.0, 0.0) : __ldg(&U[(size_t)k * a.P + gi]);
    matvec_sym<SV>(u, xs, y, dec0);
#pragma unroll
    for (int s = 0; s < SV; ++s) x[(size_t)s * tile_pts + e] = y[s];
  }
}

// Extra PassArgs fields used here: ua/ub = unique-coefficient indices of the
// potential and kinetic tables (coordinates in the table maps), err = error
// flag set when a bounded wait gives up.
// Shared memory: [psi tile SV*G*L][table NP*G*L (or G*L)][twiddles L], all
// 128-byte aligned, plus one mbarrier per phase.
template <int L, int SV>
__host__ __device__ constexpr int tma_np_tab() {
  return SV > 1 ? SV * (SV + 1) / 2 : 1;
}

// Dynamic shared memory needed by axis_pass_tma_kernel (128 bytes of slack
// for aligning the base, 64 for the four barriers and the status word).
template <int L, int SV>
inline size_t tma_smem_bytes(int G) {
  return (size_t)(SV + tma_np_tab<L, SV>()) * G * L * 16 + (size_t)L * 16 + 128 + 64;
}

// All waits go through thread 0 with a bounded spin; the outcome is shared
// through shared memory so that every thread leaves (or continues) together.
__device__ __forceinline__ bool cta_wait(unsigned long long* bar, unsigned parity, volatile int* status, int tid) {
  if (tid == 0) *status = mbar_wait(bar, parity) ? 1 : 0;
  __syncthreads();
  const bool ok = *status != 0;
  if (ok && tid != 0) mbar_wait(bar, parity);  // completes at once; acquires the copied data for this thread
  return ok;
}

template <int L, int SV>
__global__ void __launch_bounds__(256) axis_pass_tma_kernel(PassArgs a, const __grid_constant__ TmaMaps maps) {
  extern __shared__ double2 sm_raw[];
  double2* sm = (double2*)(((uintptr_t)sm_raw + 127) & ~(uintptr_t)127);
  constexpr int NP = SV * (SV + 1) / 2;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = a.G;
  const int tile_pts = G * L;
  const int nslots = SV * G * (L / 8);
  const int np_tab = SV > 1 ? NP : 1;
  double2* x = sm;
  double2* tb = sm + (size_t)SV * tile_pts;
  double2* tws = tb + (size_t)np_tab * tile_pts;
  unsigned long long* bar = (unsigned long long*)(tws + L);  // [0..2] copies, [3] wait diagnostics
  volatile int* status = (volatile int*)(bar + 4);

  // tile geometry (the same as axis_pass_kernel)
  const TileJob tj = split_tile(blockIdx.x, SV, a);
  const int surf0 = tj.surf0;
  const TileGeom tg = make_geom(tj.tile, a);
  const int Wi_log2 = tg.Wi_log2;
  const int c1 = (int)tg.i0, c3 = (int)tg.o0;
  const bool vstep = (SV > 1) && (a.U1 != nullptr);
  const bool tstep = (a.flags & PASS_T) != 0;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();  // psi is the previous pass's output
  if (tid == 0) {
    // phase 0: tile and twiddles; phase 1: table for the first table step;
    // phase 2: kinetic table of a 1-D pass that also applies the potential
    mbar_expect_tx(&bar[0], (unsigned)((SV * tile_pts + L) * sizeof(double2)));
    tma_load_5d(x, &maps.psi, 0, c1, 0, c3, surf0, &bar[0]);
    bulk_load(tws, a.tw, (unsigned)(L * sizeof(double2)), &bar[0]);
    if (vstep) {
      mbar_expect_tx(&bar[1], (unsigned)(NP * tile_pts * sizeof(double2)));
      // potential tables are [job][unique a][component]: one coordinate
      tma_load_5d(tb, &maps.tab, 0, c1, 0, c3, (int)((long long)tj.job * a.u_batch_stride / a.P) + a.ua * NP,
                  &bar[1]);
    } else if (tstep) {
      mbar_expect_tx(&bar[1], (unsigned)(tile_pts * sizeof(double2)));
      tma_load_5d(tb, &maps.tab, 0, c1, 0, c3, a.ub, &bar[1]);
    }
  }
  // copies in flight, tracked by thread 0: bit b for bar[b]
  unsigned pending = (tid == 0) ? (1u | ((vstep || tstep) ? 2u : 0u)) : 0u;
  // a wait gave up: record it and let every copy this CTA started land
  // before the CTA leaves (each drain wait again bounded)
  auto give_up = [&](int code) {
    if (tid == 0) {
      atomicExch(a.err, code);
      if (pending & 1u) mbar_wait(&bar[0], 0);
      if (pending & 2u) mbar_wait(&bar[1], 0);
      if (pending & 4u) mbar_wait(&bar[2], 0);
    }
  };
  if (!cta_wait(&bar[0], 0, status, tid)) {
    give_up(1);
    return;
  }
  pending &= ~1u;
  if (a.wait_probe > 0) {
    // diagnostics of the bounded waits: a barrier that no copy completes;
    // the wait must give up after a.wait_probe polls and record a timeout
    // (code 5).  No copy is involved, and the tile's work goes on unchanged.
    if (tid == 0) {
      mbar_init(&bar[3], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      if (!mbar_wait(&bar[3], 0, a.wait_probe)) atomicExch(a.err, 5);
    }
    __syncthreads();
  }
  pdl_trigger();

  if (a.flags & PASS_INV_FIRST) {
    tma_fft<L, true>(x, tws, G, Wi_log2, nslots, tid, nthr);
    __syncthreads();
  }
  if (vstep) {
    if (!cta_wait(&bar[1], 0, status, tid)) {
      give_up(2);
      return;
    }
    pending &= ~2u;
    tma_potential<SV>(x, tb, tile_pts, tid, nthr, a.dec0);
    __syncthreads();
    if (a.U2) {
      tma_potential_global<L, SV>(x, (const double2*)a.U2 + (size_t)tj.job * a.u_batch_stride, a, tg.o0, tg.i0,
                                  Wi_log2, tile_pts, tid, nthr, a.dec0);
      __syncthreads();
    }
    if (tstep && tid == 0) {  // 1-D grids: kinetic phases into the freed table buffer
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[2], (unsigned)(tile_pts * sizeof(double2)));
      tma_load_5d(tb, &maps.tab2, 0, c1, 0, c3, a.ub, &bar[2]);
      pending |= 4u;
    }
  }
  if (a.flags & PASS_FWD) tma_fft<L, false>(x, tws, G, Wi_log2, nslots, tid, nthr);
  if (tstep) {
    __syncthreads();
    if (!cta_wait(&bar[vstep ? 2 : 1], 0, status, tid)) {
      give_up(3);
      return;
    }
    pending = 0u;
    for (int e = tid; e < tile_pts; e += nthr) {
      const double2 ph = tb[e];
#pragma unroll
      for (int s = 0; s < SV; ++s) {
        double2* p = &x[(size_t)s * tile_pts + e];
        *p = cmul(*p, ph);
      }
    }
    __syncthreads();
    if (a.tau2) {  // second kinetic phase of a step boundary, from global memory
      const int Wi = 1 << Wi_log2;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int i = e & (Wi - 1);
        const int n = (e >> Wi_log2) & (L - 1);
        const int o = e >> (Wi_log2 + Plan<L>::log2L);
        const long long gi = (((tg.o0 + o) * L + n) << a.stride_log2) + tg.i0 + i;
        double2 ph = __ldg(&((const double2*)a.tau2)[gi]);
        ph = cscale(ph, a.tau2_scale);
#pragma unroll
        for (int s = 0; s < SV; ++s) {
          double2* p = &x[(size_t)s * tile_pts + e];
          *p = cmul(*p, ph);
        }
      }
      __syncthreads();
    }
    tma_fft<L, true>(x, tws, G, Wi_log2, nslots, tid, nthr);
  }
  // make the generic-proxy writes visible to the bulk store, then store
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    tma_store_5d(&maps.psi, 0, c1, 0, c3, surf0, x);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}


// ---------------------------------------------------------------------------
// Persistent form (variant 3).  The one-tile-per-CTA kernel above runs the
// whole grid in about one wave on the wavefunction sizes of interest, so all
// CTAs load at the same time, then all compute, then all store: the FP64
// pipe idles during the first and last phase.  Here a grid of a few CTAs per
// SM takes tiles from the per-launch queue (the two counters the persistent
// cp.async variant uses, left zeroed by the last CTA out), and every CTA
// double-buffers: while tile t is transformed in one stage buffer, the TMA
// engine fills the other with tile t+1 (wavefunction and table), and tile t
// leaves with a bulk tensor store that the next prefetch into that buffer
// waits for.  The arithmetic is that of axis_pass_tma_kernel, in the same
// order, so both variants give identical results.
//
// Passes that apply both a potential and a kinetic phase (1-D grids) are
// not handled here; the host does not select this variant for them.
//
// Shared memory: two stages of [psi SV*G*L][table np*G*L] (np = 0 when the
// pass has no table step), the twiddles, three mbarriers and a status word.
template <int L, int SV>
inline size_t tmap_smem_bytes(int G, bool has_tab) {
  const int np = has_tab ? tma_np_tab<L, SV>() : 0;
  return 2 * (size_t)(SV + np) * G * L * 16 + (size_t)L * 16 + 128 + 64;
}

template <int L, int SV>
__global__ void __launch_bounds__(256) axis_pass_tmap_kernel(PassArgs a, const __grid_constant__ TmaMaps maps,
                                                             unsigned* __restrict__ queue) {
  extern __shared__ double2 sm_raw[];
  double2* sm = (double2*)(((uintptr_t)sm_raw + 127) & ~(uintptr_t)127);
  __shared__ long long s_tile[2];
  __shared__ volatile int s_zero;
  constexpr int NP = SV * (SV + 1) / 2;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = a.G;
  const int tile_pts = G * L;
  const int nslots = SV * G * (L / 8);
  const bool vstep = (SV > 1) && (a.U1 != nullptr);
  const bool tstep = (a.flags & PASS_T) != 0;
  const bool has_tab = vstep || tstep;
  const int np_tab = has_tab ? (vstep ? NP : 1) : 0;
  const int stage_elems = (SV + (has_tab ? tma_np_tab<L, SV>() : 0)) * tile_pts;
  double2* stage0 = sm;
  double2* tws = sm + 2 * (size_t)stage_elems;
  unsigned long long* bar = (unsigned long long*)(tws + L);  // [0], [1]: stages; [2]: twiddles
  volatile int* status = (volatile int*)(bar + 3);
  const long long ntiles = (SV == a.S) ? (long long)a.nbatch * (a.lines >> a.G_log2)
                                       : (long long)a.nbatch * a.S * (a.lines >> a.G_log2);
  const unsigned tab_bytes = (unsigned)(np_tab * tile_pts * sizeof(double2));
  const unsigned psi_bytes = (unsigned)(SV * tile_pts * sizeof(double2));

  // thread 0: start the copies of tile `tile` into stage buffer `st`
  auto issue = [&](long long tile, double2* st, unsigned long long* b) {
    const TileJob tj = split_tile(tile, SV, a);
    const TileGeom tg = make_geom(tj.tile, a);
    mbar_expect_tx(b, psi_bytes + tab_bytes);
    tma_load_5d(st, &maps.psi, 0, (int)tg.i0, 0, (int)tg.o0, tj.surf0, b);
    if (vstep) {
      tma_load_5d(st + (size_t)SV * tile_pts, &maps.tab, 0, (int)tg.i0, 0, (int)tg.o0,
                  (int)((long long)tj.job * a.u_batch_stride / a.P) + a.ua * NP, b);
    } else if (tstep) {
      tma_load_5d(st + (size_t)SV * tile_pts, &maps.tab, 0, (int)tg.i0, 0, (int)tg.o0, a.ub, b);
    }
  };

  if (tid == 0) {
    s_zero = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();  // psi and the queue reset are the previous pass's
  pdl_trigger();
  if (tid == 0) {
    mbar_expect_tx(&bar[2], (unsigned)(L * sizeof(double2)));
    bulk_load(tws, a.tw, (unsigned)(L * sizeof(double2)), &bar[2]);
    const long long t0 = (long long)atomicAdd(&queue[0], 1u);
    s_tile[0] = t0;
    if (t0 < ntiles) issue(t0, stage0, &bar[0]);
  }
  // pending bit b (b < 2): a copy into stage b is in flight; bit 2: twiddles
  unsigned pending = (tid == 0 && s_tile[0] < ntiles) ? 5u : 4u;
  bool ok = cta_wait(&bar[2], 0, status, tid);
  if (ok) pending &= ~4u;
  long long cur = s_tile[0];
  int s = 0;
  unsigned phase = 0;  // bit b: parity of the next completion of stage b
  while (ok && cur < ntiles) {
    double2* x = stage0 + (size_t)s * stage_elems;
    double2* tb = x + (size_t)SV * tile_pts;
    if (tid == 0) {  // prefetch the next tile into the other stage
      const long long nxt = (long long)atomicAdd(&queue[0], 1u);
      s_tile[s ^ 1] = nxt;
      if (nxt < ntiles) {
        // the other stage's last store must have read its buffer
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        issue(nxt, stage0 + (size_t)(s ^ 1) * stage_elems, &bar[s ^ 1]);
        pending |= 1u << (s ^ 1);
      }
    }
    if (!cta_wait(&bar[s], (phase >> s) & 1u, status, tid)) {
      ok = false;
      break;
    }
    pending &= ~(1u << s);
    phase ^= 1u << s;
    const TileJob tj = split_tile(cur, SV, a);
    const TileGeom tg = make_geom(tj.tile, a);
    // Every shared-memory address of the tile work below depends only on the
    // thread index and launch constants.  Left visible, the compiler keeps
    // the addresses of one FFT call live for the next ones and across tiles,
    // and spills.  Each FFT call therefore gets its arguments offset by a
    // zero read from shared memory, which no compiler stage can fold.
#define DSO_TMAP_FFT(INV)                                                                               \
  do {                                                                                                  \
    const int z = s_zero;                                                                               \
    tma_fft<L, INV>(x + z, tws + z, G + z, tg.Wi_log2 + z, nslots + z, tid + z, nthr + z);              \
  } while (0)
    const int Wi_log2 = tg.Wi_log2;

    if (a.flags & PASS_INV_FIRST) {
      DSO_TMAP_FFT(true);
      __syncthreads();
    }
    if (vstep) {
      tma_potential<SV>(x, tb, tile_pts, tid, nthr, a.dec0);
      __syncthreads();
      if (a.U2) {
        tma_potential_global<L, SV>(x, (const double2*)a.U2 + (size_t)tj.job * a.u_batch_stride, a, tg.o0, tg.i0,
                                    Wi_log2, tile_pts, tid, nthr, a.dec0);
        __syncthreads();
      }
    }
    if (a.flags & PASS_FWD) DSO_TMAP_FFT(false);
    if (tstep) {
      __syncthreads();
      for (int e = tid; e < tile_pts; e += nthr) {
        const double2 ph = tb[e];
#pragma unroll
        for (int q = 0; q < SV; ++q) {
          double2* p = &x[(size_t)q * tile_pts + e];
          *p = cmul(*p, ph);
        }
      }
      __syncthreads();
      if (a.tau2) {  // second kinetic phase of a step boundary, from global memory
        const int Wi = 1 << Wi_log2;
        for (int e = tid; e < tile_pts; e += nthr) {
          const int i = e & (Wi - 1);
          const int n = (e >> Wi_log2) & (L - 1);
          const int o = e >> (Wi_log2 + Plan<L>::log2L);
          const long long gi = (((tg.o0 + o) * L + n) << a.stride_log2) + tg.i0 + i;
          double2 ph = __ldg(&((const double2*)a.tau2)[gi]);
          ph = cscale(ph, a.tau2_scale);
#pragma unroll
          for (int q = 0; q < SV; ++q) {
            double2* p = &x[(size_t)q * tile_pts + e];
            *p = cmul(*p, ph);
          }
        }
        __syncthreads();
      }
      DSO_TMAP_FFT(true);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tma_store_5d(&maps.psi, 0, (int)tg.i0, 0, (int)tg.o0, tj.surf0, x);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    cur = s_tile[s ^ 1];
    s ^= 1;
  }
#undef DSO_TMAP_FFT
  if (tid == 0) {
    if (!ok) {
      // a bounded wait gave up: record it and let every copy this CTA
      // started land before the CTA leaves (each wait again bounded)
      atomicExch(a.err, 4);
      if (pending & 1u) mbar_wait(&bar[0], phase & 1u);
      if (pending & 2u) mbar_wait(&bar[1], (phase >> 1) & 1u);
      if (pending & 4u) mbar_wait(&bar[2], 0);
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    // the last CTA out resets the queue for the next launch
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
