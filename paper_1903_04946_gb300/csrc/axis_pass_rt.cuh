// axis_pass_rt.cuh -- the axis pass of axis_pass.cuh with the line length
// (and the number of staged surfaces) known only at run time.
//
// The batch kernel (batch.cu) advances many jobs with different grids in one
// launch: each of its CTAs runs tiles of whatever pass of whatever job comes
// next, so the tile body cannot be specialised on the line length at compile
// time.  The arithmetic is the same, operation for operation, as in
// axis_pass_kernel -- the same Stockham stages, the same tangent-form
// radix-8 butterflies and twiddle loads, the same matvec and phase products
// in the same order -- so a job gives bitwise the same result in a batch as
// alone with the same tile layout.
//
// Two differences from axis_pass_kernel follow from running many dependent
// passes in one launch: the wavefunction is read and written through L2
// (ld.global.cg / st.global.cg), because another SM may have written it
// earlier in the same launch and an SM's L1 is not coherent with the others;
// and every CTA has a fixed 256 threads, one 8-value slot each, so a tile
// holds at most 2048 amplitudes (SV * G * L <= 2048).
#pragma once

#include "axis_pass.cuh"

namespace dso {

constexpr int kRtThreads = 256;
constexpr int kRtMaxTile = 8 * kRtThreads;  // amplitudes of one tile (all staged surfaces)

__device__ __forceinline__ double2 ld_cg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ void st_cg(double2* p, double2 v) { __stcg(p, v); }
__device__ __forceinline__ void st_cg(float2* p, float2 v) { __stcg(p, v); }

__device__ __forceinline__ void tile_elem_rt(int e, const TileGeom& tg, int L, int log2L, int& g, int& n) {
  const int i = e & (tg.Wi - 1);
  n = (e >> tg.Wi_log2) & (L - 1);
  const int o = e >> (tg.Wi_log2 + log2L);
  g = (o << tg.Wi_log2) | i;
}

// One Stockham stage of radix R (stockham_stage with one slot per thread).
template <int R, bool INV, typename C>
__device__ __forceinline__ void stage_rt(C* sm, int L, int l8, int Ls, const C* __restrict__ tw, int nslots,
                                         int tid, unsigned wmask, bool wsync, const SmemLayout lay) {
  constexpr int NB = 8 / R;
  const int Q = L / R;
  C v[8];
  const bool act = tid < nslots;
  const int line = tid >> l8;
  const int u = tid & ((1 << l8) - 1);
  C* ln = sm + (size_t)line * lay.ls;
  if (act) {
#pragma unroll
    for (int beta = 0; beta < NB; ++beta) {
      const int j = u * NB + beta;
#pragma unroll
      for (int r = 0; r < R; ++r) v[beta * R + r] = ln[lay.pos(j + r * Q)];
    }
  }
  if (wsync) __syncwarp(wmask); else __syncthreads();
  if (act) {
#pragma unroll
    for (int beta = 0; beta < NB; ++beta) {
      const int j = u * NB + beta;
      const int k = j & (Ls - 1);
      C* x = &v[beta * R];
      if (R == 8 && Ls > 1) {
        const int step = (L / (Ls * 8)) * k;
        const C w1 = __ldg(&tw[step]);
        const C w2 = __ldg(&tw[2 * step]);
        const C w4 = __ldg(&tw[4 * step]);
        const C w8 = __ldg(&tw[step + L / 8]);
        dft8_tw<INV>(x, w1, w2, w4, w8);
      } else {
        dftR<R, INV>(x);
      }
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) ln[lay.pos(base + r * Ls)] = x[r];
    }
  }
  if (wsync) __syncwarp(wmask); else __syncthreads();
}

// The radix plan of Plan<L>: the leftover factor (2 or 4) first, then
// radix-8 stages.  `wsync`: a line lies in one warp (L <= 256), which is
// the same for every thread of the block.
template <bool INV, typename C>
__device__ __forceinline__ void fft_lines_rt(C* sm, const C* __restrict__ tw, int L, int log2L, int nslots, int tid,
                                             int nthr, const SmemLayout lay) {
  const unsigned wmask = warp_lanes_mask(tid, nthr);
  const bool wsync = L <= 256;
  const int rem = log2L % 3;
  const int l8 = log2L - 3;
  int Ls;
  if (rem == 0) {
    stage_rt<8, INV>(sm, L, l8, 1, tw, nslots, tid, wmask, wsync, lay);
    Ls = 8;
  } else if (rem == 1) {
    stage_rt<2, INV>(sm, L, l8, 1, tw, nslots, tid, wmask, wsync, lay);
    Ls = 2;
  } else {
    stage_rt<4, INV>(sm, L, l8, 1, tw, nslots, tid, wmask, wsync, lay);
    Ls = 4;
  }
  const int n8 = log2L / 3 - (rem == 0 ? 1 : 0);
#pragma unroll 1
  for (int st = 0; st < n8; ++st) {
    stage_rt<8, INV>(sm, L, l8, Ls, tw, nslots, tid, wmask, wsync, lay);
    Ls *= 8;
  }
}

template <int SV, typename C>
__device__ __forceinline__ void potential_rt(C* sm, const C* __restrict__ U, const TileGeom& tg, int G, int L,
                                             int log2L, long long stride, long long P, int tid, int nthr,
                                             const SmemLayout lay, int dec0) {
  constexpr int NP = SV * (SV + 1) / 2;
  const int tile_pts = G * L;
  const int tile_sz = G * lay.ls;
  for (int e = tid; e < tile_pts; e += nthr) {
    int g, n;
    tile_elem_rt(e, tg, L, log2L, g, n);
    const long long gi = tg.addr(g, n, L, stride);
    const int off = g * lay.ls + lay.pos(n);
    C x[SV], y[SV], u[NP];
#pragma unroll
    for (int s = 0; s < SV; ++s) x[s] = sm[(size_t)s * tile_sz + off];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (SV > 2 && dec0 && k >= 1 && k < SV) {  // U_0c = 0: not loaded
        u[k] = mkc((RealT<C>)0, (RealT<C>)0);
        continue;
      }
      u[k] = __ldg(&U[(size_t)k * P + gi]);
    }
    matvec_sym<SV>(u, x, y, dec0);
#pragma unroll
    for (int s = 0; s < SV; ++s) sm[(size_t)s * tile_sz + off] = y[s];
  }
  __syncthreads();
}

template <typename C>
__device__ __forceinline__ void potential_rt_sv(int SV, C* sm, const C* U, const TileGeom& tg, int G, int L,
                                                int log2L, long long stride, long long P, int tid, int nthr,
                                                const SmemLayout lay, int dec0) {
  switch (SV) {
    case 2: potential_rt<2>(sm, U, tg, G, L, log2L, stride, P, tid, nthr, lay, dec0); break;
    case 3: potential_rt<3>(sm, U, tg, G, L, log2L, stride, P, tid, nthr, lay, dec0); break;
    case 4: potential_rt<4>(sm, U, tg, G, L, log2L, stride, P, tid, nthr, lay, dec0); break;
    default: break;
  }
}

template <typename C>
__device__ __forceinline__ void kinetic_rt(C* sm, const C* __restrict__ tau, const TileGeom& tg, int G, int L,
                                           int log2L, int SVl, long long stride, int tid, int nthr, RealT<C> scale,
                                           const SmemLayout lay, bool axis_table) {
  const int tile_pts = G * L;
  const int tile_sz = G * lay.ls;
  if (axis_table) {  // the phase of this axis alone: element n of every line takes tau[n]
    for (int e = tid; e < tile_pts; e += nthr) {
      int g, n;
      tile_elem_rt(e, tg, L, log2L, g, n);
      C t = __ldg(&tau[n]);
      if (scale != (RealT<C>)1) t = cscale(t, scale);
      const int off = g * lay.ls + lay.pos(n);
      for (int s = 0; s < SVl; ++s) {
        C* p = &sm[(size_t)s * tile_sz + off];
        *p = cmul(*p, t);
      }
    }
    __syncthreads();
    return;
  }
  if (tg.stride_log2 == 0) {  // contiguous lines: the tile's phases are one block
    const C* blk = tau + (size_t)tg.o0 * L;
    for (int e = tid; e < tile_pts; e += nthr) {
      const int g = e >> log2L, n = e & (L - 1);
      C t = __ldg(&blk[e]);
      if (scale != (RealT<C>)1) t = cscale(t, scale);
      const int off = g * lay.ls + lay.pos(n);
      for (int s = 0; s < SVl; ++s) {
        C* p = &sm[s * tile_sz + off];
        *p = cmul(*p, t);
      }
    }
    __syncthreads();
    return;
  }
  for (int e = tid; e < tile_pts; e += nthr) {
    int g, n;
    tile_elem_rt(e, tg, L, log2L, g, n);
    C t = __ldg(&tau[tg.addr(g, n, L, stride)]);
    if (scale != (RealT<C>)1) t = cscale(t, scale);
    const int off = g * lay.ls + lay.pos(n);
    for (int s = 0; s < SVl; ++s) {
      C* p = &sm[(size_t)s * tile_sz + off];
      *p = cmul(*p, t);
    }
  }
  __syncthreads();
}

template <bool CONJ, typename C>
__device__ __forceinline__ void split_twiddles_rt(C* sm, const C* __restrict__ xtw, const TileGeom& tg, int G, int L,
                                                  int log2L, int SVl, int n2_log2, int s2_log2, int tid, int nthr,
                                                  const SmemLayout lay) {
  const int tile_pts = G * L;
  const int tile_sz = G * lay.ls;
  const long long n2_mask = (1LL << n2_log2) - 1;
  for (int e = tid; e < tile_pts; e += nthr) {
    int g, n;
    tile_elem_rt(e, tg, L, log2L, g, n);
    const long long i = tg.i0 + (g & (tg.Wi - 1));
    const long long i2 = (i >> s2_log2) & n2_mask;
    const C w = __ldg(&xtw[((long long)n << n2_log2) + i2]);
    const int off = g * lay.ls + lay.pos(n);
    for (int s = 0; s < SVl; ++s) {
      C* p = &sm[(size_t)s * tile_sz + off];
      *p = CONJ ? cmulc(*p, w) : cmul(*p, w);
    }
  }
  __syncthreads();
}

// One tile of pass `a` (lines of L points, SV staged surfaces), the work of
// one axis_pass_kernel CTA.  `tile` indexes the pass's tiles as blockIdx.x
// does there.  Needs SV * G * L <= kRtMaxTile and nthr == kRtThreads.
template <typename C>
__device__ __forceinline__ void tile_pass_rt(C* sm, const PassArgs& a, int L, int log2L, int SV, long long tile,
                                             int tid, int nthr) {
  C* psi = reinterpret_cast<C*>(a.psi);
  const C* tw = reinterpret_cast<const C*>(a.tw);
  const int G = a.G;
  const int tile_pts = G * L;
  const TileJob tj = split_tile(tile, SV, a);
  const int surf0 = tj.surf0;
  const size_t uoff = (size_t)tj.job * a.u_batch_stride;
  const TileGeom tg = make_geom(tj.tile, a);
  const SmemLayout lay = tile_layout(L, (int)sizeof(C), tg.Wi);
  const int tile_sz = G * lay.ls;
  const bool contig = a.stride_log2 == 0;
  const bool one_row = !contig && a.G_log2 <= a.stride_log2;
  const long long row = ((tg.o0 * L) << a.stride_log2) + tg.i0;
  for (int s = 0; s < SV; ++s) {
    const C* src = psi + (size_t)(surf0 + s) * a.P;
    if (contig) {
      const C* blk = src + (size_t)tg.o0 * L;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int g = e >> log2L, n = e & (L - 1);
        sm[s * tile_sz + g * lay.ls + lay.pos(n)] = ld_cg(&blk[e]);
      }
    } else if (one_row) {
      const C* blk = src + row;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int i = e & (G - 1), n = e >> a.G_log2;
        sm[s * tile_sz + i * lay.ls + lay.pos(n)] = ld_cg(&blk[((long long)n << a.stride_log2) + i]);
      }
    } else {
      for (int e = tid; e < tile_pts; e += nthr) {
        int g, n;
        tile_elem_rt(e, tg, L, log2L, g, n);
        sm[(size_t)s * tile_sz + g * lay.ls + lay.pos(n)] = ld_cg(&src[tg.addr(g, n, L, a.stride)]);
      }
    }
  }
  __syncthreads();
  const int nslots = SV * G * (L / 8);
  if (a.flags & PASS_INV_FIRST) {
    if (a.flags & PASS_XTW)
      split_twiddles_rt<true>(sm, reinterpret_cast<const C*>(a.xtw), tg, G, L, log2L, SV, a.xtw_n2_log2,
                              a.xtw_s2_log2, tid, nthr, lay);
    fft_lines_rt<true>(sm, tw, L, log2L, nslots, tid, nthr, lay);
    __syncthreads();
  }
  if (SV > 1) {
    if (a.U1)
      potential_rt_sv(SV, sm, reinterpret_cast<const C*>(a.U1) + uoff, tg, G, L, log2L, a.stride, a.P, tid, nthr,
                      lay, a.dec0);
    if (a.U2)
      potential_rt_sv(SV, sm, reinterpret_cast<const C*>(a.U2) + uoff, tg, G, L, log2L, a.stride, a.P, tid, nthr,
                      lay, a.dec0);
  }
  if (a.flags & PASS_FWD) {
    fft_lines_rt<false>(sm, tw, L, log2L, nslots, tid, nthr, lay);
    if (a.flags & PASS_XTW) {
      __syncthreads();
      split_twiddles_rt<false>(sm, reinterpret_cast<const C*>(a.xtw), tg, G, L, log2L, SV, a.xtw_n2_log2,
                               a.xtw_s2_log2, tid, nthr, lay);
    }
  }
  if (a.flags & PASS_T) {
    __syncthreads();
    const bool tax = (a.flags & PASS_TAX) != 0;
    kinetic_rt(sm, reinterpret_cast<const C*>(a.tau), tg, G, L, log2L, SV, a.stride, tid, nthr, (RealT<C>)1, lay,
               tax);
    if (a.tau2)
      kinetic_rt(sm, reinterpret_cast<const C*>(a.tau2), tg, G, L, log2L, SV, a.stride, tid, nthr,
                 (RealT<C>)a.tau2_scale, lay, tax);
    fft_lines_rt<true>(sm, tw, L, log2L, nslots, tid, nthr, lay);
  }
  __syncthreads();
  for (int s = 0; s < SV; ++s) {
    C* dst = psi + (size_t)(surf0 + s) * a.P;
    if (contig) {
      C* blk = dst + (size_t)tg.o0 * L;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int g = e >> log2L, n = e & (L - 1);
        st_cg(&blk[e], sm[s * tile_sz + g * lay.ls + lay.pos(n)]);
      }
    } else if (one_row) {
      C* blk = dst + row;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int i = e & (G - 1), n = e >> a.G_log2;
        st_cg(&blk[((long long)n << a.stride_log2) + i], sm[s * tile_sz + i * lay.ls + lay.pos(n)]);
      }
    } else {
      for (int e = tid; e < tile_pts; e += nthr) {
        int g, n;
        tile_elem_rt(e, tg, L, log2L, g, n);
        st_cg(&dst[tg.addr(g, n, L, a.stride)], sm[(size_t)s * tile_sz + g * lay.ls + lay.pos(n)]);
      }
    }
  }
}

}  // namespace dso
