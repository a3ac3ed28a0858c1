// axis_pass.cuh -- fused FFT / potential / kinetic pass along one grid axis.
//
// One CTA owns a tile of whole lines along axis `a` (length L) of the grid:
// G neighbouring line positions, and for a potential pass all SV = S surfaces
// of those positions.  The tile is staged in shared memory; each FFT stage
// moves 8 complex values per thread into registers, applies the twiddles and
// a radix-8 (or radix-4/2 for the leftover factor) butterfly, and writes the
// results back in Stockham autosort order, so every transform ends in natural
// order without a bit-reversal pass.
//
// Per pass, in this order (each step optional, chosen by `flags`):
//   1. inverse FFT along the axis                              (Sec. II G)
//   2. psi(q) <- U_V(a dt) psi(q): S x S complex matvec at every grid point
//      with a precomputed unitary, then optionally a second one (the last V
//      of a time step merged into the first V of the next)     (Sec. II H)
//   3. forward FFT along the axis
//   4. psi~(p) <- tau_b(p) psi~(p) with the kinetic phase (the 1/P of the
//      inverse transforms folded in), then the inverse FFT      (Sec. II G)
// Steps 2 need the wavepacket in the position representation on all axes,
// step 4 in the momentum representation on all axes; the host orders the
// passes so that this holds.
//
// The FP64 path on this GPU is bound by the FP64 pipe (one DFMA per SM
// sub-partition every 64 cycles for a full warp), so the butterflies are
// written to minimise FP64 instructions: trivial twiddles (+-1, +-i) cost
// nothing, the (1 -+ i)/sqrt(2) factors of the radix-8 butterfly fold into
// FMAs, and everything else (indexing, shared-memory traffic, table loads)
// runs on other pipes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pass_args.h"

namespace dso {

// FP64 arithmetic of the hot path.  On this GPU the FP64 pipe issues DFMA
// about 1.19x faster than DADD or DMUL (measured: 0.599 vs 0.504 T inst/s),
// so every add, subtract and multiply is issued as an FMA: a + b = fma(a, 1, b)
// and a * b = fma(a, b, -0), both exactly rounded like the plain operation.
// The 1.0 and -0.0 come from the kernel arguments: with literal constants the
// compiler folds the FMA back into DADD/DMUL.
struct DPK {
  double one;  // 1.0 at run time
  double mz;   // -0.0 at run time
};
__device__ __forceinline__ double dadd(double a, double b, const DPK& k) { return fma(a, k.one, b); }
__device__ __forceinline__ double dsub(double a, double b, const DPK& k) { return fma(-b, k.one, a); }
__device__ __forceinline__ double dmul(double a, double b, const DPK& k) { return fma(a, b, k.mz); }

__device__ __forceinline__ double2 cmul(double2 a, double2 b, const DPK& k) {
  return make_double2(fma(a.x, b.x, dmul(-a.y, b.y, k)), fma(a.x, b.y, dmul(a.y, b.x, k)));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b, const DPK& k) {
  return make_double2(fma(a.x, b.x, dmul(a.y, b.y, k)), fma(a.y, b.x, dmul(-a.x, b.y, k)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b, const DPK& k) {
  return make_double2(dadd(a.x, b.x, k), dadd(a.y, b.y, k));
}
__device__ __forceinline__ double2 csub(double2 a, double2 b, const DPK& k) {
  return make_double2(dsub(a.x, b.x, k), dsub(a.y, b.y, k));
}
// multiply by -i (forward) or +i (inverse): free, no FP64 instruction
template <bool INV>
__device__ __forceinline__ double2 rot_i(double2 a) {
  return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// In-place DFT of length 2, 4, 8 with sign -1 (forward) or +1 (INV).
template <bool INV>
__device__ __forceinline__ void dft2(double2& a, double2& b, const DPK& k) {
  double2 t = a;
  a = cadd(t, b, k);
  b = csub(t, b, k);
}

template <bool INV>
__device__ __forceinline__ void dft4(double2& a0, double2& a1, double2& a2, double2& a3, const DPK& k) {
  double2 t0 = cadd(a0, a2, k), t1 = csub(a0, a2, k);
  double2 t2 = cadd(a1, a3, k), t3 = rot_i<INV>(csub(a1, a3, k));
  a0 = cadd(t0, t2, k);
  a2 = csub(t0, t2, k);
  a1 = cadd(t1, t3, k);
  a3 = csub(t1, t3, k);
}

// 8-point DFT by one radix-2 split into two 4-point DFTs:
// y_k = E_k + w^k O_k, y_{k+4} = E_k - w^k O_k, w = exp(-+2 pi i / 8).
template <bool INV>
__device__ __forceinline__ void dft8(double2* x, const DPK& k) {
  const double c = 0.70710678118654752440;  // 1/sqrt(2)
  double2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  double2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3, k);
  dft4<INV>(o0, o1, o2, o3, k);
  // k = 0
  x[0] = cadd(e0, o0, k);
  x[4] = csub(e0, o0, k);
  // k = 2: w^2 = -+i
  double2 r2 = rot_i<INV>(o2);
  x[2] = cadd(e2, r2, k);
  x[6] = csub(e2, r2, k);
  // k = 1: w = (1 -+ i)/sqrt(2); w*o = c * u
  double2 u1 = INV ? make_double2(dsub(o1.x, o1.y, k), dadd(o1.x, o1.y, k))
                   : make_double2(dadd(o1.x, o1.y, k), dsub(o1.y, o1.x, k));
  x[1] = make_double2(fma(c, u1.x, e1.x), fma(c, u1.y, e1.y));
  x[5] = make_double2(fma(-c, u1.x, e1.x), fma(-c, u1.y, e1.y));
  // k = 3: w^3 = (-1 -+ i)/sqrt(2)
  double2 u3 = INV ? make_double2(-dadd(o3.x, o3.y, k), dsub(o3.x, o3.y, k))
                   : make_double2(dsub(o3.y, o3.x, k), -dadd(o3.x, o3.y, k));
  x[3] = make_double2(fma(c, u3.x, e3.x), fma(c, u3.y, e3.y));
  x[7] = make_double2(fma(-c, u3.x, e3.x), fma(-c, u3.y, e3.y));
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(double2* x, const DPK& k) {
  if constexpr (R == 8) {
    dft8<INV>(x, k);
  } else if constexpr (R == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3], k);
  } else {
    dft2<INV>(x[0], x[1], k);
  }
}

// Radix plan of a length-L transform: as many radix-8 stages as possible,
// the leftover factor (2 or 4) as the first stage, whose twiddles are all 1.
template <int L>
struct Plan {
  static constexpr int log2L = (L >= 4096) ? 12 : (L >= 2048) ? 11 : (L >= 1024) ? 10 : (L >= 512) ? 9
                             : (L >= 256) ? 8 : (L >= 128) ? 7 : (L >= 64) ? 6 : (L >= 32) ? 5 : (L >= 16) ? 4 : 3;
  static constexpr int rem = log2L % 3;           // 0, 1 or 2 leftover binary stages
  static constexpr int first = rem == 0 ? 8 : (rem == 1 ? 2 : 4);
  static constexpr int n8 = log2L / 3 - (rem == 0 ? 1 : 0);  // radix-8 stages after the first
};

// Between FFT stages only the threads of one line exchange data.  A line of
// length L is handled by L/8 consecutive threads, so for L <= 256 it lies in
// one warp and a warp barrier suffices; longer lines span warps.
// `wmask` holds the lanes of this thread's warp that exist in the block.
template <int L>
__device__ __forceinline__ void stage_sync(unsigned wmask) {
  if constexpr (L <= 256) {
    __syncwarp(wmask);
  } else {
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned warp_lanes_mask(int tid, int nthr) {
  const int left = nthr - (tid & ~31);
  return left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
}

// One Stockham stage of radix R on every line of the tile held in `sm`.
// Thread-slot s of this thread owns 8 consecutive butterfly inputs' worth of
// work: 8/R butterflies j = u*(8/R) + beta of line `line`.
template <int L, int R, bool INV, int K>
__device__ __forceinline__ void stockham_stage(double2* sm, int Ls, const double2* __restrict__ tw,
                                               int nslots, int tid, int nthr, unsigned wmask, const DPK& dk) {
  constexpr int NB = 8 / R;      // butterflies per slot
  constexpr int Q = L / R;       // butterflies per line
  double2 v[K][8];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int gid = s * nthr + tid;
    if (gid < nslots) {
      const int line = gid / (L / 8);
      const int u = gid % (L / 8);
      const double2* ln = sm + (size_t)line * L;
#pragma unroll
      for (int beta = 0; beta < NB; ++beta) {
        const int j = u * NB + beta;
#pragma unroll
        for (int r = 0; r < R; ++r) v[s][beta * R + r] = ln[j + r * Q];
      }
    }
  }
  stage_sync<L>(wmask);
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int gid = s * nthr + tid;
    if (gid < nslots) {
      const int line = gid / (L / 8);
      const int u = gid % (L / 8);
      double2* ln = sm + (size_t)line * L;
#pragma unroll
      for (int beta = 0; beta < NB; ++beta) {
        const int j = u * NB + beta;
        const int k = j & (Ls - 1);
        double2* x = &v[s][beta * R];
        if (Ls > 1) {
          const int step = (L / (Ls * R)) * k;
#pragma unroll
          for (int r = 1; r < R; ++r) {
            const double2 w = __ldg(&tw[r * step]);
            x[r] = INV ? cmulc(x[r], w, dk) : cmul(x[r], w, dk);
          }
        }
        dftR<R, INV>(x, dk);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) ln[base + r * Ls] = x[r];
      }
    }
  }
  stage_sync<L>(wmask);
}

template <int L, bool INV, int K>
__device__ __forceinline__ void fft_lines(double2* sm, const double2* __restrict__ tw, int nslots, int tid, int nthr,
                                          const DPK& dk) {
  using PL = Plan<L>;
  const unsigned wmask = warp_lanes_mask(tid, nthr);
  stockham_stage<L, PL::first, INV, K>(sm, 1, tw, nslots, tid, nthr, wmask, dk);
  int Ls = PL::first;
#pragma unroll 1
  for (int st = 0; st < PL::n8; ++st) {
    stockham_stage<L, 8, INV, K>(sm, Ls, tw, nslots, tid, nthr, wmask, dk);
    Ls *= 8;
  }
}

// Global address (within one surface) of element n of tile line g.  Axis
// lengths, strides and tile line counts are powers of two, so all index
// arithmetic is shifts and masks.
struct TileGeom {
  long long o0;      // first outer index of the tile
  long long i0;      // first inner index of the tile
  int Wi;            // inner positions per outer row in the tile
  int Wi_log2;
  int stride_log2;
  __device__ __forceinline__ long long addr(int g, int n, long long L, long long /*stride*/) const {
    const long long o = o0 + (g >> Wi_log2);
    const long long i = i0 + (g & (Wi - 1));
    return ((o * L + n) << stride_log2) + i;
  }
};

__device__ __forceinline__ TileGeom make_geom(long long tile, const PassArgs& a) {
  TileGeom tg;
  const long long lam0 = tile << a.G_log2;
  tg.Wi_log2 = a.stride_log2 < a.G_log2 ? a.stride_log2 : a.G_log2;
  tg.Wi = 1 << tg.Wi_log2;
  tg.stride_log2 = a.stride_log2;
  tg.o0 = lam0 >> a.stride_log2;
  tg.i0 = lam0 & ((1LL << a.stride_log2) - 1);
  return tg;
}

// Element e of the tile in address order -> (g, n); consecutive e are
// consecutive addresses whenever the axis stride allows it.
template <int L>
__device__ __forceinline__ void tile_elem(int e, const TileGeom& tg, int& g, int& n) {
  const int i = e & (tg.Wi - 1);
  n = (e >> tg.Wi_log2) & (L - 1);
  const int o = e >> (tg.Wi_log2 + Plan<L>::log2L);
  g = (o << tg.Wi_log2) | i;
}

template <int L, int SV>
__device__ __forceinline__ void apply_potential(double2* sm, const double2* __restrict__ U, const TileGeom& tg,
                                                int G, long long stride, long long P, int tid, int nthr,
                                                const DPK& dk) {
  constexpr int NP = SV * (SV + 1) / 2;
  const int tile_pts = G * L;
  for (int e = tid; e < tile_pts; e += nthr) {
    int g, n;
    tile_elem<L>(e, tg, g, n);
    const long long gi = tg.addr(g, n, L, stride);
    const int off = g * L + n;
    double2 x[SV], y[SV];
#pragma unroll
    for (int s = 0; s < SV; ++s) x[s] = sm[(size_t)s * tile_pts + off];
    double2 u[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) u[k] = __ldg(&U[(size_t)k * P + gi]);
#pragma unroll
    for (int r = 0; r < SV; ++r) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < SV; ++c) {
        const int lo = r < c ? r : c, hi = r < c ? c : r;
        const int k = lo * SV - lo * (lo - 1) / 2 + (hi - lo);
        if (c == 0) {
          acc = cmul(u[k], x[c], dk);
        } else {
          acc.x = fma(u[k].x, x[c].x, acc.x);
          acc.x = fma(-u[k].y, x[c].y, acc.x);
          acc.y = fma(u[k].x, x[c].y, acc.y);
          acc.y = fma(u[k].y, x[c].x, acc.y);
        }
      }
      y[r] = acc;
    }
#pragma unroll
    for (int s = 0; s < SV; ++s) sm[(size_t)s * tile_pts + off] = y[s];
  }
  __syncthreads();
}

// `scale` multiplies the phase (1 for the first kinetic table; P for a second
// one, whose 1/P factor belongs to an inverse FFT that does not run twice).
template <int L>
__device__ __forceinline__ void apply_kinetic(double2* sm, const double2* __restrict__ tau, const TileGeom& tg,
                                              int G, int SVl, long long stride, int tid, int nthr, const DPK& dk,
                                              double scale = 1.0) {
  const int tile_pts = G * L;
  for (int e = tid; e < tile_pts; e += nthr) {
    int g, n;
    tile_elem<L>(e, tg, g, n);
    double2 t = __ldg(&tau[tg.addr(g, n, L, stride)]);
    if (scale != 1.0) t = make_double2(dmul(t.x, scale, dk), dmul(t.y, scale, dk));
    const int off = g * L + n;
    for (int s = 0; s < SVl; ++s) {
      double2* p = &sm[(size_t)s * tile_pts + off];
      *p = cmul(*p, t, dk);
    }
  }
  __syncthreads();
}

// SV: surfaces staged together (S for passes with a potential step, 1 else).
// Each thread owns one 8-element work slot per FFT stage, so a CTA has
// SV * G * L / 8 threads; MaxThreads<L, SV> bounds it.
template <int L, int SV>
struct MaxThreads {
  static constexpr int value = (SV * L / 8 > 256) ? SV * L / 8 : 256;
};

template <int L, int SV>
__global__ void __launch_bounds__(MaxThreads<L, SV>::value) axis_pass_kernel(PassArgs a) {
  constexpr int K = 1;
  extern __shared__ double2 sm[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = a.G;
  const int tile_pts = G * L;
  const long long tiles_per_surface = a.lines / G;
  long long tile = blockIdx.x;
  int surf0 = 0;
  if (SV == 1) {
    surf0 = (int)(tile / tiles_per_surface);
    tile = tile - (long long)surf0 * tiles_per_surface;
  }
  // line id lambda = o * stride + i; the tile covers lambdas [tile*G, tile*G+G)
  const TileGeom tg = make_geom(tile, a);

  // load
  for (int s = 0; s < SV; ++s) {
    const double2* src = a.psi + (size_t)(surf0 + s) * a.P;
    for (int e = tid; e < tile_pts; e += nthr) {
      int g, n;
      tile_elem<L>(e, tg, g, n);
      sm[(size_t)s * tile_pts + g * L + n] = src[tg.addr(g, n, L, a.stride)];
    }
  }
  __syncthreads();

  const int nslots = SV * G * (L / 8);
  const DPK dk{a.one, a.mz};
  // The tile-wide steps (load, potential, kinetic phase, store) walk the tile
  // in address order and end with a block barrier; the FFT stages in between
  // only synchronise the threads of each line.
  if (a.flags & PASS_INV_FIRST) {
    fft_lines<L, true, K>(sm, a.tw, nslots, tid, nthr, dk);
    __syncthreads();
  }
  if (SV > 1) {  // the host sets U1/U2 only for passes that stage all S surfaces
    if (a.U1) apply_potential<L, SV>(sm, a.U1, tg, G, a.stride, a.P, tid, nthr, dk);
    if (a.U2) apply_potential<L, SV>(sm, a.U2, tg, G, a.stride, a.P, tid, nthr, dk);
  }
  if (a.flags & PASS_FWD) fft_lines<L, false, K>(sm, a.tw, nslots, tid, nthr, dk);
  if (a.flags & PASS_T) {
    __syncthreads();
    apply_kinetic<L>(sm, a.tau, tg, G, SV, a.stride, tid, nthr, dk);
    if (a.tau2) apply_kinetic<L>(sm, a.tau2, tg, G, SV, a.stride, tid, nthr, dk, a.tau2_scale);
    fft_lines<L, true, K>(sm, a.tw, nslots, tid, nthr, dk);
  }
  __syncthreads();

  // store
  for (int s = 0; s < SV; ++s) {
    double2* dst = a.psi + (size_t)(surf0 + s) * a.P;
    for (int e = tid; e < tile_pts; e += nthr) {
      int g, n;
      tile_elem<L>(e, tg, g, n);
      dst[tg.addr(g, n, L, a.stride)] = sm[(size_t)s * tile_pts + g * L + n];
    }
  }
}

}  // namespace dso
