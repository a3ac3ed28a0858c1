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
// The FP64 path on this GPU is bound by the FP64 pipe: 2 FP64 lanes per SM
// per clock, and (measured) 0.50 T instructions/s for DADD, DMUL and for a
// DFMA with two per-thread register operands, as in these butterflies.  The
// butterflies are written to minimise FP64 instructions: trivial twiddles
// (+-1, +-i) cost nothing, the (1 -+ i)/sqrt(2) factors of the radix-8
// butterfly fold into FMAs, and everything else (indexing, shared-memory
// traffic, table loads) runs on other pipes.
//
// Every routine is generic over the complex type C: double2 for the FP64
// path, float2 for the FP32 storage-and-FFT mode.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pass_args.h"

namespace dso {

template <typename C>
struct CxT;
template <>
struct CxT<double2> {
  using R = double;
};
template <>
struct CxT<float2> {
  using R = float;
};
template <typename C>
using RealT = typename CxT<C>::R;

__device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {
  return mkc(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  return mkc(a.x + b.x, a.y + b.y);
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  return mkc(a.x - b.x, a.y - b.y);
}
template <typename C>
__device__ __forceinline__ C cscale(C a, RealT<C> s) {
  return mkc(a.x * s, a.y * s);
}
// multiply by -i (forward) or +i (inverse): free, no floating-point instruction
template <bool INV, typename C>
__device__ __forceinline__ C rot_i(C a) {
  return INV ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
}

// Programmatic dependent launch.  Consecutive passes are launched so that a
// pass's CTAs may become resident while the previous pass is still running
// (its tail); `pdl_wait` blocks until the previous pass has completed and its
// writes are visible, so it comes before any read of data that pass wrote.
// `pdl_trigger` tells the scheduler that this CTA no longer needs the next
// pass held back; once every CTA has triggered (or exited) the next pass
// launches.  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// In-place DFT of length 2, 4, 8 with sign -1 (forward) or +1 (INV).
template <bool INV, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2);
  C t2 = cadd(a1, a3), t3 = rot_i<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// 8-point DFT by one radix-2 split into two 4-point DFTs:
// y_k = E_k + w^k O_k, y_{k+4} = E_k - w^k O_k, w = exp(-+2 pi i / 8).
template <bool INV, typename C>
__device__ __forceinline__ void dft8(C* x) {
  using R = RealT<C>;
  const R c = (R)0.70710678118654752440;  // 1/sqrt(2)
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // k = 0
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  // k = 2: w^2 = -+i
  C r2 = rot_i<INV>(o2);
  x[2] = cadd(e2, r2);
  x[6] = csub(e2, r2);
  // k = 1: w = (1 -+ i)/sqrt(2); w*o = c * u
  C u1 = INV ? mkc(o1.x - o1.y, o1.x + o1.y) : mkc(o1.x + o1.y, o1.y - o1.x);
  x[1] = mkc(fma(c, u1.x, e1.x), fma(c, u1.y, e1.y));
  x[5] = mkc(fma(-c, u1.x, e1.x), fma(-c, u1.y, e1.y));
  // k = 3: w^3 = (-1 -+ i)/sqrt(2)
  C u3 = INV ? mkc(-(o3.x + o3.y), o3.x - o3.y) : mkc(o3.y - o3.x, -(o3.x + o3.y));
  x[3] = mkc(fma(c, u3.x, e3.x), fma(c, u3.y, e3.y));
  x[7] = mkc(fma(-c, u3.x, e3.x), fma(-c, u3.y, e3.y));
}

// Twiddled radix-8 butterfly in tangent form.  A twiddle w = c + i s is
// stored as (c, t) with t = s / c, so that w b = c (b + i t b): the rotation
// b + i t b costs two FMAs, and both outputs a +- w b of a radix-2 pair then
// cost two FMAs each, 6 FP64 instructions per pair instead of the 8 of a
// complex multiply and two complex additions.  In a decimation-in-time
// radix-8 stage the seven input twiddles are the powers w^r of one twiddle
// w; splitting the 8-point DFT into three radix-2 layers and factoring the
// common powers out of each pair leaves four distinct factors,
//   w^4 (first layer), w^2 (second layer), w and W8 w (last layer),
// with W8 = exp(-+ 2 pi i / 8) and the factors -+i of the other pairs free.
// That is 12 pairs, 72 FP64 instructions per 8 points, against 7 complex
// multiplies (28) plus the 52 of the butterfly.  A twiddle with c = 0 is
// stored with c = 2^-500 (2^-60 in FP32) and t = s / c; the product c (b + i t b)
// is then exact up to a relative error far below one ulp.
template <bool INV, bool ROT, typename C>
__device__ __forceinline__ void tan_pair(C& a, C& b, C w) {
  // (a, b) <- (a + f b, a - f b), f = w (or conj w when INV), times -+i when ROT
  const auto t = INV ? -w.y : w.y;
  const auto c = w.x;
  const auto zx = fma(-t, b.y, b.x);
  const auto zy = fma(t, b.x, b.y);
  C p, q;
  if (!ROT) {
    p = mkc(fma(c, zx, a.x), fma(c, zy, a.y));
    q = mkc(fma(-c, zx, a.x), fma(-c, zy, a.y));
  } else if (!INV) {  // -i (c z) = (c zy, -c zx)
    p = mkc(fma(c, zy, a.x), fma(-c, zx, a.y));
    q = mkc(fma(-c, zy, a.x), fma(c, zx, a.y));
  } else {            // +i (c z) = (-c zy, c zx)
    p = mkc(fma(-c, zy, a.x), fma(c, zx, a.y));
    q = mkc(fma(c, zy, a.x), fma(-c, zx, a.y));
  }
  a = p;
  b = q;
}

// 8-point DFT of (w^r x_r), r = 0..7, in place and in natural output order,
// given the tangent-form factors w1 = w, w2 = w^2, w4 = w^4, w8 = W8 w.
template <bool INV, typename C>
__device__ __forceinline__ void dft8_tw(C* x, C w1, C w2, C w4, C w8) {
  // first layer: pairs (r, r+4) with factor w^4
  tan_pair<INV, false>(x[0], x[4], w4);
  tan_pair<INV, false>(x[2], x[6], w4);
  tan_pair<INV, false>(x[1], x[5], w4);
  tan_pair<INV, false>(x[3], x[7], w4);
  // second layer: 4-point DFTs of the even and odd halves, factor w^2
  tan_pair<INV, false>(x[0], x[2], w2);
  tan_pair<INV, true>(x[4], x[6], w2);
  tan_pair<INV, false>(x[1], x[3], w2);
  tan_pair<INV, true>(x[5], x[7], w2);
  // now x0, x4, x2, x6 hold E_0..E_3 and x1, x5, x3, x7 hold O'_0..O'_3;
  // last layer: y_k = E_k + W8^k w O'_k, y_{k+4} = E_k - W8^k w O'_k
  tan_pair<INV, false>(x[0], x[1], w1);  // k = 0
  tan_pair<INV, false>(x[4], x[5], w8);  // k = 1
  tan_pair<INV, true>(x[2], x[3], w1);   // k = 2: W8^2 = -+i
  tan_pair<INV, true>(x[6], x[7], w8);   // k = 3: W8^3 w = -+i W8 w
  // outputs: y0 = x0, y4 = x1, y1 = x4, y5 = x5, y2 = x2, y6 = x3, y3 = x6, y7 = x7
  const C y1 = x[4], y4 = x[1], y3 = x[6], y6 = x[3];
  x[1] = y1;
  x[4] = y4;
  x[3] = y3;
  x[6] = y6;
}

// Loads the four tangent-form factors of the butterfly with twiddle index
// `step` (w = tw[step]) from a length-L tangent-form table, in global memory
// (read-only path) or, with SHARED, in shared memory.
template <int L, bool SHARED = false, typename C>
__device__ __forceinline__ void load_tw8(const C* __restrict__ tw, int step, C& w1, C& w2, C& w4, C& w8) {
  if constexpr (SHARED) {
    w1 = tw[step];
    w2 = tw[2 * step];
    w4 = tw[4 * step];
    w8 = tw[step + L / 8];
  } else {
    w1 = __ldg(&tw[step]);
    w2 = __ldg(&tw[2 * step]);
    w4 = __ldg(&tw[4 * step]);
    w8 = __ldg(&tw[step + L / 8]);
  }
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void dftR(C* x) {
  if constexpr (R == 8) {
    dft8<INV>(x);
  } else if constexpr (R == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3]);
  } else {
    dft2<INV>(x[0], x[1]);
  }
}

// Radix plan of a length-L transform: as many radix-8 stages as possible,
// the leftover factor (2 or 4) as the first stage, whose twiddles are all 1.
template <int L>
struct Plan {
  static constexpr int log2L = (L >= 8192) ? 13 : (L >= 4096) ? 12 : (L >= 2048) ? 11 : (L >= 1024) ? 10
                             : (L >= 512) ? 9 : (L >= 256) ? 8 : (L >= 128) ? 7 : (L >= 64) ? 6 : (L >= 32) ? 5
                             : (L >= 16) ? 4 : 3;
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

// Shared-memory layout of the lines of a tile.  Element n of a line sits at
// n + (n >> plog), one pad element after every 2^plog, and consecutive lines
// are ls elements apart.  Unpadded, the Stockham stores of the early stages
// (outputs Ls apart, Ls small) and the tile loads of strided axes (lines L
// apart, L a multiple of the 32 banks) hit a few banks many times: 2.4-4.4x
// the minimum number of shared-memory wavefronts, which in the FP32 mode made
// the passes shared-memory bound (L1TEX 95 % busy, mio_throttle the top
// stall).  The pad spacing (8 elements for 16-byte complex numbers, 16 for
// 8-byte ones on lines of 128 or more) and the extra line offset X, chosen
// with the tile's inner width Wi (Wi lines of consecutive addresses load
// together), bring every stage and loop of the tile kernel to the minimum
// (FP64, L >= 64) or within 1.3x of it (FP32, L >= 128), counted with a
// model of the 32 banks over each warp-wide access.
struct SmemLayout {
  int ls;    // elements from one line to the next
  int plog;  // log2 of the pad spacing (31: no padding)
  __host__ __device__ __forceinline__ int pos(int n) const { return n + (n >> plog); }
};

__host__ __device__ inline SmemLayout tile_layout(int L, int esz, int Wi) {
  SmemLayout s;
  int X;
  if (esz == 16) {
    s.plog = 3;
    X = (L >= 64) ? (Wi <= 8 ? 8 / Wi : 1) : 0;
  } else if (L >= 128) {
    s.plog = 4;
    X = Wi <= 16 ? 16 / Wi : 1;
  } else {
    s.plog = 3;
    X = 0;
  }
  s.ls = L + (L >> s.plog) + X;
  return s;
}

__host__ __device__ inline SmemLayout plain_layout(int L) {
  SmemLayout s;
  s.ls = L;
  s.plog = 31;
  return s;
}

// One Stockham stage of radix R on every line of the tile held in `sm`.
// Thread-slot s of this thread owns 8 consecutive butterfly inputs' worth of
// work: 8/R butterflies j = u*(8/R) + beta of line `line`.
template <int L, int R, bool INV, int K, typename C>
__device__ __forceinline__ void stockham_stage(C* sm, int Ls, const C* __restrict__ tw, int nslots, int tid,
                                               int nthr, unsigned wmask, const SmemLayout lay) {
  constexpr int NB = 8 / R;      // butterflies per slot
  constexpr int Q = L / R;       // butterflies per line
  C v[K][8];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int gid = s * nthr + tid;
    if (gid < nslots) {
      const int line = gid / (L / 8);
      const int u = gid % (L / 8);
      const C* ln = sm + (size_t)line * lay.ls;
#pragma unroll
      for (int beta = 0; beta < NB; ++beta) {
        const int j = u * NB + beta;
#pragma unroll
        for (int r = 0; r < R; ++r) v[s][beta * R + r] = ln[lay.pos(j + r * Q)];
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
      C* ln = sm + (size_t)line * lay.ls;
#pragma unroll
      for (int beta = 0; beta < NB; ++beta) {
        const int j = u * NB + beta;
        const int k = j & (Ls - 1);
        C* x = &v[s][beta * R];
        if (R == 8 && Ls > 1) {  // twiddled stages are radix 8 (the leftover radix goes first)
          C w1, w2, w4, w8;
          load_tw8<L>(tw, (L / (Ls * 8)) * k, w1, w2, w4, w8);
          dft8_tw<INV>(x, w1, w2, w4, w8);
        } else {
          dftR<R, INV>(x);
        }
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) ln[lay.pos(base + r * Ls)] = x[r];
      }
    }
  }
  stage_sync<L>(wmask);
}

template <int L, bool INV, int K, typename C>
__device__ __forceinline__ void fft_lines(C* sm, const C* __restrict__ tw, int nslots, int tid, int nthr,
                                          const SmemLayout lay) {
  using PL = Plan<L>;
  const unsigned wmask = warp_lanes_mask(tid, nthr);
  stockham_stage<L, PL::first, INV, K>(sm, 1, tw, nslots, tid, nthr, wmask, lay);
  int Ls = PL::first;
#pragma unroll 1
  for (int st = 0; st < PL::n8; ++st) {
    stockham_stage<L, 8, INV, K>(sm, Ls, tw, nslots, tid, nthr, wmask, lay);
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

__device__ __forceinline__ TileJob split_tile(long long tile, int SV, const PassArgs& a) {
  TileJob t;
  const long long per_set = a.lines >> a.G_log2;  // tiles per line set (one surface, or one job's S)
  const long long set = tile / per_set;
  t.tile = tile - set * per_set;
  if (SV == 1) {
    t.surf0 = (int)set;
    t.job = (int)(set / a.S);
  } else {
    t.job = (int)set;
    t.surf0 = (int)set * a.S;
  }
  return t;
}

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

// S x S complex matvec with the packed complex-symmetric unitary (entries
// in C, products accumulated in C's precision).  With dec0, surface 0 is
// uncoupled from the others (its off-diagonal potential entries vanish on the
// whole grid, as in the paper's pyrazine model), so U is block diagonal:
// U_0c = 0 for c > 0 and those products are skipped.  The branch is uniform
// across the launch.
template <int SV, typename C>
__device__ __forceinline__ void matvec_rows(const C (&u)[SV * (SV + 1) / 2], const C (&x)[SV], C (&y)[SV],
                                            int r0) {
#pragma unroll
  for (int r = 0; r < SV; ++r) {
    if (r < r0) continue;
    C acc = mkc((RealT<C>)0, (RealT<C>)0);
#pragma unroll
    for (int c = 0; c < SV; ++c) {
      if (c < r0) continue;
      const int lo = r < c ? r : c, hi = r < c ? c : r;
      const int k = lo * SV - lo * (lo - 1) / 2 + (hi - lo);
      if (c == r0) {
        acc = cmul(u[k], x[c]);
      } else {
        acc.x = fma(u[k].x, x[c].x, acc.x);
        acc.x = fma(-u[k].y, x[c].y, acc.x);
        acc.y = fma(u[k].x, x[c].y, acc.y);
        acc.y = fma(u[k].y, x[c].x, acc.y);
      }
    }
    y[r] = acc;
  }
}

template <int SV, typename C>
__device__ __forceinline__ void matvec_sym(const C (&u)[SV * (SV + 1) / 2], const C (&x)[SV], C (&y)[SV],
                                           int dec0 = 0) {
  if (SV > 2 && dec0) {
    y[0] = cmul(u[0], x[0]);
    matvec_rows<SV>(u, x, y, 1);
  } else {
    matvec_rows<SV>(u, x, y, 0);
  }
}

// With DSO_DEBUG_BOUNDS every global access of the tile kernel is checked
// against its allocation; a bad index sets *err and the access is skipped.
#ifdef DSO_DEBUG_BOUNDS
#define DSO_CHECK_INDEX(idx, extent, code, err) \
  (((idx) >= 0 && (idx) < (extent)) ? true : (atomicExch((err), (code)), false))
// first bad access of the tile kernel, with its tile context: err[1..15]
#define DSO_RECORD(err, v0, v1, v2, v3, v4, v5, v6, v7)                    \
  do {                                                                  \
    if (atomicCAS((err) + 1, 0, 1) == 0) {                              \
      (err)[2] = (int)(v0); (err)[3] = (int)(v1); (err)[4] = (int)(v2); \
      (err)[5] = (int)(v3); (err)[6] = (int)(v4); (err)[7] = (int)(v5); \
      (err)[8] = (int)(v6); (err)[9] = (int)(v7);                       \
    }                                                                   \
  } while (0)
#else
#define DSO_CHECK_INDEX(idx, extent, code, err) true
#endif

template <int L, int SV, typename C>
__device__ __forceinline__ void apply_potential(C* sm, const C* __restrict__ U, const TileGeom& tg, int G,
                                                long long stride, long long P, int tid, int nthr,
                                                const SmemLayout lay, const PassArgs* dbg = nullptr) {
  constexpr int NP = SV * (SV + 1) / 2;
  const int tile_pts = G * L;
  const int tile_sz = G * lay.ls;  // shared-memory elements per staged surface
  const int dec0 = dbg ? dbg->dec0 : 0;
  for (int e = tid; e < tile_pts; e += nthr) {
    int g, n;
    tile_elem<L>(e, tg, g, n);
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
#ifdef DSO_DEBUG_BOUNDS
      if (dbg) {
        const long long off = (long long)(&U[(size_t)k * P + gi] - (const C*)dbg->U_base);
        if (!DSO_CHECK_INDEX(off, dbg->u_elems, 102, dbg->err)) {
          u[k] = mkc((RealT<C>)0, (RealT<C>)0);
          continue;
        }
      }
#endif
      u[k] = __ldg(&U[(size_t)k * P + gi]);
    }
    matvec_sym<SV>(u, x, y, dec0);
#pragma unroll
    for (int s = 0; s < SV; ++s) sm[(size_t)s * tile_sz + off] = y[s];
  }
  __syncthreads();
}

// `scale` multiplies the phase (1 for the first kinetic table; P for a second
// one, whose 1/P factor belongs to an inverse FFT that does not run twice).
// With `axis_table` the phase is this axis's alone: element n of every line
// takes tau[n] (separable kinetic step).
template <int L, typename C>
__device__ __forceinline__ void apply_kinetic(C* sm, const C* __restrict__ tau, const TileGeom& tg, int G, int SVl,
                                              long long stride, int tid, int nthr, RealT<C> scale,
                                              const SmemLayout lay, const PassArgs* dbg = nullptr,
                                              bool axis_table = false) {
  const int tile_pts = G * L;
  const int tile_sz = G * lay.ls;
  if (axis_table) {
    for (int e = tid; e < tile_pts; e += nthr) {
      int g, n;
      tile_elem<L>(e, tg, g, n);
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
      const int g = e >> Plan<L>::log2L, n = e & (L - 1);
#ifdef DSO_DEBUG_BOUNDS
      if (dbg && !DSO_CHECK_INDEX((long long)(&blk[e] - (const C*)dbg->tau_base), dbg->tau_elems, 103, dbg->err))
        continue;
#endif
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
    tile_elem<L>(e, tg, g, n);
#ifdef DSO_DEBUG_BOUNDS
    if (dbg) {
      const long long off = (long long)(&tau[tg.addr(g, n, L, stride)] - (const C*)dbg->tau_base);
      if (!DSO_CHECK_INDEX(off, dbg->tau_elems, 103, dbg->err)) continue;
    }
#endif
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

// Four-step twiddles of a split axis (see VLayout): the element at position
// k1 of a line along the first factor, whose line sits at index i2 of the
// second factor, is multiplied by w_n^(k1 i2) after the forward FFT along the
// line, or by its conjugate before the inverse FFT.  The table is laid out
// [n1][n2], so the factor of (k1, i2) is xtw[k1 n2 + i2].
template <int L, bool CONJ, typename C>
__device__ __forceinline__ void apply_split_twiddles(C* sm, const C* __restrict__ xtw, const TileGeom& tg, int G,
                                                     int SVl, int n2_log2, int s2_log2, int tid, int nthr,
                                                     const SmemLayout lay) {
  const int tile_pts = G * L;
  const int tile_sz = G * lay.ls;
  const long long n2_mask = (1LL << n2_log2) - 1;
  for (int e = tid; e < tile_pts; e += nthr) {
    int g, n;
    tile_elem<L>(e, tg, g, n);
    const long long i = tg.i0 + (g & (tg.Wi - 1));  // inner index of the line
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

// SV: surfaces staged together (S for passes with a potential step, 1 else).
// Each thread owns one 8-element work slot per FFT stage, so a CTA has
// SV * G * L / 8 threads; MaxThreads<L, SV> bounds it.
template <int L, int SV>
struct MaxThreads {
  static constexpr int value = (SV * L / 8 > 256) ? SV * L / 8 : 256;
};

template <int L, int SV, typename C>
__global__ void __launch_bounds__(MaxThreads<L, SV>::value) axis_pass_kernel(PassArgs a) {
  constexpr int K = 1;
  extern __shared__ __align__(16) unsigned char sm_bytes[];
  C* sm = reinterpret_cast<C*>(sm_bytes);
  C* psi = reinterpret_cast<C*>(a.psi);
  const C* tw = reinterpret_cast<const C*>(a.tw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = a.G;
  const int tile_pts = G * L;
  const TileJob tj = split_tile(blockIdx.x, SV, a);
  const int surf0 = tj.surf0;
  const size_t uoff = (size_t)tj.job * a.u_batch_stride;
  // line id lambda = o * stride + i; the tile covers lambdas [tile*G, tile*G+G)
  const TileGeom tg = make_geom(tj.tile, a);
  const SmemLayout lay = tile_layout(L, (int)sizeof(C), tg.Wi);
  const int tile_sz = G * lay.ls;  // shared-memory elements per staged surface

  pdl_wait();  // psi is the previous pass's output
  // load.  Two common tile shapes are addressed directly: lines along the
  // contiguous axis (the tile is one contiguous block), and tiles of G
  // consecutive inner positions of one outer row (G <= stride: element
  // (n, i) sits at row + n * stride + i).
  const bool contig = a.stride_log2 == 0;
  const bool one_row = !contig && a.G_log2 <= a.stride_log2;
  const long long row = ((tg.o0 * L) << a.stride_log2) + tg.i0;  // first element of a one-row tile
  for (int s = 0; s < SV; ++s) {
    const C* src = psi + (size_t)(surf0 + s) * a.P;
    if (contig) {
      const C* blk = src + (size_t)tg.o0 * L;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int g = e >> Plan<L>::log2L, n = e & (L - 1);
        if (DSO_CHECK_INDEX((long long)(surf0 + s) * a.P + tg.o0 * L + e, a.psi_elems, 100, a.err))
          sm[s * tile_sz + g * lay.ls + lay.pos(n)] = blk[e];
      }
      continue;
    }
    if (one_row) {
      const C* blk = src + row;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int i = e & (G - 1), n = e >> a.G_log2;
        const long long off = ((long long)n << a.stride_log2) + i;
        if (DSO_CHECK_INDEX((long long)(surf0 + s) * a.P + row + off, a.psi_elems, 100, a.err))
          sm[s * tile_sz + i * lay.ls + lay.pos(n)] = blk[off];
      }
      continue;
    }
    for (int e = tid; e < tile_pts; e += nthr) {
      int g, n;
      tile_elem<L>(e, tg, g, n);
      const long long gidx = (long long)(surf0 + s) * a.P + tg.addr(g, n, L, a.stride);
      if (DSO_CHECK_INDEX(gidx, a.psi_elems, 100, a.err))
        sm[(size_t)s * tile_sz + g * lay.ls + lay.pos(n)] = src[tg.addr(g, n, L, a.stride)];
    }
  }
  __syncthreads();
  pdl_trigger();

  const int nslots = SV * G * (L / 8);
  // The tile-wide steps (load, potential, kinetic phase, store) walk the tile
  // in address order and end with a block barrier; the FFT stages in between
  // only synchronise the threads of each line.
  if (a.flags & PASS_INV_FIRST) {
    if (a.flags & PASS_XTW)
      apply_split_twiddles<L, true>(sm, reinterpret_cast<const C*>(a.xtw), tg, G, SV, a.xtw_n2_log2,
                                    a.xtw_s2_log2, tid, nthr, lay);
    fft_lines<L, true, K>(sm, tw, nslots, tid, nthr, lay);
    __syncthreads();
  }
  if (SV > 1) {  // the host sets U1/U2 only for passes that stage all S surfaces
    if (a.U1)
      apply_potential<L, SV>(sm, reinterpret_cast<const C*>(a.U1) + uoff, tg, G, a.stride, a.P, tid, nthr, lay,
                             &a);
    if (a.U2)
      apply_potential<L, SV>(sm, reinterpret_cast<const C*>(a.U2) + uoff, tg, G, a.stride, a.P, tid, nthr, lay,
                             &a);
  }
  if (a.flags & PASS_FWD) {
    fft_lines<L, false, K>(sm, tw, nslots, tid, nthr, lay);
    if (a.flags & PASS_XTW) {
      __syncthreads();
      apply_split_twiddles<L, false>(sm, reinterpret_cast<const C*>(a.xtw), tg, G, SV, a.xtw_n2_log2,
                                     a.xtw_s2_log2, tid, nthr, lay);
    }
  }
  if (a.flags & PASS_T) {
    __syncthreads();
    const bool tax = (a.flags & PASS_TAX) != 0;
    apply_kinetic<L>(sm, reinterpret_cast<const C*>(a.tau), tg, G, SV, a.stride, tid, nthr, (RealT<C>)1, lay, &a,
                     tax);
    if (a.tau2)
      apply_kinetic<L>(sm, reinterpret_cast<const C*>(a.tau2), tg, G, SV, a.stride, tid, nthr,
                       (RealT<C>)a.tau2_scale, lay, &a, tax);
    fft_lines<L, true, K>(sm, tw, nslots, tid, nthr, lay);
  }
  __syncthreads();

  // store
  for (int s = 0; s < SV; ++s) {
    C* dst = psi + (size_t)(surf0 + s) * a.P;
    if (contig) {
      C* blk = dst + (size_t)tg.o0 * L;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int g = e >> Plan<L>::log2L, n = e & (L - 1);
        if (DSO_CHECK_INDEX((long long)(surf0 + s) * a.P + tg.o0 * L + e, a.psi_elems, 101, a.err))
          blk[e] = sm[s * tile_sz + g * lay.ls + lay.pos(n)];
      }
      continue;
    }
    if (one_row) {
      C* blk = dst + row;
      for (int e = tid; e < tile_pts; e += nthr) {
        const int i = e & (G - 1), n = e >> a.G_log2;
        const long long off = ((long long)n << a.stride_log2) + i;
        if (DSO_CHECK_INDEX((long long)(surf0 + s) * a.P + row + off, a.psi_elems, 101, a.err))
          blk[off] = sm[s * tile_sz + i * lay.ls + lay.pos(n)];
      }
      continue;
    }
    for (int e = tid; e < tile_pts; e += nthr) {
      int g, n;
      tile_elem<L>(e, tg, g, n);
      const long long gidx = (long long)(surf0 + s) * a.P + tg.addr(g, n, L, a.stride);
#ifdef DSO_DEBUG_BOUNDS
      if (gidx < 0 || gidx >= a.psi_elems)
        DSO_RECORD(a.err, blockIdx.x, surf0, tg.o0, tg.i0, g, n, a.G, (a.stride_log2 << 16) | (tg.Wi_log2 << 8) | s);
#endif
      if (DSO_CHECK_INDEX(gidx, a.psi_elems, 101, a.err))
        dst[tg.addr(g, n, L, a.stride)] = sm[(size_t)s * tile_sz + g * lay.ls + lay.pos(n)];
    }
  }
}

}  // namespace dso
