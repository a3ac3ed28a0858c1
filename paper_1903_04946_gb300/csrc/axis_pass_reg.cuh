// axis_pass_reg.cuh -- register-resident axis pass for lines of 32, 64 and
// 128 points: FFT-only passes, kinetic passes [F T I] and, for passes that
// stage all S surfaces, the potential step ([I0 V F0], [V F0 T0 I0], [V]).
//
// The tile kernel (axis_pass.cuh) moves a tile through shared memory once per
// Stockham stage, and for FP32 data its passes issue ~110 thread instructions
// per amplitude, most of them shared-memory traffic and index arithmetic
// around ~20 FP32 instructions of FFT work.  Here each line is held by TPL
// threads, thread t holding the elements t + TPL m (m = 0..VPT-1), loaded
// straight from global memory.  For these lengths the data of the first
// Stockham stage(s) lies in one thread, so those stages run in registers and
// one shared-memory exchange brings each thread the inputs of the last stage,
// whose outputs land again in the distribution t + TPL m: a forward FFT, the
// kinetic phase and the inverse FFT follow each other without any reordering.
// Every butterfly is the tile kernel's -- the same radix plan (Plan<L>), the
// same tangent-form twiddles and the same inputs in the same order -- so the
// two kernels give bitwise the same results (for L = 128 up to the sign of a
// zero: the butterflies with twiddle index 0 skip their exact unit factors):
//   L =  32: radix 4 (butterflies j = t, t + 4) then radix 8 (j = t);
//   L =  64: radix 8 (j = t) then radix 8 (j = t);
//   L = 128: radix 2 (j = t + 8r), radix 8 (j = 2t, 2t + 1), then radix 8
//            (j = t, t + 8).
// A thread holds its elements of the lines of all SV staged surfaces at one
// line position, so the potential step (a matvec over the surfaces at each
// point) needs no data movement at all.  Lines along the contiguous axis put
// the TPL threads of a line in one warp (a warp barrier between the halves of
// the exchange); strided lines put 16 or more consecutive lines in a warp
// (coalesced loads) and the TPL parts of a line in different warps (a block
// barrier).  The exchange buffers are padded as a 32-bank model of the two
// access patterns finds conflict-free (L = 64, 128).
#pragma once

#include "axis_pass.cuh"

namespace dso {

template <int L>
struct RegPlan;
template <>
struct RegPlan<32> {
  static constexpr int TPL = 4, VPT = 8;
};
template <>
struct RegPlan<64> {
  static constexpr int TPL = 8, VPT = 8;
};
template <>
struct RegPlan<128> {
  static constexpr int TPL = 8, VPT = 16;
};

// Threads per CTA: 128, four CTAs per SM for one staged surface and two for
// S surfaces (whose amplitudes take most of a thread's registers), so that
// one CTA's loads overlap another's FFTs and a pass's last CTAs are short.
template <int SV>
__host__ __device__ constexpr int reg_threads() {
  return 128;
}

// Line positions per CTA (the tile line count G the host must use).
template <int L, int SV>
__host__ __device__ constexpr int reg_lines() {
  return reg_threads<SV>() / RegPlan<L>::TPL;
}

// Exchange buffer of one line: element n at n + (n >> plog), lines LS apart.
template <int L, bool WL>
struct RegLayout {
  static constexpr int plog = WL ? (L == 128 ? 4 : 3) : 31;
  static constexpr int LS = WL ? L + (L >> plog) : L + 1;
  __device__ __forceinline__ static int pos(int n) { return plog < 31 ? n + (n >> plog) : n; }
};

template <bool WL>
__device__ __forceinline__ void reg_sync() {
  if (WL) __syncwarp(); else __syncthreads();
}

// The butterflies of axis_pass.cuh with the transform's direction as a
// runtime sign sg = +1 (forward, exp(-i ..)) or -1 (inverse): every INV
// branch there becomes a multiplication by sg, which is exact, so each
// output is the template version's, bit for bit.  One body serves both
// directions, halving the kernel's straight-line code.
template <typename C>
__device__ __forceinline__ C rot_i_s(C a, RealT<C> sg) {  // -i a (forward), +i a (inverse)
  return mkc(sg * a.y, -sg * a.x);
}

template <typename C>
__device__ __forceinline__ void dft4_s(C& a0, C& a1, C& a2, C& a3, RealT<C> sg) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2);
  C t2 = cadd(a1, a3), t3 = rot_i_s(csub(a1, a3), sg);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <typename C>
__device__ __forceinline__ void dft8_s(C* x, RealT<C> sg) {
  using R = RealT<C>;
  const R c = (R)0.70710678118654752440;  // 1/sqrt(2)
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4_s(e0, e1, e2, e3, sg);
  dft4_s(o0, o1, o2, o3, sg);
  x[0] = cadd(e0, o0);
  x[4] = csub(e0, o0);
  C r2 = rot_i_s(o2, sg);
  x[2] = cadd(e2, r2);
  x[6] = csub(e2, r2);
  // forward (x + y, y - x), inverse (x - y, x + y)
  C u1 = mkc(o1.x + sg * o1.y, o1.y - sg * o1.x);
  x[1] = mkc(fma(c, u1.x, e1.x), fma(c, u1.y, e1.y));
  x[5] = mkc(fma(-c, u1.x, e1.x), fma(-c, u1.y, e1.y));
  // forward (y - x, -(x + y)), inverse (-(x + y), x - y)
  C u3 = mkc(sg * o3.y - o3.x, -sg * o3.x - o3.y);
  x[3] = mkc(fma(c, u3.x, e3.x), fma(c, u3.y, e3.y));
  x[7] = mkc(fma(-c, u3.x, e3.x), fma(-c, u3.y, e3.y));
}

// tan_pair with the twiddle's tangent already signed (ts = sg t) and, for
// the rotated pairs, its cosine signed (cs = sg c).
template <bool ROT, typename C>
__device__ __forceinline__ void tan_pair_s(C& a, C& b, RealT<C> c, RealT<C> ts, RealT<C> cs) {
  const auto zx = fma(-ts, b.y, b.x);
  const auto zy = fma(ts, b.x, b.y);
  C p, q;
  if (!ROT) {
    p = mkc(fma(c, zx, a.x), fma(c, zy, a.y));
    q = mkc(fma(-c, zx, a.x), fma(-c, zy, a.y));
  } else {
    p = mkc(fma(cs, zy, a.x), fma(-cs, zx, a.y));
    q = mkc(fma(-cs, zy, a.x), fma(cs, zx, a.y));
  }
  a = p;
  b = q;
}

template <typename C>
__device__ __forceinline__ void dft8_tw_s(C* x, C w1, C w2, C w4, C w8, RealT<C> sg) {
  const auto t1 = sg * w1.y, t2 = sg * w2.y, t4 = sg * w4.y, t8 = sg * w8.y;
  const auto c1 = sg * w1.x, c2 = sg * w2.x, c8 = sg * w8.x;
  tan_pair_s<false>(x[0], x[4], w4.x, t4, t4);
  tan_pair_s<false>(x[2], x[6], w4.x, t4, t4);
  tan_pair_s<false>(x[1], x[5], w4.x, t4, t4);
  tan_pair_s<false>(x[3], x[7], w4.x, t4, t4);
  tan_pair_s<false>(x[0], x[2], w2.x, t2, c2);
  tan_pair_s<true>(x[4], x[6], w2.x, t2, c2);
  tan_pair_s<false>(x[1], x[3], w2.x, t2, c2);
  tan_pair_s<true>(x[5], x[7], w2.x, t2, c2);
  tan_pair_s<false>(x[0], x[1], w1.x, t1, c1);
  tan_pair_s<false>(x[4], x[5], w8.x, t8, c8);
  tan_pair_s<true>(x[2], x[3], w1.x, t1, c1);
  tan_pair_s<true>(x[6], x[7], w8.x, t8, c8);
  const C y1 = x[4], y4 = x[1], y3 = x[6], y6 = x[3];
  x[1] = y1;
  x[4] = y4;
  x[3] = y3;
  x[6] = y6;
}

// dft8_tw_s for butterfly k = 0, whose twiddles w1 = w2 = w4 = (1, 0)
// exactly: with tangent 0 and cosine 1 each of their tangent pairs is the
// sum and difference of its operands (or of a and -+i b), rounded once as
// the FMAs round it, so only the w8 pairs keep the tangent form.  The
// outputs are dft8_tw_s's up to the sign of a zero.
template <typename C>
__device__ __forceinline__ void pair_add(C& a, C& b) {
  const C p = cadd(a, b), q = csub(a, b);
  a = p;
  b = q;
}
template <typename C>
__device__ __forceinline__ void pair_rot(C& a, C& b, RealT<C> sg) {  // (a -+ i b, a +- i b)
  const C p = mkc(fma(sg, b.y, a.x), fma(-sg, b.x, a.y));
  const C q = mkc(fma(-sg, b.y, a.x), fma(sg, b.x, a.y));
  a = p;
  b = q;
}
template <typename C>
__device__ __forceinline__ void dft8_k0_s(C* x, C w8, RealT<C> sg) {
  const auto t8 = sg * w8.y, c8 = sg * w8.x;
  pair_add(x[0], x[4]);
  pair_add(x[2], x[6]);
  pair_add(x[1], x[5]);
  pair_add(x[3], x[7]);
  pair_add(x[0], x[2]);
  pair_rot(x[4], x[6], sg);
  pair_add(x[1], x[3]);
  pair_rot(x[5], x[7], sg);
  pair_add(x[0], x[1]);
  tan_pair_s<false>(x[4], x[5], w8.x, t8, c8);
  pair_rot(x[2], x[3], sg);
  tan_pair_s<true>(x[6], x[7], w8.x, t8, c8);
  const C y1 = x[4], y4 = x[1], y3 = x[6], y6 = x[3];
  x[1] = y1;
  x[4] = y4;
  x[3] = y3;
  x[6] = y6;
}

// Inverse or forward FFT of SV lines (one per staged surface) at this
// thread's line position.  The register stages of all SV lines share the
// twiddle loads; the lines go through the one exchange buffer (G lines) in
// turn.
template <int L, int SV, bool WL, typename C>
__device__ __forceinline__ void fft_reg(C (&v)[SV][RegPlan<L>::VPT], C* ln, int t, const C* __restrict__ tw,
                                        RealT<C> sg) {
  using LY = RegLayout<L, WL>;
  C w1, w2, w4, w8;
  if constexpr (L == 64) {
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_s(v[s], sg);  // stage 1 (Ls = 1): j = t on x[t + 8r]; y[8t + r]
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      reg_sync<WL>();  // earlier readers of the buffer are done
#pragma unroll
      for (int r = 0; r < 8; ++r) ln[LY::pos(8 * t + r)] = v[s][r];
      reg_sync<WL>();
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][r] = ln[LY::pos(t + 8 * r)];
    }
    load_tw8<64>(tw, t, w1, w2, w4, w8);  // stage 2 (Ls = 8): butterfly k = t
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_tw_s(v[s], w1, w2, w4, w8, sg);  // X[t + 8r] = v[r]
  } else if constexpr (L == 128) {
#pragma unroll
    for (int s = 0; s < SV; ++s) {
#pragma unroll
      for (int r = 0; r < 8; ++r) dft2<false>(v[s][r], v[s][r + 8]);  // stage 1: j = t + 8r -> y[2j], y[2j + 1]
    }
    w8 = __ldg(&tw[128 / 8]);  // stage 2 (Ls = 2): j = 2t (k = 0), inputs y[2t + 16r]
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_k0_s(&v[s][0], w8, sg);
    load_tw8<128>(tw, 8, w1, w2, w4, w8);  // j = 2t + 1 (k = 1), inputs y[2t + 1 + 16r]
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_tw_s(&v[s][8], w1, w2, w4, w8, sg);
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      reg_sync<WL>();
#pragma unroll
      for (int r = 0; r < 8; ++r) {  // z[16t + 2r] from j = 2t, z[16t + 2r + 1] from j = 2t + 1
        ln[LY::pos(16 * t + 2 * r)] = v[s][r];
        ln[LY::pos(16 * t + 2 * r + 1)] = v[s][8 + r];
      }
      reg_sync<WL>();
#pragma unroll
      for (int r = 0; r < 8; ++r) {  // z[t + 16r], z[t + 8 + 16r]: the elements t + 8m, m = 2r, 2r + 1
        v[s][2 * r] = ln[LY::pos(t + 16 * r)];
        v[s][2 * r + 1] = ln[LY::pos(t + 8 + 16 * r)];
      }
    }
    load_tw8<128>(tw, t, w1, w2, w4, w8);  // stage 3 (Ls = 16): k = t
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      C a[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = v[s][2 * r];
      dft8_tw_s(a, w1, w2, w4, w8, sg);  // X[t + 16r]
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][2 * r] = a[r];
    }
    load_tw8<128>(tw, t + 8, w1, w2, w4, w8);  // k = t + 8
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      C b[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) b[r] = v[s][2 * r + 1];
      dft8_tw_s(b, w1, w2, w4, w8, sg);  // X[t + 8 + 16r]
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][2 * r + 1] = b[r];
    }
  } else {  // L == 32
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      dft4_s(v[s][0], v[s][2], v[s][4], v[s][6], sg);  // stage 1: j = t on x[t + 8r]; y[4t + r]
      dft4_s(v[s][1], v[s][3], v[s][5], v[s][7], sg);  // j = t + 4 on x[t + 4 + 8r]; y[4t + 16 + r]
    }
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      reg_sync<WL>();
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        ln[LY::pos(4 * t + r)] = v[s][2 * r];
        ln[LY::pos(4 * t + 16 + r)] = v[s][2 * r + 1];
      }
      reg_sync<WL>();
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][r] = ln[LY::pos(t + 4 * r)];
    }
    load_tw8<32>(tw, t, w1, w2, w4, w8);  // stage 2 (Ls = 4): butterfly k = t
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_tw_s(v[s], w1, w2, w4, w8, sg);  // X[t + 4r] = v[r]
  }
}

// Asynchronous copy of one complex number (8 or 16 bytes) into shared memory.
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* dst, const C* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(C) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

// Slot of packed potential entry k in the staging buffer: with dec0 the
// entries U_0c, c = 1..SV-1 (k = 1..SV-1) vanish and are not staged.
template <int SV>
__device__ __forceinline__ int staged_slot(int k, int dec0) {
  return (SV > 2 && dec0 && k >= SV) ? k - (SV - 1) : k;
}

// Copies (cp.async) this thread's entries of the packed unitary U into its
// own slots of `us`, [slot][m][thread]: every thread later reads back only
// what it copied, so no barrier is involved.
template <int L, int SV, int NT, typename C>
__device__ __forceinline__ void stage_potential(C* us, const C* __restrict__ U, long long P, int t, int sh, int dec0,
                                                int tid) {
  constexpr int TPL = RegPlan<L>::TPL, VPT = RegPlan<L>::VPT, NP = SV * (SV + 1) / 2;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (SV > 2 && dec0 && k >= 1 && k < SV) continue;  // U_0c = 0: not loaded
    const int sl = staged_slot<SV>(k, dec0);
#pragma unroll
    for (int m = 0; m < VPT; ++m)
      cp_async_elem(&us[(sl * VPT + m) * NT + tid], &U[(size_t)k * P + ((unsigned)(t + TPL * m) << sh)]);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ unsigned low_bits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned low_bits(double x) { return (unsigned)__double2loint(x); }

// The potential step at this thread's points, as apply_potential: the packed
// unitary's entries of each point (staged in `us` by stage_potential) and
// matvec_sym on the SV values.  Returns 0, computed from every entry read, so
// that copies reusing the slots can be made to issue after those reads.
template <int L, int SV, int NT, typename C>
__device__ __forceinline__ unsigned potential_reg(C (&v)[SV][RegPlan<L>::VPT], const C* us, int dec0, int tid) {
  constexpr int VPT = RegPlan<L>::VPT, NP = SV * (SV + 1) / 2;
  unsigned tok = 0;
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // this thread's copies landed
#pragma unroll
  for (int m = 0; m < VPT; ++m) {
    C x[SV], y[SV], u[NP];
#pragma unroll
    for (int s = 0; s < SV; ++s) x[s] = v[s][m];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (SV > 2 && dec0 && k >= 1 && k < SV) {  // U_0c = 0: not loaded
        u[k] = mkc((RealT<C>)0, (RealT<C>)0);
        continue;
      }
      u[k] = us[(staged_slot<SV>(k, dec0) * VPT + m) * NT + tid];
      tok |= low_bits(u[k].x);
    }
    matvec_sym<SV>(u, x, y, dec0);
#pragma unroll
    for (int s = 0; s < SV; ++s) v[s][m] = y[s];
  }
  unsigned zero;
  asm volatile("and.b32 %0, %1, 0;" : "=r"(zero) : "r"(tok));
  return zero;
}

// Registers the variant may spend on the amplitudes a thread holds.
template <int L, int SV, typename C>
__host__ __device__ constexpr bool reg_fits() {
  return SV * RegPlan<L>::VPT * (int)(sizeof(C) / 4) <= 96;
}

// The kinetic phase(s) at this thread's elements, as apply_kinetic: from a
// table of the grid (element at line + off(m)) or of this axis alone
// (element t + TPL m, PASS_TAX).
template <int L, int SV, typename C>
__device__ __forceinline__ void kinetic_reg(C (&v)[SV][RegPlan<L>::VPT], const PassArgs& a, long long line, int sh,
                                            int t) {
  constexpr int TPL = RegPlan<L>::TPL, VPT = RegPlan<L>::VPT;
  const bool tax = (a.flags & PASS_TAX) != 0;
  const long long tline = tax ? 0 : line;
  const int tsh = tax ? 0 : sh;
  const C* tau = reinterpret_cast<const C*>(a.tau) + tline;
#pragma unroll
  for (int m = 0; m < VPT; ++m) {
    const C ph = __ldg(&tau[(unsigned)(t + TPL * m) << tsh]);
#pragma unroll
    for (int s = 0; s < SV; ++s) v[s][m] = cmul(v[s][m], ph);
  }
  if (a.tau2) {
    const C* tau2 = reinterpret_cast<const C*>(a.tau2) + tline;
#pragma unroll
    for (int m = 0; m < VPT; ++m) {
      C ph = __ldg(&tau2[(unsigned)(t + TPL * m) << tsh]);
      if ((RealT<C>)a.tau2_scale != (RealT<C>)1) ph = cscale(ph, (RealT<C>)a.tau2_scale);
#pragma unroll
      for (int s = 0; s < SV; ++s) v[s][m] = cmul(v[s][m], ph);
    }
  }
}

// One tile: reg_lines<L, SV>() line positions of SV surfaces of one job,
// starting at its surface s_first.  Optional inverse FFT, potential step(s),
// forward FFT, kinetic phase(s) and inverse FFT, as the tile kernel; no
// split-axis twiddles.  With `pot` the potential tables' packed entries
// u0 .. u0 + SV(SV+1)/2 - 1 of each point form the SV x SV unitary (dec0:
// its first row and column vanish, see matvec_sym).  Shared memory: the
// exchange buffer (G lines), then the staging buffer of the unitary's
// entries.  The potential tables do not change during a propagation, so their
// copies are issued before the wait for the previous pass and land while
// this tile's wavefunction loads and inverse FFT run.
template <int L, int SV, bool CONTIG, typename C>
__device__ __forceinline__ void reg_tile(const PassArgs& a, const TileJob& tj, int s_first, int u0, int dec0,
                                         bool pot, C* sm) {
  constexpr int TPL = RegPlan<L>::TPL, VPT = RegPlan<L>::VPT, G = reg_lines<L, SV>(), NT = reg_threads<SV>();
  constexpr bool WL = CONTIG;  // a line's threads in one warp (contiguous lines)
  using LY = RegLayout<L, WL>;
  const int tid = threadIdx.x;
  // contiguous lines: a line's TPL threads are consecutive lanes (a warp
  // barrier in the exchange); strided lines: consecutive lanes take
  // consecutive lines (coalesced; a block barrier).  A mapping of strided
  // lines with a line's threads in one warp (rows of 32 bytes per access)
  // measured 1.45x slower on 128-point FP32 lines.
  const int g = WL ? tid / TPL : tid % G;
  const int t = WL ? tid % TPL : tid / G;
  const TileGeom tg = make_geom(tj.tile, a);
  // Element m of this thread's part of the line sits at line + off(m); the
  // offsets within a line are below P <= 2^30 and kept in 32 bits.
  long long line;
  int sh;
  if (CONTIG) {  // lines o0 + g, contiguous
    line = (tg.o0 + g) * (long long)L;
    sh = 0;
  } else {  // one outer row: lines at inner positions i0 + g
    line = ((tg.o0 * L) << a.stride_log2) + tg.i0 + g;
    sh = a.stride_log2;
  }
  C* ln = sm + g * LY::LS;
  C* us = sm + G * LY::LS;
  const size_t uoff = (size_t)tj.job * a.u_batch_stride + (size_t)u0 * a.P + line;
  if (pot) stage_potential<L, SV, NT>(us, reinterpret_cast<const C*>(a.U1) + uoff, a.P, t, sh, dec0, tid);
  C* psi = reinterpret_cast<C*>(a.psi) + (size_t)(tj.surf0 + s_first) * a.P + line;
  const C* tw = reinterpret_cast<const C*>(a.tw);
  C v[SV][VPT];
  pdl_wait();  // psi is the previous pass's output
#pragma unroll
  for (int s = 0; s < SV; ++s) {
#pragma unroll
    for (int m = 0; m < VPT; ++m) v[s][m] = psi[(size_t)s * a.P + ((unsigned)(t + TPL * m) << sh)];
  }
  pdl_trigger();
  const int f = a.flags;
  auto potential = [&]() {
    const unsigned after = potential_reg<L, SV, NT>(v, us, dec0, tid);
    if (a.U2) {  // the second table goes through the same slots of this thread, copied once they are read
      stage_potential<L, SV, NT>(us + after, reinterpret_cast<const C*>(a.U2) + uoff, a.P, t, sh, dec0, tid);
      potential_reg<L, SV, NT>(v, us, dec0, tid);
    }
  };
  if constexpr (SV == 1) {  // one surface: the steps unrolled (fewer registers)
    if (f & PASS_INV_FIRST) fft_reg<L, SV, WL>(v, ln, t, tw, (RealT<C>)-1);
    if (pot) potential();
    if (f & PASS_FWD) fft_reg<L, SV, WL>(v, ln, t, tw, (RealT<C>)1);
    if ((f & PASS_FWD) && (f & PASS_T)) kinetic_reg<L, SV>(v, a, line, sh, t);
    if ((f & PASS_FWD) && (f & PASS_T)) fft_reg<L, SV, WL>(v, ln, t, tw, (RealT<C>)-1);
  } else {
    // With several surfaces the steps run as one loop whose body holds one
    // FFT (the sign a runtime value), so that the straight-line code -- run
    // once per tile -- stays small: unrolled, the three-surface body's
    // instruction fetches stalled its warps as often as its memory loads did.
#pragma unroll 1
    for (int j = 0; j < 5; ++j) {
      const bool fft = (j == 0 && (f & PASS_INV_FIRST)) || (j == 2 && (f & PASS_FWD)) ||
                       (j == 4 && (f & PASS_FWD) && (f & PASS_T));
      if (fft) {
        fft_reg<L, SV, WL>(v, ln, t, tw, j == 2 ? (RealT<C>)1 : (RealT<C>)-1);
      } else if (j == 1 && pot) {
        potential();
      } else if (j == 3 && (f & PASS_FWD) && (f & PASS_T)) {
        kinetic_reg<L, SV>(v, a, line, sh, t);
      }
    }
  }
  // With several surfaces the store addresses are recomputed from an opaque
  // copy of the shift: kept from the loads, the SV x VPT 64-bit addresses of
  // a strided tile would hold as many registers as its amplitudes.
  int sh_st = sh;
  if (SV > 1) asm volatile("mov.b32 %0, %1;" : "=r"(sh_st) : "r"(sh));
#pragma unroll
  for (int s = 0; s < SV; ++s) {
#pragma unroll
    for (int m = 0; m < VPT; ++m) psi[(size_t)s * a.P + ((unsigned)(t + TPL * m) << sh_st)] = v[s][m];
  }
}

// One tile of reg_lines<L, SV>() line positions of the SV staged surfaces
// (SV = 1: one surface; SV = S: all surfaces of one job).
template <int L, int SV, bool CONTIG, typename C>
__global__ void __launch_bounds__(reg_threads<SV>(), SV == 1 ? 4 : 2) axis_pass_reg_kernel(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const TileJob tj = split_tile(blockIdx.x, SV, a);
  // the host sets U1/U2 only for passes that stage all S surfaces
  reg_tile<L, SV, CONTIG>(a, tj, 0, 0, a.dec0, SV > 1 && a.U1, reinterpret_cast<C*>(smraw));
}

// Passes that stage all S > 2 surfaces with surface 0 decoupled (dec0: the
// unitary is block diagonal, U_00 and the S-1 x S-1 block of the others):
// every tile is two CTAs, one transforming surface 0 with the diagonal entry
// U_00 (packed entry 0), one surfaces 1..S-1 with the block (packed entries
// S .. S(S+1)/2 - 1, in the packed order of an S-1 matrix).  The products are
// those of matvec_sym with dec0, bit for bit, and each CTA holds the
// amplitudes of fewer surfaces, so more CTAs share an SM.  The first half of
// the grid takes the blocks (the longer CTAs, started first), the second half
// surface 0, so that an SM mostly runs one role's code at a time.
template <int L, int S, bool CONTIG, typename C>
__global__ void __launch_bounds__(reg_threads<S>(), 3) axis_pass_reg_split_kernel(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const unsigned half = gridDim.x >> 1;
  const bool block = blockIdx.x < half;
  const TileJob tj = split_tile(block ? blockIdx.x : blockIdx.x - half, S, a);
  C* sm = reinterpret_cast<C*>(smraw);
  if (!block)
    reg_tile<L, 1, CONTIG>(a, tj, 0, 0, 0, a.U1 != nullptr, sm);
  else
    reg_tile<L, S - 1, CONTIG>(a, tj, 1, S, 0, a.U1 != nullptr, sm);
}

// Shared memory of a tile: the exchange buffer and, with a potential step,
// the staging buffer of the np_staged packed entries the pass loads.
template <int L, int SV>
inline size_t reg_smem_bytes(bool wl, bool fp32, int np_staged) {
  const int LS = wl ? RegLayout<L, true>::LS : RegLayout<L, false>::LS;
  const size_t esz = fp32 ? 8 : 16;
  return ((size_t)reg_lines<L, SV>() * LS + (size_t)np_staged * RegPlan<L>::VPT * reg_threads<SV>()) * esz;
}

}  // namespace dso
