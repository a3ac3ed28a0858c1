// axis_pass_reg.cuh -- register-resident axis pass for lines of 32, 64 and
// 128 points: the FFT-only passes and the fused kinetic pass [F T I].
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
// two kernels give bitwise the same results:
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

// Threads per CTA: 256 for one staged surface; 128 for S surfaces, whose
// amplitudes take most of a thread's registers, so that two CTAs share an
// SM and one's loads overlap the other's FFTs.
template <int SV>
__host__ __device__ constexpr int reg_threads() {
  return SV == 1 ? 256 : 128;
}

// Line positions per CTA (the tile line count G the host must use).
template <int L, int SV>
__host__ __device__ constexpr int reg_lines() {
  return reg_threads<SV>() / RegPlan<L>::TPL;
}

// Exchange buffer of one line: element n at n + (n >> plog), lines LS apart.
template <int L, bool CONTIG>
struct RegLayout {
  static constexpr int plog = CONTIG ? (L == 128 ? 4 : 3) : 31;
  static constexpr int LS = CONTIG ? L + (L >> plog) : L + 1;
  __device__ __forceinline__ static int pos(int n) { return plog < 31 ? n + (n >> plog) : n; }
};

template <bool CONTIG>
__device__ __forceinline__ void reg_sync() {
  if (CONTIG) __syncwarp(); else __syncthreads();
}

// Inverse or forward FFT of SV lines (one per staged surface) at this
// thread's line position.  The register stages of all SV lines share the
// twiddle loads; the lines go through the one exchange buffer (G lines) in
// turn.
template <int L, int SV, bool INV, bool CONTIG, typename C>
__device__ __forceinline__ void fft_reg(C (&v)[SV][RegPlan<L>::VPT], C* ln, int t, const C* __restrict__ tw) {
  using LY = RegLayout<L, CONTIG>;
  C w1, w2, w4, w8;
  if constexpr (L == 64) {
#pragma unroll
    for (int s = 0; s < SV; ++s) dftR<8, INV>(v[s]);  // stage 1 (Ls = 1): j = t on x[t + 8r]; y[8t + r]
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      reg_sync<CONTIG>();  // earlier readers of the buffer are done
#pragma unroll
      for (int r = 0; r < 8; ++r) ln[LY::pos(8 * t + r)] = v[s][r];
      reg_sync<CONTIG>();
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][r] = ln[LY::pos(t + 8 * r)];
    }
    load_tw8<64>(tw, t, w1, w2, w4, w8);  // stage 2 (Ls = 8): butterfly k = t
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_tw<INV>(v[s], w1, w2, w4, w8);  // X[t + 8r] = v[r]
  } else if constexpr (L == 128) {
#pragma unroll
    for (int s = 0; s < SV; ++s) {
#pragma unroll
      for (int r = 0; r < 8; ++r) dft2<INV>(v[s][r], v[s][r + 8]);  // stage 1: j = t + 8r -> y[2j], y[2j + 1]
    }
    load_tw8<128>(tw, 0, w1, w2, w4, w8);  // stage 2 (Ls = 2): j = 2t (k = 0), inputs y[2t + 16r]
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_tw<INV>(&v[s][0], w1, w2, w4, w8);
    load_tw8<128>(tw, 8, w1, w2, w4, w8);  // j = 2t + 1 (k = 1), inputs y[2t + 1 + 16r]
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_tw<INV>(&v[s][8], w1, w2, w4, w8);
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      reg_sync<CONTIG>();
#pragma unroll
      for (int r = 0; r < 8; ++r) {  // z[16t + 2r] from j = 2t, z[16t + 2r + 1] from j = 2t + 1
        ln[LY::pos(16 * t + 2 * r)] = v[s][r];
        ln[LY::pos(16 * t + 2 * r + 1)] = v[s][8 + r];
      }
      reg_sync<CONTIG>();
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
      dft8_tw<INV>(a, w1, w2, w4, w8);  // X[t + 16r]
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][2 * r] = a[r];
    }
    load_tw8<128>(tw, t + 8, w1, w2, w4, w8);  // k = t + 8
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      C b[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) b[r] = v[s][2 * r + 1];
      dft8_tw<INV>(b, w1, w2, w4, w8);  // X[t + 8 + 16r]
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][2 * r + 1] = b[r];
    }
  } else {  // L == 32
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      dft4<INV>(v[s][0], v[s][2], v[s][4], v[s][6]);  // stage 1: j = t on x[t + 8r]; y[4t + r]
      dft4<INV>(v[s][1], v[s][3], v[s][5], v[s][7]);  // j = t + 4 on x[t + 4 + 8r]; y[4t + 16 + r]
    }
#pragma unroll
    for (int s = 0; s < SV; ++s) {
      reg_sync<CONTIG>();
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        ln[LY::pos(4 * t + r)] = v[s][2 * r];
        ln[LY::pos(4 * t + 16 + r)] = v[s][2 * r + 1];
      }
      reg_sync<CONTIG>();
#pragma unroll
      for (int r = 0; r < 8; ++r) v[s][r] = ln[LY::pos(t + 4 * r)];
    }
    load_tw8<32>(tw, t, w1, w2, w4, w8);  // stage 2 (Ls = 4): butterfly k = t
#pragma unroll
    for (int s = 0; s < SV; ++s) dft8_tw<INV>(v[s], w1, w2, w4, w8);  // X[t + 4r] = v[r]
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

// One tile: reg_lines<L, SV>() line positions of the SV staged surfaces (SV = 1:
// one surface; SV = S: all surfaces of one job).  Optional inverse FFT,
// potential step(s), forward FFT, kinetic phase(s) and inverse FFT, as the
// tile kernel; no split-axis twiddles.  Shared memory: the exchange buffer
// (G lines), then, for a pass with a potential step, the staging buffer of
// the unitary's entries.  The potential tables do not change during a
// propagation, so their copies are issued before the wait for the previous
// pass and land while this tile's wavefunction loads and inverse FFT run.
template <int L, int SV, bool CONTIG, typename C>
__global__ void __launch_bounds__(reg_threads<SV>(), 2) axis_pass_reg_kernel(PassArgs a) {
  constexpr int TPL = RegPlan<L>::TPL, VPT = RegPlan<L>::VPT, G = reg_lines<L, SV>(), NT = reg_threads<SV>();
  using LY = RegLayout<L, CONTIG>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int tid = threadIdx.x;
  // contiguous lines: a line's TPL threads are consecutive lanes; strided
  // lines: consecutive lanes take consecutive lines (coalesced)
  const int g = CONTIG ? tid / TPL : tid % G;
  const int t = CONTIG ? tid % TPL : tid / G;
  const TileJob tj = split_tile(blockIdx.x, SV, a);
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
  const size_t uoff = (size_t)tj.job * a.u_batch_stride + line;
  if (SV > 1 && a.U1)  // the host sets U1/U2 only for passes that stage all S surfaces
    stage_potential<L, SV, NT>(us, reinterpret_cast<const C*>(a.U1) + uoff, a.P, t, sh, a.dec0, tid);
  C* psi = reinterpret_cast<C*>(a.psi) + (size_t)tj.surf0 * a.P + line;
  const C* tw = reinterpret_cast<const C*>(a.tw);
  C v[SV][VPT];
  pdl_wait();  // psi is the previous pass's output
#pragma unroll
  for (int s = 0; s < SV; ++s) {
#pragma unroll
    for (int m = 0; m < VPT; ++m) v[s][m] = psi[(size_t)s * a.P + ((unsigned)(t + TPL * m) << sh)];
  }
  pdl_trigger();
  if (a.flags & PASS_INV_FIRST) fft_reg<L, SV, true, CONTIG>(v, ln, t, tw);
  if (SV > 1 && a.U1) {
    const unsigned after = potential_reg<L, SV, NT>(v, us, a.dec0, tid);
    if (a.U2) {  // the second table goes through the same slots of this thread, copied once they are read
      stage_potential<L, SV, NT>(us + after, reinterpret_cast<const C*>(a.U2) + uoff, a.P, t, sh, a.dec0, tid);
      potential_reg<L, SV, NT>(v, us, a.dec0, tid);
    }
  }
  if (a.flags & PASS_FWD) {
    fft_reg<L, SV, false, CONTIG>(v, ln, t, tw);
    if (a.flags & PASS_T) {  // the kinetic phase(s), as apply_kinetic, then the inverse FFT
      const C* tau = reinterpret_cast<const C*>(a.tau) + line;
#pragma unroll
      for (int m = 0; m < VPT; ++m) {
        const C ph = __ldg(&tau[(unsigned)(t + TPL * m) << sh]);
#pragma unroll
        for (int s = 0; s < SV; ++s) v[s][m] = cmul(v[s][m], ph);
      }
      if (a.tau2) {
        const C* tau2 = reinterpret_cast<const C*>(a.tau2) + line;
#pragma unroll
        for (int m = 0; m < VPT; ++m) {
          C ph = __ldg(&tau2[(unsigned)(t + TPL * m) << sh]);
          if ((RealT<C>)a.tau2_scale != (RealT<C>)1) ph = cscale(ph, (RealT<C>)a.tau2_scale);
#pragma unroll
          for (int s = 0; s < SV; ++s) v[s][m] = cmul(v[s][m], ph);
        }
      }
      fft_reg<L, SV, true, CONTIG>(v, ln, t, tw);
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

// Shared memory of a tile: the exchange buffer and, with a potential step,
// the staging buffer of the np_staged packed entries the pass loads.
template <int L, int SV>
inline size_t reg_smem_bytes(bool contig, bool fp32, int np_staged) {
  const int LS = contig ? RegLayout<L, true>::LS : RegLayout<L, false>::LS;
  const size_t esz = fp32 ? 8 : 16;
  return ((size_t)reg_lines<L, SV>() * LS + (size_t)np_staged * RegPlan<L>::VPT * reg_threads<SV>()) * esz;
}

}  // namespace dso
