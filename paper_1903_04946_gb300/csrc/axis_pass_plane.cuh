// axis_pass_plane.cuh -- the separable kinetic step's passes over the last
// two axes of a 3-D grid in one launch: [F_a T_a I_a] then [F_b T_b I_b] on
// every LA x LB plane, axis a = D-2 (LA points, stride LB) and axis b = D-1
// (LB points, contiguous).
//
// The kinetic propagator of Eq. (diab_mol_ham)'s separable kinetic energy is
// a product of one phase per axis, each diagonal in its own momentum index,
// so the kinetic step factors into one [F_d T_d I_d] per axis (Sec. II G's
// FFTs taken one axis at a time).  The line passes of axis_pass_reg.cuh do
// that with one round trip of the wavefunction through global memory per
// axis; here the two last axes share one round trip.  A plane of one surface
// is one thread-block cluster of K CTAs:
//   phase A: CTA c loads the columns (lines along a) at b = c WB .. c WB +
//     WB - 1, transforms them in registers (the register-resident FFT, phase
//     and inverse FFT of axis_pass_reg.cuh, strided mapping) and stores each
//     amplitude into the shared memory of the CTA that owns its row
//     (distributed shared memory, rows of WA = LA / K per CTA);
//   cluster barrier;
//   phase B: CTA c reads its WA rows (lines along b) from its own shared
//     memory, transforms them (contiguous mapping) and stores them.
// Every FFT, phase multiplication and inverse FFT is the line passes' own,
// with the same tables and operands in the same order, so the results are
// bitwise those of the two line passes (and of the tile kernel).
#pragma once

#include "axis_pass_reg.cuh"

namespace dso {

template <int LA, int LB, typename C>
struct PlaneGeom {
  static constexpr int GA = reg_lines<LA, 1>();  // columns per phase-A tile
  static constexpr int GB = reg_lines<LB, 1>();  // rows per phase-B tile
  static constexpr int K0 = (LA / GB < LB / GA) ? LA / GB : LB / GA;
  static constexpr int K = K0 > 8 ? 8 : (K0 < 1 ? 1 : K0);  // CTAs per plane (portable cluster size)
  static constexpr int WB = LB / K;                          // columns of a CTA in phase A
  static constexpr int WA = LA / K;                          // rows of a CTA in phase B
  static constexpr int NA = WB / GA, NB = WA / GB;           // tiles of a CTA per phase
  // rows of the row buffer RS elements apart: 64 bytes of padding, so that
  // the four rows a warp reads in phase B fall in two bank-disjoint pairs
  static constexpr int RS = LB + 64 / (int)sizeof(C);
  static constexpr int XA = GA * RegLayout<LA, false>::LS, XB = GB * RegLayout<LB, true>::LS;
  static constexpr int XE = XA > XB ? XA : XB;  // exchange buffer (elements)
  static constexpr int RE = WA * RS;            // row buffer (elements)
  static_assert(K * WB == LB && K * WA == LA && NA * GA == WB && NB * GB == WA, "plane split");
};

template <int LA, int LB, typename C>
__host__ __device__ constexpr size_t plane_smem_bytes() {
  return (size_t)(PlaneGeom<LA, LB, C>::XE + PlaneGeom<LA, LB, C>::RE) * sizeof(C);
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Cluster barrier halves: arrive (release: this thread's earlier shared
// memory writes, local or remote, become visible to the waiters; relaxed:
// no ordering, only "started") and wait (acquire).
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Store one complex number at shared address `sa` of this CTA, mapped into
// the shared memory of cluster CTA `rank`.
__device__ __forceinline__ void st_cluster(unsigned sa, unsigned rank, float2 v) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sa), "r"(rank));
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(ra), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(unsigned sa, unsigned rank, double2 v) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sa), "r"(rank));
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(ra), "d"(v.x), "d"(v.y) : "memory");
}

// One plane of one surface per cluster: blockIdx.x / K is the plane (over
// all jobs, surfaces and outer indices: planes are LA LB elements apart),
// the cluster rank the CTA's share.  a.tau (a.tau2) is axis a's phase table,
// axis b's follows it (LA entries on); a.tau2_scale is LA.
// Five CTAs per SM for FP32 (96 registers, no spills: 41.7 against 43.4 us
// at four on 128 x 128 planes, 44.7 at six), four for FP64.
template <int LA, int LB, typename C>
__global__ void __launch_bounds__(128, sizeof(C) == 8 ? 5 : 4) axis_pass_plane_kernel(PassArgs a) {
  using PG = PlaneGeom<LA, LB, C>;
  constexpr int TPA = RegPlan<LA>::TPL, VA = RegPlan<LA>::VPT;
  constexpr int TPB = RegPlan<LB>::TPL, VB = RegPlan<LB>::VPT;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* X = reinterpret_cast<C*>(smraw);  // FFT exchange buffer
  C* R = X + PG::XE;                   // this CTA's rows [WA][RS], written by the whole cluster
  const int tid = threadIdx.x;
  const unsigned rank = cluster_rank();
  // every CTA of the cluster has started before any writes into another's
  // shared memory (the wait sits just before the first remote store)
  cluster_arrive_relaxed();
  C* psi = reinterpret_cast<C*>(a.psi) + (size_t)(blockIdx.x / PG::K) * (LA * LB);
  const C* tw_a = reinterpret_cast<const C*>(a.tw);
  const C* tw_b = reinterpret_cast<const C*>(a.tw2);  // axis b's twiddles
  PassArgs ab = a;  // axis b's phase tables
  ab.tau = reinterpret_cast<const C*>(a.tau) + LA;
  ab.tau2 = a.tau2 ? reinterpret_cast<const C*>(a.tau2) + LA : nullptr;
  ab.tau2_scale = (double)LB;
  const unsigned rbase = (unsigned)__cvta_generic_to_shared(R);
  // phase A: columns, strided mapping (consecutive lanes take consecutive
  // columns, coalesced rows), thread t holds rows t + TPA m
  {
    const int g = tid % PG::GA, t = tid / PG::GA;
    C* ln = X + g * RegLayout<LA, false>::LS;
    pdl_wait();  // psi is the previous pass's output
#pragma unroll 1
    for (int it = 0; it < PG::NA; ++it) {
      const int col = (int)rank * PG::WB + it * PG::GA + g;
      C v[1][VA];
#pragma unroll
      for (int m = 0; m < VA; ++m) v[0][m] = psi[(t + TPA * m) * LB + col];
      if (it == PG::NA - 1) pdl_trigger();
      fft_reg<LA, 1, false>(v, ln, t, tw_a, (RealT<C>)1);
      kinetic_reg<LA, 1>(v, a, 0, 0, t);
      fft_reg<LA, 1, false>(v, ln, t, tw_a, (RealT<C>)-1);
      if (it == 0) cluster_wait();
#pragma unroll
      for (int m = 0; m < VA; ++m) {
        const int row = t + TPA * m;  // owner: CTA row / WA, at its row row % WA
        st_cluster(rbase + (unsigned)(((row % PG::WA) * PG::RS + col) * (int)sizeof(C)), (unsigned)(row / PG::WA),
                   v[0][m]);
      }
    }
  }
  cluster_arrive_release();  // this CTA's stores into the cluster's row buffers are done
  cluster_wait();            // and every other CTA's into this one's
  // phase B: rows, contiguous mapping (a row's TPB threads in one warp)
  {
    const int g = tid / TPB, t = tid % TPB;
    C* ln = X + g * RegLayout<LB, true>::LS;
#pragma unroll 1
    for (int it = 0; it < PG::NB; ++it) {
      const int r = it * PG::GB + g;
      C v[1][VB];
#pragma unroll
      for (int m = 0; m < VB; ++m) v[0][m] = R[r * PG::RS + t + TPB * m];
      fft_reg<LB, 1, true>(v, ln, t, tw_b, (RealT<C>)1);
      kinetic_reg<LB, 1>(v, ab, 0, 0, t);
      fft_reg<LB, 1, true>(v, ln, t, tw_b, (RealT<C>)-1);
      C* out = psi + (size_t)((int)rank * PG::WA + r) * LB;
#pragma unroll
      for (int m = 0; m < VB; ++m) out[t + TPB * m] = v[0][m];
    }
  }
}

// The joint kinetic step's passes over the same planes, [F_a | F_b T I_b |
// I_a]: the forward FFT along a, then along b, the phase of the whole grid
// (one entry per grid point, Sec. II G's joint form), the inverse FFT along
// b and the inverse FFT along a -- the line passes [F_a] [F_b T I_b] [I_a]
// in one launch.  As axis_pass_plane_kernel, with a second exchange: after
// phase B each amplitude goes into the shared memory of the CTA that owns
// its column (a column buffer, WB columns of LA + 1 elements), and phase C
// transforms the columns back and stores them.  The row and column buffers
// are separate, so no CTA writes where another may still read.
template <int LA, int LB, typename C>
struct PlaneJoint {
  using PG = PlaneGeom<LA, LB, C>;
  static constexpr int CS = LA + 1;            // column stride (odd: the strided reads are conflict-free)
  static constexpr int CE = PG::WB * CS;       // column buffer (elements)
};

template <int LA, int LB, typename C>
__host__ __device__ constexpr size_t plane_joint_smem_bytes() {
  return (size_t)(PlaneGeom<LA, LB, C>::XE + PlaneGeom<LA, LB, C>::RE + PlaneJoint<LA, LB, C>::CE) * sizeof(C);
}

// a.tau (a.tau2) is the grid's phase table ([P] per unique coefficient, 1/P
// folded in); a.tau2_scale is P.
template <int LA, int LB, typename C>
__global__ void __launch_bounds__(128, 4) axis_pass_plane_joint_kernel(PassArgs a) {
  using PG = PlaneGeom<LA, LB, C>;
  using PJ = PlaneJoint<LA, LB, C>;
  constexpr int TPA = RegPlan<LA>::TPL, VA = RegPlan<LA>::VPT;
  constexpr int TPB = RegPlan<LB>::TPL, VB = RegPlan<LB>::VPT;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* X = reinterpret_cast<C*>(smraw);  // FFT exchange buffer
  C* R = X + PG::XE;                   // this CTA's rows [WA][RS]
  C* Q = R + PG::RE;                   // this CTA's columns [WB][CS]
  const int tid = threadIdx.x;
  const unsigned rank = cluster_rank();
  cluster_arrive_relaxed();  // waited for before the first remote store
  const long long plane = blockIdx.x / PG::K;
  C* psi = reinterpret_cast<C*>(a.psi) + (size_t)plane * (LA * LB);
  // the plane's first point in the grid-sized phase table (planes of every
  // job and surface share the grid's table)
  const long long tplane = (plane % (a.P / (LA * LB))) * (LA * LB);
  const C* tw_a = reinterpret_cast<const C*>(a.tw);
  const C* tw_b = reinterpret_cast<const C*>(a.tw2);
  const unsigned rbase = (unsigned)__cvta_generic_to_shared(R);
  const unsigned qbase = (unsigned)__cvta_generic_to_shared(Q);
  // phase A: columns, forward FFT along a; each amplitude to its row's owner
  {
    const int g = tid % PG::GA, t = tid / PG::GA;
    C* ln = X + g * RegLayout<LA, false>::LS;
    pdl_wait();  // psi is the previous pass's output
#pragma unroll 1
    for (int it = 0; it < PG::NA; ++it) {
      const int col = (int)rank * PG::WB + it * PG::GA + g;
      C v[1][VA];
#pragma unroll
      for (int m = 0; m < VA; ++m) v[0][m] = psi[(t + TPA * m) * LB + col];
      if (it == PG::NA - 1) pdl_trigger();
      fft_reg<LA, 1, false>(v, ln, t, tw_a, (RealT<C>)1);
      if (it == 0) cluster_wait();
#pragma unroll
      for (int m = 0; m < VA; ++m) {
        const int row = t + TPA * m;
        st_cluster(rbase + (unsigned)(((row % PG::WA) * PG::RS + col) * (int)sizeof(C)), (unsigned)(row / PG::WA),
                   v[0][m]);
      }
    }
  }
  cluster_arrive_release();
  cluster_wait();  // every row complete
  // phase B: rows, forward FFT along b, the phase, inverse FFT along b; each
  // amplitude to its column's owner
  {
    const int g = tid / TPB, t = tid % TPB;
    C* ln = X + g * RegLayout<LB, true>::LS;
#pragma unroll 1
    for (int it = 0; it < PG::NB; ++it) {
      const int r = it * PG::GB + g, row = (int)rank * PG::WA + r;
      C v[1][VB];
#pragma unroll
      for (int m = 0; m < VB; ++m) v[0][m] = R[r * PG::RS + t + TPB * m];
      fft_reg<LB, 1, true>(v, ln, t, tw_b, (RealT<C>)1);
      kinetic_reg<LB, 1>(v, a, tplane + (long long)row * LB, 0, t);
      fft_reg<LB, 1, true>(v, ln, t, tw_b, (RealT<C>)-1);
#pragma unroll
      for (int m = 0; m < VB; ++m) {
        const int col = t + TPB * m;
        st_cluster(qbase + (unsigned)(((col % PG::WB) * PJ::CS + row) * (int)sizeof(C)), (unsigned)(col / PG::WB),
                   v[0][m]);
      }
    }
  }
  cluster_arrive_release();
  cluster_wait();  // every column complete
  // phase C: columns, inverse FFT along a, stored
  {
    const int g = tid % PG::GA, t = tid / PG::GA;
    C* ln = X + g * RegLayout<LA, false>::LS;
#pragma unroll 1
    for (int it = 0; it < PG::NA; ++it) {
      const int cl = it * PG::GA + g, col = (int)rank * PG::WB + cl;
      C v[1][VA];
#pragma unroll
      for (int m = 0; m < VA; ++m) v[0][m] = Q[cl * PJ::CS + t + TPA * m];
      fft_reg<LA, 1, false>(v, ln, t, tw_a, (RealT<C>)-1);
#pragma unroll
      for (int m = 0; m < VA; ++m) psi[(t + TPA * m) * LB + col] = v[0][m];
    }
  }
}

}  // namespace dso
