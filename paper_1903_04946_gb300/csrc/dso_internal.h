// dso_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pass_args.h"

#include <cuda.h>

#define DSO_OBS_COLS 6  // up to 4 populations, <V>, <T>

namespace dso {

// Virtual axes of the passes.  A pass transforms whole lines of one axis held
// in shared memory, which bounds a line's length (4096 points, and S x 8192
// for the potential pass that stages all S surfaces of an axis-0 line).  A
// longer grid axis of n points is viewed as two axes, index i1 * n2 + i2 with
// n = n1 * n2, and transformed in four steps: FFTs of length n1 along i1, a
// twiddle multiplication by w_n^(k1 i2), FFTs of length n2 along i2 (the
// Cooley-Tukey splitting behind the FFTs of Sec. II G).  Frequency
// k1 + n1 k2 then sits at storage position (k1, k2): the momentum
// representation is stored permuted along a split axis, which only the
// kinetic phases and <T> need to know.
#define DSO_MAX_VAXES 6
#define DSO_MAX_LINE 4096  // longest line of a pass
#define DSO_MAX_GRID_AXIS (1 << 22)
struct VLayout {
  int Dv;                       // virtual axes (row-major, last contiguous)
  int64_t nv[DSO_MAX_VAXES];    // their lengths
  int part[DSO_MAX_VAXES];      // 0: a whole grid axis, 1: first factor (n1) of a split one, 2: second (n2)
  int D;                        // grid axes
  int64_t n[3];                 // grid axis lengths
};

// Momentum index along every grid axis of storage position g of the
// momentum representation (after forward FFTs along every virtual axis).
__host__ __device__ inline void momentum_indices(const VLayout& v, long long g, int64_t (&k)[3]) {
  int64_t kv[DSO_MAX_VAXES];
  for (int a = v.Dv - 1; a >= 0; --a) {
    kv[a] = g & (v.nv[a] - 1);  // lengths are powers of two
    g /= v.nv[a];
  }
  int d = 0;
  for (int a = 0; a < v.Dv; ++a) {
    if (v.part[a] == 1) {
      k[d++] = kv[a] + v.nv[a] * kv[a + 1];
      ++a;
    } else {
      k[d++] = kv[a];
    }
  }
}

// Pruned splitting coefficients of one composed scheme (Sec. II D-F).
struct Coeffs {
  std::vector<double> a, b;          // a~ (N_B + 1 entries), b~ (N_B entries)
  std::vector<int> ia, ib;           // 0-based indices into a_unq / b_unq
  std::vector<double> a_unq, b_unq;  // unique values, first-occurrence order
};

// order in {2,4,...}, scheme 0 = triple jump, 1 = Suzuki fractal.
Coeffs build_coefficients(int order, int scheme);
// Pruned coefficients of the composition of second-order steps with the
// elementary coefficients g (time order, symmetric).
Coeffs coefficients_from_gammas(const std::vector<long double>& g);

// Axis-pass launch: L = line length, SV = surfaces staged per tile.
bool axis_pass_supported(int L, int SV);
int axis_pass_max_tile_lines(int L, int SV);  // largest G allowed by the thread bound
struct TmaMaps;
// variant 0: one CTA per tile (axis_pass.cuh); variant 1: persistent CTAs
// with a tile queue and cp.async prefetch (axis_pass_pq.cuh), which needs
// `queue` (two zeroed unsigned counters owned by the caller's context);
// variant 2: one CTA per tile with TMA tile and table movement
// (axis_pass_tma.cuh), which needs the tensor maps in `maps`; variant 3:
// persistent CTAs with double-buffered TMA movement (axis_pass_tma.cuh),
// which needs both `queue` and `maps`; variant 4: lines of 32..128 points
// held in registers (axis_pass_reg.cuh), axis_pass_reg_lines(L, SV) lines
// per tile, where the amplitudes of the SV surfaces fit a thread's registers.
cudaError_t launch_axis_pass(int L, int SV, int variant, const PassArgs& args, long long ntiles, unsigned* queue,
                             const TmaMaps* maps, cudaStream_t st);
bool axis_pass_pq_supported(int L, int SV, int G);
bool axis_pass_tma_supported(int L, int SV, int G);
bool axis_pass_tmap_supported(int L, int SV, int G);
// tile lines of the register-resident variant, 0 where it does not apply
int axis_pass_reg_lines(int L, int SV);
// the register-resident variant takes lines of L points along an axis of
// `stride` with SV surfaces staged (dec0: surface 0 decoupled)
bool axis_pass_reg_supported(int L, int SV, bool fp32, long long stride, bool dec0);
// Plane pass (axis_pass_plane.cuh) over axes D-2 (LA points, stride LB)
// and D-1 (LB points) of a 3-D grid, one cluster of CTAs per LA x LB plane of
// one surface: with PASS_TAX [F T I] along each axis in turn (per-axis
// phases), without it [F_a | F_b T I_b | I_a] (the grid's phase); `args` is
// the axis D-2 pass's with PASS_PLANE and tw2 the twiddles of LB points.
bool axis_pass_plane_supported(int LA, int LB, bool fp32);
cudaError_t launch_axis_pass_plane(int LA, int LB, const PassArgs& args, long long nplanes, cudaStream_t st);
// per-SV launchers (one translation unit each)
cudaError_t launch_axis_pass_sv1(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);
cudaError_t launch_axis_pass_sv2(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);
cudaError_t launch_axis_pass_sv3(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);
cudaError_t launch_axis_pass_sv4(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);

// Batch slots (batch.cu): one pass of one job, with the tile line count the
// batch chose for it, and a segment of the launch's work list (one pass of
// one job; its tiles are items item0 .. item0 + ntiles - 1; `prev` is the
// segment of the job's previous pass in this launch, or -1).
struct BatchPass {
  PassArgs a;
  int L, log2L, SV;
  long long ntiles;
};
struct BatchSeg {
  long long item0;
  int pass;  // index into the launch's BatchPass table
  int prev;
};
size_t batch_tile_smem(int L, int SV, int G, int Wi, bool fp32);
int batch_max_tile_amplitudes();  // SV * G * L of one tile of the batch kernel
cudaError_t launch_batch_worklist(bool fp32, const BatchSeg* segs, int nseg, const BatchPass* passes, long long total,
                                  unsigned long long* head, unsigned* done, int* err, size_t smem, cudaStream_t st);

// Operator tables (tables.cu).
// Twiddles w_m = exp(-2 pi i m / L), m = 0..L-1, in the tangent form the
// FFT stages use: (cos, sin / cos), computed on the host in long double and
// rounded once (a zero cosine is replaced by 2^-500, or 2^-60 for the FP32
// table, so that the tangent stays finite).
std::vector<double2> host_twiddles(int L, bool fp32);
// Kinetic phase coefficients: the phase of unique b (nb of them) at momentum
// index kk_d (folded to [-n_d/2, n_d/2)) is sum_d C[u][d] kk_d^2 with
// C = -b dt (2 pi / extent_d)^2 / (2 m_d), computed on the host in long double
// and passed as an unevaluated sum hi + lo of two doubles per (u, d):
// coef[(u * D + d) * 2 + {0, 1}].
std::vector<double> host_kinetic_coefficients(int D, const double* qmin, const double* qmax, const double* mass,
                                              const std::vector<double>& b_unq, double dt);
// tau[u][g] = exp(i phase_u(k(g))) / P at every storage position g of the
// momentum representation (momentum_indices), the phase summed in
// double-double and exponentiated with one sincos plus a first-order
// correction for the low part.  Output is double2, or float2 rounded once.
cudaError_t launch_kinetic_tables(void* tau, bool fp32, const double* coef, int nb, const VLayout& v, long long P,
                                  cudaStream_t st);
// Separable kinetic tables: tau[u][off_d + k], the phase of axis d alone at
// momentum index k (natural FFT order) for every unique coefficient, 1/n_d
// folded in; off_d = n_0 + .. + n_{d-1}.
cudaError_t launch_axis_kinetic_tables(void* tau, bool fp32, const double* coef, int nb, int D, const int64_t* n,
                                       cudaStream_t st);
// Twiddles of a split axis of n = n1 * n2 points: xtw[k1 * n2 + i2] =
// exp(-2 pi i (k1 i2 mod n) / n) (sincospi of an exact argument), double2
// or rounded once to float2.
cudaError_t launch_split_twiddles(void* xtw, bool fp32, int64_t n1, int64_t n2, cudaStream_t st);
// U[u][k][g] = exp(-i a_u dt V(q_g)) packed upper, for every unique a.
// FP64 throughout; stored as double2, or rounded once to float2 when fp32.
cudaError_t launch_potential_tables(void* U, bool fp32, const double* V, const double* tau_a, int na, int S,
                                    long long P, cudaStream_t st);
// Operators built per action (dso_set_operator_mode): the coefficient-free
// part of every point's U -- for S = 2 the mean, half difference and
// coupling of V and the rotation rate, for S >= 3 the eigenvectors and
// eigenvalues of V -- stored once as [eig_cache_doubles(S)][P] doubles, and
// U for the one coefficient tau_a[0] assembled from it into U ([NP][P]) with
// potential_table_kernel's arithmetic (bitwise its table).
int eig_cache_doubles(int S);
cudaError_t launch_eig_cache(double* E, const double* V, int S, long long P, cudaStream_t st);
cudaError_t launch_unitary_from_cache(void* U, bool fp32, const double* E, const double* tau_a, int S, long long P,
                                      cudaStream_t st);

// Observables (observables.cu): per-block partial sums then a fixed-order
// final reduction.  `spec` holds |psi~|^2-weighting per axis (p^2 / 2m).
struct ObsArgs {
  const void* psi;        // position representation [S][P] (double2, or float2 when fp32)
  const void* psik;       // momentum representation [S][P] (unnormalised FFT, storage order of vl)
  const double* V;        // packed potential [S(S+1)/2][P]
  const double* Tax;      // concatenated per-axis p_k^2/(2 m_d), natural momentum order
  VLayout vl;             // storage order of psik
  int S;
  long long P;
  int fp32;
};
int obs_partial_blocks();
cudaError_t launch_observables(const ObsArgs& a, double* partials, double* out, cudaStream_t st);

}  // namespace dso
