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
// which needs both `queue` and `maps`.
cudaError_t launch_axis_pass(int L, int SV, int variant, const PassArgs& args, long long ntiles, unsigned* queue,
                             const TmaMaps* maps, cudaStream_t st);
bool axis_pass_pq_supported(int L, int SV, int G);
bool axis_pass_tma_supported(int L, int SV, int G);
bool axis_pass_tmap_supported(int L, int SV, int G);
// per-SV launchers (one translation unit each)
cudaError_t launch_axis_pass_sv1(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);
cudaError_t launch_axis_pass_sv2(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);
cudaError_t launch_axis_pass_sv3(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);
cudaError_t launch_axis_pass_sv4(int L, int variant, const PassArgs& a, long long ntiles, unsigned* queue,
                                 const TmaMaps* maps, cudaStream_t st);

// Operator tables (tables.cu).
// Twiddles w_m = exp(-2 pi i m / L), m = 0..L-1, in the tangent form the
// FFT stages use: (cos, sin / cos), computed on the host in long double and
// rounded once (a zero cosine is replaced by 2^-500, or 2^-60 for the FP32
// table, so that the tangent stays finite).
std::vector<double2> host_twiddles(int L, bool fp32);
// Kinetic phase factors per axis: for each unique b (nb of them), the
// D 1-D factor tables exp(-i b dt p_k^2 / (2 m_d)) concatenated over axes
// (sum n_d entries), 1/P folded into axis 0.  Host long double.
std::vector<double2> host_kinetic_factors(int D, const int64_t* n, const double* qmin, const double* qmax,
                                          const double* mass, const std::vector<double>& b_unq, double dt);
// tau[u][g] = prod_d factor_d(u, k_d(g)) on the device.
// Output is double2, or float2 rounded from the FP64 product when fp32.
cudaError_t launch_kinetic_tables(void* tau, bool fp32, const double2* factors, int nb, int D, const int64_t* n,
                                  long long P, cudaStream_t st);
// U[u][k][g] = exp(-i a_u dt V(q_g)) packed upper, for every unique a.
// FP64 throughout; stored as double2, or rounded once to float2 when fp32.
cudaError_t launch_potential_tables(void* U, bool fp32, const double* V, const double* tau_a, int na, int S,
                                    long long P, cudaStream_t st);

// Observables (observables.cu): per-block partial sums then a fixed-order
// final reduction.  `spec` holds |psi~|^2-weighting per axis (p^2 / 2m).
struct ObsArgs {
  const void* psi;        // position representation [S][P] (double2, or float2 when fp32)
  const void* psik;       // momentum representation [S][P] (unnormalised FFT)
  const double* V;        // packed potential [S(S+1)/2][P]
  const double* Tax;      // concatenated per-axis p_k^2/(2 m_d)
  int64_t n[3];
  int D, S;
  long long P;
  int fp32;
};
int obs_partial_blocks();
cudaError_t launch_observables(const ObsArgs& a, double* partials, double* out, cudaStream_t st);

}  // namespace dso
