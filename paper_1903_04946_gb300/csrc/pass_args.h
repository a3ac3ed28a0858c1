// pass_args.h -- host-visible parameters of one axis pass (axis_pass.cuh).
#pragma once

#include <cuda_runtime.h>

namespace dso {

enum PassFlags : int {
  PASS_INV_FIRST = 1,  // inverse FFT before the potential step
  PASS_FWD = 2,        // forward FFT after the potential step
  PASS_T = 4,          // kinetic phase then inverse FFT after the forward FFT
  PASS_XTW = 8,        // the axis is the first factor of a split axis: conj twiddles
                       // before the inverse FFT, twiddles after the forward FFT
  PASS_TAX = 16,       // with PASS_T: the phase of this axis alone, a table of L entries
                       // indexed by the momentum index along the line (separable kinetic step)
  PASS_PLANE = 32,     // with PASS_FWD | PASS_T on axis D-2 of a 3-D grid, one launch for the
                       // planes of axes D-2 and D-1 (axis_pass_plane.cuh): with PASS_TAX
                       // [F T I] along each axis in turn; without, [F_a | F_b T I_b | I_a]
};

// Complex arrays are double2 (FP64 path) or float2 (FP32 storage mode).
struct PassArgs {
  void* psi;               // [S][P] wavefunction (in/out)
  const void* U1;          // [S(S+1)/2][P] potential unitary, or null
  const void* U2;          // second potential unitary, or null
  const void* tau;         // [P] kinetic phase (1/P folded in), or null; with PASS_TAX
                           // [L] the phase of this axis (1/L folded in)
  const void* tau2;        // second kinetic phase (TVT step boundary), or null;
                           // its folded 1/P (1/L) is undone by tau2_scale = P (L), exact
  const void* tw;          // [L] exp(-2 pi i m / L), m = 0..L-1
  long long P;             // grid points per surface
  long long stride;        // element stride of the axis (product of later axes)
  long long lines;         // lines per surface = P / L
  int S;                   // surfaces
  int G;                   // lines per surface in one tile (power of two)
  int flags;
  int stride_log2;         // log2(stride); every stride is a power of two
  int G_log2;              // log2(G)
  int ua;                  // unique-coefficient index of U1 (TMA variant)
  int ub;                  // unique-coefficient index of tau (TMA variant)
  int* err;                // device flag set when a bounded wait gives up
  double tau2_scale;       // P (L): both kinetic tables carry 1/P (1/L), one inverse FFT runs
  int fp32;                // 1: complex arrays are float2 (FP32 storage mode)
  int nbatch;              // independent jobs sharing the grid: psi is [nbatch][S][P]
  long long u_batch_stride;  // elements between one job's potential tables and the next
  // allocation extents (elements) for the bounds-checked debug build
  const void* U_base;      // start of the potential tables
  const void* tau_base;    // start of the kinetic tables
  long long psi_elems, u_elems, tau_elems;
  int dec0;                // surface 0 uncoupled (block-diagonal potential): skip its zero products
  int ctas_per_sm;         // host side, persistent variants: resident CTAs per SM (0: as many as fit)
  int pdl;                 // host side: launch with programmatic dependent launch
  const void* xtw;         // PASS_XTW: split-axis twiddles [n1][n2], w_n^(k1 i2), or null
  int xtw_n2_log2;         // log2 n2 (length of the second factor of the split axis)
  int xtw_s2_log2;         // log2 of the second factor's stride (product of the later axes)
  int wait_probe;          // > 0: TMA variant's bounded-wait diagnostics (polls of a barrier no copy completes)
  const void* tw2;         // PASS_PLANE: twiddles of axis D-1, or null
};

// Tile index -> (first staged surface over all jobs, job).  A pass staging
// all S surfaces (SV = S) has nbatch * lines / G tiles; one staging a single
// surface has nbatch * S * lines / G.
struct TileJob {
  long long tile;  // tile index within its line set
  int surf0;       // first surface (counted over all jobs) of the tile
  int job;
};

}  // namespace dso
