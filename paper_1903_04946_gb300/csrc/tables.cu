// tables.cu -- operator tables built once per (potential, scheme, dt).
//
// Sec. II F: for a time-independent separable Hamiltonian the evolution
// operators U_V(a dt) and U_T(b dt) can be precomputed once for every unique
// coefficient and stored; the index arrays I^a, I^b then say which one each
// action uses.  This file builds
//   * FFT twiddles exp(-2 pi i m / L) in tangent form (cos, tan), host long
//     double;
//   * kinetic phases tau_b(p) = exp(-i b dt T(p)) / P with
//     T(p) = sum_d p_d^2 / (2 m_d) (Eq. (diab_mol_ham)): the phase from
//     long-double coefficients, accumulated in double-double on the device
//     and exponentiated once (the 1/P of the unnormalised inverse FFTs is an
//     exact power of two);
//   * twiddles of split (long) axes for the four-step FFT;
//   * potential unitaries U_a(q) = exp(-i a dt V(q)) (Sec. II H): for S = 2 the
//     closed form that one Jacobi rotation gives; for S >= 3 cyclic Jacobi to
//     convergence, then U = W diag(exp(-i a dt lambda)) W^T.  Stored packed
//     (U is complex symmetric because V is real symmetric).
#include <cmath>

#include "dso_internal.h"

namespace dso {

std::vector<double2> host_twiddles(int L, bool fp32) {
  std::vector<double2> tw(L);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  // c = 0 (m = L/4) is stored as a tiny power of two: t = s / c stays finite
  // and c (b + i t b) keeps the exact value to far below one ulp
  const long double tiny = fp32 ? ldexpl(1.0L, -60) : ldexpl(1.0L, -500);
  for (int m = 0; m < L; ++m) {
    const long double ang = -two_pi * (long double)m / (long double)L;
    long double c = cosl(ang);
    const long double sn = sinl(ang);
    if (fabsl(c) < tiny) c = tiny;
    tw[m] = make_double2((double)c, (double)(sn / c));
  }
  return tw;
}

std::vector<double> host_kinetic_coefficients(int D, const double* qmin, const double* qmax, const double* mass,
                                              const std::vector<double>& b_unq, double dt) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  std::vector<double> out(b_unq.size() * (size_t)D * 2);
  for (size_t u = 0; u < b_unq.size(); ++u) {
    const long double tb = (long double)b_unq[u] * (long double)dt;
    for (int d = 0; d < D; ++d) {
      const long double w = two_pi / ((long double)qmax[d] - (long double)qmin[d]);  // 2 pi / (n dq)
      const long double C = -tb * w * w / (2.0L * (long double)mass[d]);
      const double hi = (double)C;
      out[(u * D + d) * 2] = hi;
      out[(u * D + d) * 2 + 1] = (double)(C - (long double)hi);
    }
  }
  return out;
}

__device__ __forceinline__ void store_c(double2* p, double x, double y) { *p = make_double2(x, y); }
__device__ __forceinline__ void store_c(float2* p, double x, double y) { *p = make_float2((float)x, (float)y); }

// tau[u][g]: the kinetic phase of every unique b at storage position g.  The
// angle sum_d C_d kk_d^2 is accumulated as hi + lo (kk_d^2 < 2^42 is exact;
// fma gives the exact error of each product, Knuth's two-sum that of each
// addition), so it carries the long-double coefficients to about 1e-30
// relative; exp(i (hi + lo)) = (cos hi + i sin hi)(1 + i lo) to first order
// in |lo| <= a few ulp of hi.
template <typename OutC>
__global__ void kinetic_table_kernel(OutC* __restrict__ tau, const double* __restrict__ coef, int nb, VLayout v,
                                     long long P, double inv_P) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= P) return;
  const int u = blockIdx.y;
  int64_t k[3] = {0, 0, 0};
  momentum_indices(v, g, k);
  double hi = 0.0, lo = 0.0;
  for (int d = 0; d < v.D; ++d) {
    const int64_t kk = (k[d] < v.n[d] / 2) ? k[d] : k[d] - v.n[d];
    const double x = (double)(kk * kk);
    const double ch = coef[(u * v.D + d) * 2], cl = coef[(u * v.D + d) * 2 + 1];
    const double p = ch * x;
    const double pe = fma(ch, x, -p);  // exact error of the product
    const double s = hi + p;           // two-sum
    const double bb = s - hi;
    const double se = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += se + pe + cl * x;
  }
  const double r = hi + lo;  // renormalise
  lo = lo - (r - hi);
  hi = r;
  double sn, cs;
  sincos(hi, &sn, &cs);
  store_c(&tau[(size_t)u * P + g], inv_P * (cs - sn * lo), inv_P * (sn + cs * lo));
}

cudaError_t launch_kinetic_tables(void* tau, bool fp32, const double* coef, int nb, const VLayout& v, long long P,
                                  cudaStream_t st) {
  dim3 grid((unsigned)((P + 255) / 256), (unsigned)nb);
  const double inv_P = 1.0 / (double)P;  // a power of two: exact
  if (fp32)
    kinetic_table_kernel<<<grid, 256, 0, st>>>((float2*)tau, coef, nb, v, P, inv_P);
  else
    kinetic_table_kernel<<<grid, 256, 0, st>>>((double2*)tau, coef, nb, v, P, inv_P);
  return cudaGetLastError();
}

// tau[u][off_d + k]: the phase of axis d alone, exp(i C_d kk^2) / n_d, with
// the angle carried as hi + lo as in kinetic_table_kernel (one term).
struct AxisSizes {
  int64_t n[3];
};

template <typename OutC>
__global__ void axis_kinetic_table_kernel(OutC* __restrict__ tau, const double* __restrict__ coef, int D,
                                          AxisSizes ax, long long len) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= len) return;
  const int u = blockIdx.y;
  int d = 0;
  long long k = idx;
  while (d + 1 < D && k >= ax.n[d]) k -= ax.n[d++];
  const long long n = ax.n[d];
  const long long kk = (k < n / 2) ? k : k - n;
  const double x = (double)(kk * kk);
  const double ch = coef[(u * D + d) * 2], cl = coef[(u * D + d) * 2 + 1];
  double hi = ch * x;
  double lo = fma(ch, x, -hi) + cl * x;
  const double r = hi + lo;  // renormalise
  lo = lo - (r - hi);
  hi = r;
  double sn, cs;
  sincos(hi, &sn, &cs);
  const double inv_n = 1.0 / (double)n;  // a power of two: exact
  store_c(&tau[(size_t)u * len + idx], inv_n * (cs - sn * lo), inv_n * (sn + cs * lo));
}

cudaError_t launch_axis_kinetic_tables(void* tau, bool fp32, const double* coef, int nb, int D, const int64_t* n,
                                       cudaStream_t st) {
  AxisSizes ax{};
  long long len = 0;
  for (int d = 0; d < D && d < 3; ++d) {
    ax.n[d] = n[d];
    len += n[d];
  }
  dim3 grid((unsigned)((len + 255) / 256), (unsigned)nb);
  if (fp32)
    axis_kinetic_table_kernel<<<grid, 256, 0, st>>>((float2*)tau, coef, D, ax, len);
  else
    axis_kinetic_table_kernel<<<grid, 256, 0, st>>>((double2*)tau, coef, D, ax, len);
  return cudaGetLastError();
}

// Split-axis twiddles w_n^(k1 i2) in the [n1][n2] layout of the passes.
template <typename OutC>
__global__ void split_twiddle_kernel(OutC* __restrict__ xtw, int64_t n1, int64_t n2) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = n1 * n2;
  if (idx >= n) return;
  const long long k1 = idx / n2, i2 = idx - k1 * n2;
  const long long m = (k1 * i2) & (n - 1);
  double sn, cs;
  sincospi(-2.0 * (double)m / (double)n, &sn, &cs);  // m / n is exact (n a power of two)
  store_c(&xtw[idx], cs, sn);
}

cudaError_t launch_split_twiddles(void* xtw, bool fp32, int64_t n1, int64_t n2, cudaStream_t st) {
  const long long n = n1 * n2;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (fp32)
    split_twiddle_kernel<<<blocks, 256, 0, st>>>((float2*)xtw, n1, n2);
  else
    split_twiddle_kernel<<<blocks, 256, 0, st>>>((double2*)xtw, n1, n2);
  return cudaGetLastError();
}

namespace {

// Cyclic Jacobi eigendecomposition of a real symmetric S x S matrix:
// A = W diag(lam) W^T.  Rotations zero one off-diagonal pair at a time
// (Golub & Van Loan, Sec. 8.5); stops when the off-diagonal mass is below
// 1e-32 of the total, or after 50 sweeps.
template <int S>
__device__ void jacobi_eig(double (&A)[S][S], double (&W)[S][S], double (&lam)[S]) {
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) W[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < S; ++i)
      for (int j = 0; j < S; ++j) {
        const double v = A[i][j] * A[i][j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < S - 1; ++p)
      for (int q = p + 1; q < S; ++q) {
        const double apq = A[p][q];
        if (apq == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0);
        const double s = t * c;
        for (int k = 0; k < S; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < S; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < S; ++k) {  // W <- W J
          const double wkp = W[k][p], wkq = W[k][q];
          W[k][p] = c * wkp - s * wkq;
          W[k][q] = s * wkp + c * wkq;
        }
      }
  }
  for (int i = 0; i < S; ++i) lam[i] = A[i][i];
}

// The per-point part of U_a(q) = exp(-i a dt V(q)) that does not depend on
// the coefficient: for S = 2 the mean, the half difference and the coupling
// of the diagonal entries and the rotation rate r; for S >= 3 the
// eigenvectors W and eigenvalues lam of V(q).  NC doubles per point.
template <int S>
struct EigPoint {
  static constexpr int NC = S == 2 ? 4 : S * S + S;
  double v0, vz, vx, r;       // S = 2
  double W[S][S], lam[S];     // S >= 3
};

template <int S>
__device__ __forceinline__ void eig_point(const double* __restrict__ V, long long g, long long P, EigPoint<S>& e) {
  if constexpr (S == 2) {
    const double v11 = V[g], v12 = V[P + g], v22 = V[2 * P + g];
    e.v0 = 0.5 * (v11 + v22);
    e.vz = 0.5 * (v11 - v22);
    e.vx = v12;
    e.r = sqrt(e.vx * e.vx + e.vz * e.vz);
  } else {
    double A[S][S];
    int k = 0;
    for (int r = 0; r < S; ++r)
      for (int c = r; c < S; ++c) {
        const double v = V[(size_t)k * P + g];
        A[r][c] = v;
        A[c][r] = v;
        ++k;
      }
    jacobi_eig<S>(A, e.W, e.lam);
  }
}

// The packed S(S+1)/2 entries of U at point g for coefficient t = a dt.
template <int S, typename OutC>
__device__ __forceinline__ void store_unitary(const EigPoint<S>& e, double t, OutC* __restrict__ out, long long g,
                                              long long P) {
  if constexpr (S == 2) {
    double sr, cr, sg, cg;
    sincos(e.r * t, &sr, &cr);
    const double s_over_r = (e.r > 0.0) ? sr / e.r : t;
    sincos(-t * e.v0, &sg, &cg);  // exp(-i t v0) = cg + i sg
    // U = exp(-i t v0) [cos(r t) 1 - i sin(r t)/r (vx sx + vz sz)]
    const double2 d0 = make_double2(cr, -s_over_r * e.vz);  // c - i s vz
    const double2 d1 = make_double2(cr, s_over_r * e.vz);   // c + i s vz
    const double2 od = make_double2(0.0, -s_over_r * e.vx); // -i s vx
    store_c(&out[g], cg * d0.x - sg * d0.y, cg * d0.y + sg * d0.x);
    store_c(&out[P + g], cg * od.x - sg * od.y, cg * od.y + sg * od.x);
    store_c(&out[2 * P + g], cg * d1.x - sg * d1.y, cg * d1.y + sg * d1.x);
  } else {
    double ph_re[S], ph_im[S];
    for (int m = 0; m < S; ++m) sincos(-t * e.lam[m], &ph_im[m], &ph_re[m]);
    int kk = 0;
    for (int r = 0; r < S; ++r)
      for (int c = r; c < S; ++c) {
        double re = 0.0, im = 0.0;
        for (int m = 0; m < S; ++m) {
          const double w = e.W[r][m] * e.W[c][m];
          re += w * ph_re[m];
          im += w * ph_im[m];
        }
        store_c(&out[(size_t)kk * P + g], re, im);
        ++kk;
      }
  }
}

template <int S, typename OutC>
__global__ void potential_table_kernel(OutC* __restrict__ U, const double* __restrict__ V,
                                       const double* __restrict__ tau_a, int na, long long P) {
  constexpr int NP = S * (S + 1) / 2;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= P) return;
  EigPoint<S> e;
  eig_point<S>(V, g, P, e);
  for (int u = 0; u < na; ++u) store_unitary<S>(e, tau_a[u], U + (size_t)u * NP * P, g, P);
}

// The coefficient-independent part of every point, stored [NC][P].
template <int S>
__global__ void eig_cache_kernel(double* __restrict__ E, const double* __restrict__ V, long long P) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= P) return;
  EigPoint<S> e;
  eig_point<S>(V, g, P, e);
  if constexpr (S == 2) {
    E[g] = e.v0;
    E[P + g] = e.vz;
    E[2 * P + g] = e.vx;
    E[3 * P + g] = e.r;
  } else {
    for (int r = 0; r < S; ++r)
      for (int c = 0; c < S; ++c) E[(size_t)(r * S + c) * P + g] = e.W[r][c];
    for (int m = 0; m < S; ++m) E[(size_t)(S * S + m) * P + g] = e.lam[m];
  }
}

// U for the one coefficient tau_a[0] from the stored part: the values are
// reloaded exactly, so the entries are potential_table_kernel's, bit for bit.
template <int S, typename OutC>
__global__ void unitary_from_cache_kernel(OutC* __restrict__ U, const double* __restrict__ E,
                                          const double* __restrict__ tau_a, long long P) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= P) return;
  EigPoint<S> e;
  if constexpr (S == 2) {
    e.v0 = E[g];
    e.vz = E[P + g];
    e.vx = E[2 * P + g];
    e.r = E[3 * P + g];
  } else {
    for (int r = 0; r < S; ++r)
      for (int c = 0; c < S; ++c) e.W[r][c] = E[(size_t)(r * S + c) * P + g];
    for (int m = 0; m < S; ++m) e.lam[m] = E[(size_t)(S * S + m) * P + g];
  }
  store_unitary<S>(e, tau_a[0], U, g, P);
}

template <typename OutC>
cudaError_t launch_potential_tables_t(OutC* U, const double* V, const double* tau_a, int na, int S, long long P,
                                      cudaStream_t st) {
  const unsigned blocks = (unsigned)((P + 127) / 128);
  switch (S) {
    case 2: potential_table_kernel<2><<<blocks, 128, 0, st>>>(U, V, tau_a, na, P); break;
    case 3: potential_table_kernel<3><<<blocks, 128, 0, st>>>(U, V, tau_a, na, P); break;
    case 4: potential_table_kernel<4><<<blocks, 128, 0, st>>>(U, V, tau_a, na, P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename OutC>
cudaError_t launch_unitary_from_cache_t(OutC* U, const double* E, const double* tau_a, int S, long long P,
                                        cudaStream_t st) {
  const unsigned blocks = (unsigned)((P + 127) / 128);
  switch (S) {
    case 2: unitary_from_cache_kernel<2><<<blocks, 128, 0, st>>>(U, E, tau_a, P); break;
    case 3: unitary_from_cache_kernel<3><<<blocks, 128, 0, st>>>(U, E, tau_a, P); break;
    case 4: unitary_from_cache_kernel<4><<<blocks, 128, 0, st>>>(U, E, tau_a, P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_potential_tables(void* U, bool fp32, const double* V, const double* tau_a, int na, int S,
                                    long long P, cudaStream_t st) {
  return fp32 ? launch_potential_tables_t((float2*)U, V, tau_a, na, S, P, st)
              : launch_potential_tables_t((double2*)U, V, tau_a, na, S, P, st);
}

int eig_cache_doubles(int S) { return S == 2 ? 4 : S * S + S; }

cudaError_t launch_eig_cache(double* E, const double* V, int S, long long P, cudaStream_t st) {
  const unsigned blocks = (unsigned)((P + 127) / 128);
  switch (S) {
    case 2: eig_cache_kernel<2><<<blocks, 128, 0, st>>>(E, V, P); break;
    case 3: eig_cache_kernel<3><<<blocks, 128, 0, st>>>(E, V, P); break;
    case 4: eig_cache_kernel<4><<<blocks, 128, 0, st>>>(E, V, P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_unitary_from_cache(void* U, bool fp32, const double* E, const double* tau_a, int S, long long P,
                                      cudaStream_t st) {
  return fp32 ? launch_unitary_from_cache_t((float2*)U, E, tau_a, S, P, st)
              : launch_unitary_from_cache_t((double2*)U, E, tau_a, S, P, st);
}

}  // namespace dso
