// tables.cu -- operator tables built once per (potential, scheme, dt).
//
// Sec. II F: for a time-independent separable Hamiltonian the evolution
// operators U_V(a dt) and U_T(b dt) can be precomputed once for every unique
// coefficient and stored; the index arrays I^a, I^b then say which one each
// action uses.  This file builds
//   * FFT twiddles exp(-2 pi i m / L) in tangent form (cos, tan), host long
//     double;
//   * kinetic phases tau_b(p) = exp(-i b dt T(p)) / P with
//     T(p) = sum_d p_d^2 / (2 m_d) (Eq. (diab_mol_ham)), as a product of 1-D
//     factors computed on the host in long double (the 1/P of the unnormalised
//     inverse FFT is an exact power of two folded into axis 0);
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

std::vector<double2> host_kinetic_factors(int D, const int64_t* n, const double* qmin, const double* qmax,
                                          const double* mass, const std::vector<double>& b_unq, double dt) {
  int64_t tot = 0, P = 1;
  for (int d = 0; d < D; ++d) {
    tot += n[d];
    P *= n[d];
  }
  const long double two_pi = 6.283185307179586476925286766559005768L;
  std::vector<double2> out((size_t)tot * b_unq.size());
  for (size_t u = 0; u < b_unq.size(); ++u) {
    const long double tb = (long double)b_unq[u] * (long double)dt;
    int64_t off = 0;
    for (int d = 0; d < D; ++d) {
      const long double extent = (long double)qmax[d] - (long double)qmin[d];
      const long double scale = (d == 0) ? 1.0L / (long double)P : 1.0L;
      for (int64_t k = 0; k < n[d]; ++k) {
        const int64_t kk = (k < n[d] / 2) ? k : k - n[d];
        const long double p = two_pi * (long double)kk / extent;  // 2 pi k / (n dq)
        const long double ang = -tb * p * p / (2.0L * (long double)mass[d]);
        out[u * tot + off + k] = make_double2((double)(scale * cosl(ang)), (double)(scale * sinl(ang)));
      }
      off += n[d];
    }
  }
  return out;
}

__device__ __forceinline__ void store_c(double2* p, double x, double y) { *p = make_double2(x, y); }
__device__ __forceinline__ void store_c(float2* p, double x, double y) { *p = make_float2((float)x, (float)y); }

template <typename OutC>
__global__ void kinetic_table_kernel(OutC* __restrict__ tau, const double2* __restrict__ fac, int nb, int D,
                                     int64_t n0, int64_t n1, int64_t n2, long long P) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= P) return;
  const int u = blockIdx.y;
  const int64_t tot = n0 + (D > 1 ? n1 : 0) + (D > 2 ? n2 : 0);
  const double2* f = fac + (size_t)u * tot;
  int64_t k[3];
  long long r = g;
  const int64_t nn[3] = {n0, n1, n2};
  for (int d = D - 1; d >= 0; --d) {
    k[d] = r % nn[d];
    r /= nn[d];
  }
  double2 t = f[k[0]];
  int64_t off = n0;
  for (int d = 1; d < D; ++d) {
    const double2 x = f[off + k[d]];
    t = make_double2(t.x * x.x - t.y * x.y, t.x * x.y + t.y * x.x);
    off += nn[d];
  }
  store_c(&tau[(size_t)u * P + g], t.x, t.y);
}

cudaError_t launch_kinetic_tables(void* tau, bool fp32, const double2* factors, int nb, int D, const int64_t* n,
                                  long long P, cudaStream_t st) {
  dim3 grid((unsigned)((P + 255) / 256), (unsigned)nb);
  if (fp32)
    kinetic_table_kernel<<<grid, 256, 0, st>>>((float2*)tau, factors, nb, D, n[0], D > 1 ? n[1] : 1,
                                               D > 2 ? n[2] : 1, P);
  else
    kinetic_table_kernel<<<grid, 256, 0, st>>>((double2*)tau, factors, nb, D, n[0], D > 1 ? n[1] : 1,
                                               D > 2 ? n[2] : 1, P);
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

template <int S, typename OutC>
__global__ void potential_table_kernel(OutC* __restrict__ U, const double* __restrict__ V,
                                       const double* __restrict__ tau_a, int na, long long P) {
  constexpr int NP = S * (S + 1) / 2;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= P) return;
  if constexpr (S == 2) {
    const double v11 = V[g], v12 = V[P + g], v22 = V[2 * P + g];
    const double v0 = 0.5 * (v11 + v22), vz = 0.5 * (v11 - v22), vx = v12;
    const double r = sqrt(vx * vx + vz * vz);
    for (int u = 0; u < na; ++u) {
      const double t = tau_a[u];
      double sr, cr, sg, cg;
      sincos(r * t, &sr, &cr);
      const double s_over_r = (r > 0.0) ? sr / r : t;
      sincos(-t * v0, &sg, &cg);  // exp(-i t v0) = cg + i sg
      // U = exp(-i t v0) [cos(r t) 1 - i sin(r t)/r (vx sx + vz sz)]
      const double2 d0 = make_double2(cr, -s_over_r * vz);  // c - i s vz
      const double2 d1 = make_double2(cr, s_over_r * vz);   // c + i s vz
      const double2 od = make_double2(0.0, -s_over_r * vx); // -i s vx
      OutC* out = U + (size_t)u * NP * P;
      store_c(&out[g], cg * d0.x - sg * d0.y, cg * d0.y + sg * d0.x);
      store_c(&out[P + g], cg * od.x - sg * od.y, cg * od.y + sg * od.x);
      store_c(&out[2 * P + g], cg * d1.x - sg * d1.y, cg * d1.y + sg * d1.x);
    }
  } else {
    double A[S][S], W[S][S], lam[S];
    int k = 0;
    for (int r = 0; r < S; ++r)
      for (int c = r; c < S; ++c) {
        const double v = V[(size_t)k * P + g];
        A[r][c] = v;
        A[c][r] = v;
        ++k;
      }
    jacobi_eig<S>(A, W, lam);
    for (int u = 0; u < na; ++u) {
      const double t = tau_a[u];
      double ph_re[S], ph_im[S];
      for (int m = 0; m < S; ++m) sincos(-t * lam[m], &ph_im[m], &ph_re[m]);
      OutC* out = U + (size_t)u * NP * P;
      int kk = 0;
      for (int r = 0; r < S; ++r)
        for (int c = r; c < S; ++c) {
          double re = 0.0, im = 0.0;
          for (int m = 0; m < S; ++m) {
            const double w = W[r][m] * W[c][m];
            re += w * ph_re[m];
            im += w * ph_im[m];
          }
          store_c(&out[(size_t)kk * P + g], re, im);
          ++kk;
        }
    }
  }
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

}  // namespace

cudaError_t launch_potential_tables(void* U, bool fp32, const double* V, const double* tau_a, int na, int S,
                                    long long P, cudaStream_t st) {
  return fp32 ? launch_potential_tables_t((float2*)U, V, tau_a, na, S, P, st)
              : launch_potential_tables_t((double2*)U, V, tau_a, na, S, P, st);
}

}  // namespace dso
