// coeffs.cpp -- composition and pruned splitting coefficients.
//
// Sec. II D: a symmetric method of even order p composed with coefficients
// gamma_1..gamma_M (sum 1, symmetric) is of order p + 2:
//   triple jump (M = 3):  gamma = (x, 1 - 2x, x),       x = 1/(2 - 2^(1/(p+1)))
//   Suzuki fractal (M=5): gamma = (y, y, 1 - 4y, y, y), y = 1/(4 - 4^(1/(p+1)))
// (the paper prints p = 2, Eqs. (triple_jump_fourth_order_so) and
// (suzukis_fractals_fourth_order_so); 1 - 2x = -2^(1/(p+1)) x).  Applied
// recursively from p = 2, the outer coefficient scales the whole inner
// sequence.  Sec. II E: each elementary second-order step of length gamma dt
// contributes a = (gamma/2, gamma/2), b = (gamma, 0).  Sec. II F, Eq.
// (merging_splitting_coeff_b_zero): a zero b_j (j != N) is removed and
// a_j, a_{j+1} merged; the trailing b_N = 0 is dropped, so N_A = N_B + 1.
// Repeated values are found on the first half of the symmetric sequence and
// mirrored (Eq. (range_index_unq), indices 0-based here).
//
// The "optimal" compositions of Sec. II D (Table II's last rows) are not
// recursive: they take the 9-stage (order 6) and 17-stage (order 8)
// symmetric coefficients that Kahan and Li (Math. Comp. 66, 1089 (1997))
// obtained by numerical optimisation, listed below to 20 significant digits
// (first half and middle coefficient).
//
// Arithmetic is in long double; values are rounded to double once.
#include <cmath>
#include <cstdlib>
#include <stdexcept>

#include "dso_internal.h"

namespace dso {

namespace {

std::vector<long double> outer_gamma(int p, int scheme) {
  const long double e = 1.0L / (long double)(p + 1);
  if (scheme == 0) {
    const long double x = 1.0L / (2.0L - powl(2.0L, e));
    return {x, 1.0L - 2.0L * x, x};
  }
  const long double y = 1.0L / (4.0L - powl(4.0L, e));
  return {y, y, 1.0L - 4.0L * y, y, y};
}

void find_unique(const std::vector<long double>& v, std::vector<double>& uniq, std::vector<int>& idx) {
  const size_t n = v.size(), half = (n + 1) / 2;
  std::vector<long double> u;
  idx.assign(n, -1);
  for (size_t j = 0; j < half; ++j) {
    int found = -1;
    for (size_t k = 0; k < u.size(); ++k) {
      const long double scale = fmaxl(fabsl(v[j]), fabsl(u[k]));
      if (fabsl(v[j] - u[k]) <= 1e-12L * scale) {
        found = (int)k;
        break;
      }
    }
    if (found < 0) {
      u.push_back(v[j]);
      found = (int)u.size() - 1;
    }
    idx[j] = found;
  }
  for (size_t j = half; j < n; ++j) idx[j] = idx[n - 1 - j];
  uniq.clear();
  for (long double x : u) uniq.push_back((double)x);
}

// First half and middle of the optimal compositions (time order).
const char* const kOptimal6[] = {"0.39216144400731413928", "0.33259913678935943860", "-0.70624617255763935981",
                                 "0.082213596293550800230", "0.79854399093482996340"};
const char* const kOptimal8[] = {"0.13020248308889008088", "0.56116298177510838456", "-0.38947496264484728641",
                                 "0.15884190655515560090", "-0.39590389413323757734", "0.18453964097831570709",
                                 "0.25837438768632204729", "0.29501172360931029887", "-0.60550853383003451170"};

std::vector<long double> optimal_gamma(int order) {
  const char* const* half = order == 6 ? kOptimal6 : kOptimal8;
  const int nh = order == 6 ? 5 : 9;
  std::vector<long double> h;
  for (int k = 0; k < nh; ++k) h.push_back(strtold(half[k], nullptr));
  std::vector<long double> g(h.begin(), h.end() - 1);
  g.push_back(h.back());
  for (int k = nh - 2; k >= 0; --k) g.push_back(h[k]);
  return g;
}

}  // namespace

Coeffs coefficients_from_gammas(const std::vector<long double>& g) {
  // expand and prune in one scan: a's accumulate until a nonzero b closes them
  std::vector<long double> at, bt;
  long double pending = 0.0L;
  bool open = false;
  for (long double gam : g) {
    const long double half = gam / 2.0L;
    // first half-step V(gamma/2), kinetic T(gamma), second half-step V(gamma/2), kinetic T(0)
    pending = open ? pending + half : half;
    open = true;
    at.push_back(pending);
    bt.push_back(gam);
    pending = half;  // opens the next accumulation; T(0) is pruned
  }
  at.push_back(pending);
  Coeffs c;
  for (long double x : at) c.a.push_back((double)x);
  for (long double x : bt) c.b.push_back((double)x);
  find_unique(at, c.a_unq, c.ia);
  find_unique(bt, c.b_unq, c.ib);
  return c;
}

Coeffs build_coefficients(int order, int scheme) {
  if (order == 1) {  // first-order VT / TV (Sec. II E): a = (1, 0), b = (1)
    Coeffs c;
    c.a = {1.0, 0.0};
    c.b = {1.0};
    c.ia = {0, 1};
    c.ib = {0};
    c.a_unq = {1.0, 0.0};
    c.b_unq = {1.0};
    return c;
  }
  if (order < 2 || order % 2 != 0 || order > 10) throw std::invalid_argument("order must be 1, 2, 4, 6, 8 or 10");
  if (scheme == 2) {
    if (order != 6 && order != 8) throw std::invalid_argument("the optimal compositions have orders 6 and 8");
    return coefficients_from_gammas(optimal_gamma(order));
  }
  if (scheme != 0 && scheme != 1) throw std::invalid_argument("unknown composition scheme");
  std::vector<long double> g{1.0L};
  for (int p = 2; p < order; p += 2) {
    const std::vector<long double> out = outer_gamma(p, scheme);
    std::vector<long double> next;
    next.reserve(out.size() * g.size());
    for (long double go : out)
      for (long double gi : g) next.push_back(go * gi);
    g.swap(next);
  }
  return coefficients_from_gammas(g);
}

}  // namespace dso
