/* rabi.c -- the library from plain C, through include/dso.h.
 *
 * Two flat surfaces coupled by a constant c on a 1-D grid: V = [[0, c],
 * [c, 0]] does not depend on q, so it commutes with the kinetic energy and
 * every split-operator composition is exact at any dt.  A packet started on
 * surface 1 then transfers population as P2(t) = sin^2(c t) (Rabi
 * oscillation).  The program propagates with the Suzuki order-6 composition,
 * reads the populations after every chunk of steps and exits non-zero if
 * any differs from sin^2(c t) by more than 1e-12.
 *
 * Build (the library is built in-tree by paper_1903_04946_gb300/build.py):
 *   gcc -O2 -I include paper_1903_04946_gb300/examples/rabi.c \
 *       -L paper_1903_04946_gb300 -ldso_gb300 -Wl,-rpath,$PWD/paper_1903_04946_gb300 -lm -o rabi
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "dso.h"

#define CHECK(call)                                                              \
  do {                                                                           \
    dso_status s_ = (call);                                                      \
    if (s_ != DSO_OK) {                                                          \
      fprintf(stderr, "%s failed (%d): %s\n", #call, (int)s_, dso_last_error()); \
      return 2;                                                                  \
    }                                                                            \
  } while (0)

int main(void) {
  const int64_t n = 256;
  const double qmin = -10.0, qmax = 10.0, mass = 1.0, c = 0.05, dt = 0.5;
  const int S = 2, chunks = 8, steps_per_chunk = 10;
  double V[3 * 256];  /* packed upper triangle: V11, V12, V22 */
  double psi[2 * 2 * 256];  /* complex128 [S][n] as (re, im) pairs */
  const double dq = (qmax - qmin) / (double)n;
  double norm2 = 0.0;
  for (int k = 0; k < n; ++k) {
    const double q = qmin + k * dq;
    V[k] = 0.0;
    V[n + k] = c;
    V[2 * n + k] = 0.0;
    const double g = exp(-0.5 * (q - 1.0) * (q - 1.0));
    psi[2 * k] = g * cos(0.7 * q); /* surface 1 */
    psi[2 * k + 1] = g * sin(0.7 * q);
    psi[2 * (n + k)] = 0.0; /* surface 2 */
    psi[2 * (n + k) + 1] = 0.0;
    norm2 += g * g * dq;
  }
  for (int k = 0; k < 2 * n; ++k) psi[k] /= sqrt(norm2);

  dso_ctx* ctx = NULL;
  CHECK(dso_create(&ctx, 0, DSO_FP64, NULL));
  CHECK(dso_set_grid(ctx, 1, &n, &qmin, &qmax));
  CHECK(dso_set_masses(ctx, &mass));
  CHECK(dso_load_potential(ctx, S, V, DSO_HOST));
  CHECK(dso_set_scheme(ctx, 6, DSO_SUZUKI, DSO_VTV, 1));
  CHECK(dso_set_psi(ctx, psi, DSO_HOST));

  double worst = 0.0;
  for (int i = 1; i <= chunks; ++i) {
    CHECK(dso_propagate(ctx, steps_per_chunk * dt, dt));
    double norm, energy, pops[2];
    CHECK(dso_observables(ctx, &norm, &energy, pops));
    const double t = i * steps_per_chunk * dt, exact = sin(c * t) * sin(c * t);
    const double err = fabs(pops[1] - exact);
    if (err > worst) worst = err;
    printf("t = %6.1f  P2 = %.15f  sin^2(ct) = %.15f  norm = %.15f\n", t, pops[1], exact, norm);
  }
  dso_destroy(ctx);
  printf("max |P2 - sin^2(ct)| = %.3e\n", worst);
  return worst <= 1e-12 ? 0 : 1;
}
