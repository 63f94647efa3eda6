/* A plain C caller of libmpopf: a 3-bus, 3-branch network with one generator
 * and one load over T = 2 periods, evaluated through the host-buffer sweep (no
 * CUDA calls in this program).  Prints n, m, nnz and every output, one value
 * per line, for the test that compares them with the CPU reference. */
#include <stdio.h>
#include <stdlib.h>

#include "mpopf.h"

int main(void) {
  const double gs[3] = {0.0, 0.02, 0.0}, bs[3] = {0.0, 0.1, 0.0};
  const double vmin[3] = {0.9, 0.9, 0.9}, vmax[3] = {1.1, 1.1, 1.1};
  const int32_t f[3] = {0, 1, 0}, t[3] = {1, 2, 2};
  const double r[3] = {0.01, 0.02, 0.015}, x[3] = {0.1, 0.12, 0.08}, b[3] = {0.02, 0.01, 0.0};
  const double tap[3] = {1.0, 1.03, 1.0}, shift[3] = {0.0, 0.0, 0.05};
  const double smax[3] = {1.5, 1.2, 1.0}, amin[3] = {-0.5, -0.5, -0.5}, amax[3] = {0.5, 0.5, 0.5};
  const int32_t gbus[1] = {0}, lbus[1] = {2};
  const double c2[1] = {0.05}, c1[1] = {20.0}, c0[1] = {1.0}, pmin[1] = {0.0}, pmax[1] = {3.0};
  const double qmin[1] = {-1.5}, qmax[1] = {1.5}, ramp[1] = {0.6};
  const double pd[2] = {0.8, 0.9}, qd[2] = {0.2, 0.25};
  mpopf_network net = {3, 3, 1, 1, 0, gs, bs, vmin, vmax, f, t, r, x, b, tap, shift, smax, amin, amax,
                       gbus, c2, c1, c0, pmin, pmax, qmin, qmax, ramp, lbus, NULL};
  mpopf_handle *h = NULL;
  mpopf_pattern pat;
  if (mpopf_setup(&net, 2, pd, qd, &h, &pat) != MPOPF_OK) {
    fprintf(stderr, "setup: %s\n", mpopf_last_error());
    return 1;
  }
  const int64_t n = pat.n, m = pat.m;
  double *xv = malloc(n * sizeof(double)), *lam = malloc(m * sizeof(double));
  double *sx = malloc(n * sizeof(double)), *dv = malloc(m * sizeof(double));
  double *grad = malloc(n * sizeof(double)), *c = malloc(m * sizeof(double));
  double *jv = malloc(pat.nnz_jac * sizeof(double)), *hv = malloc(pat.nnz_hess * sizeof(double));
  double *kv = malloc(pat.nnz_kkt * sizeof(double)), fval = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    xv[i] = 1.0 + 0.01 * (double)((i * 7) % 11 - 5);
    sx[i] = 0.5 + 0.25 * (double)(i % 3);
  }
  for (int64_t i = 0; i < m; ++i) {
    lam[i] = 0.1 * (double)((i * 5) % 9 - 4);
    dv[i] = 1.0 + 0.5 * (double)(i % 4);
  }
  if (mpopf_sweep_host(h, xv, lam, 1.0, sx, dv, 1e-8, &fval, grad, c, jv, hv, kv, NULL) != MPOPF_OK) {
    fprintf(stderr, "sweep: %s\n", mpopf_last_error());
    return 1;
  }
  printf("%lld %lld %lld %lld %lld\n", (long long)n, (long long)m, (long long)pat.nnz_jac, (long long)pat.nnz_hess,
         (long long)pat.nnz_kkt);
  printf("%.17g\n", fval);
  for (int64_t i = 0; i < n; ++i) printf("%.17g\n", grad[i]);
  for (int64_t i = 0; i < m; ++i) printf("%.17g\n", c[i]);
  for (int64_t i = 0; i < pat.nnz_jac; ++i) printf("%.17g\n", jv[i]);
  for (int64_t i = 0; i < pat.nnz_hess; ++i) printf("%.17g\n", hv[i]);
  for (int64_t i = 0; i < pat.nnz_kkt; ++i) printf("%.17g\n", kv[i]);
  mpopf_destroy(h);
  free(xv); free(lam); free(sx); free(dv); free(grad); free(c); free(jv); free(hv); free(kv);
  return 0;
}
