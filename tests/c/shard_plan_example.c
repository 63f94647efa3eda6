/* A plain C caller of the period-shard layout (mpopf_shard_plan): a 3-bus,
 * 3-branch network with one generator and one load, T = 5 periods split into
 * [0, 2), [2, 3), [3, 5).  Host computation only: no device is needed.  Prints
 * for every shard its local sizes and halo offsets, then its ranges (kind,
 * local start, whole-horizon start, count), for the test that compares them
 * with the Python binding's. */
#include <stdio.h>

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
  mpopf_network net = {3, 3, 1, 1, 0, gs, bs, vmin, vmax, f, t, r, x, b, tap, shift, smax, amin, amax,
                       gbus, c2, c1, c0, pmin, pmax, qmin, qmax, ramp, lbus, NULL};
  const int32_t spans[3][2] = {{0, 2}, {2, 3}, {3, 5}};
  for (int k = 0; k < 3; ++k) {
    mpopf_shard_layout lay;
    if (mpopf_shard_plan(&net, 5, spans[k][0], spans[k][1], &lay) != MPOPF_OK) {
      fprintf(stderr, "plan: %s\n", mpopf_last_error());
      return 1;
    }
    printf("%d %d %d %d %d %lld %lld %lld %lld %lld %lld %lld %lld %lld %d\n", lay.t0, lay.t1, lay.local_periods,
           lay.own0, lay.own1, (long long)lay.n, (long long)lay.m, (long long)lay.nnz_jac, (long long)lay.nnz_hess,
           (long long)lay.nnz_kkt, (long long)lay.x_recv[0], (long long)lay.x_send[0], (long long)lay.d_recv[0],
           (long long)lay.d_send[0], lay.n_ranges);
    for (int32_t i = 0; i < lay.n_ranges; ++i)
      printf("%d %lld %lld %lld\n", lay.ranges[i].what, (long long)lay.ranges[i].local,
             (long long)lay.ranges[i].global, (long long)lay.ranges[i].count);
  }
  /* a bad split is refused on the host */
  mpopf_shard_layout bad;
  if (mpopf_shard_plan(&net, 5, 3, 3, &bad) != MPOPF_ERR_ARG) return 2;
  return 0;
}
