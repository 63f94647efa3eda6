// Interior-point algebra around the condensed matrix (Sec. III-B of the paper):
// the diagonal scalings Sigma_x, Sigma_s, C, D from the bounds and duals (with
// the relaxation of equality rows to [g - eps, g + eps]), the condensed
// right-hand side q_x + A^T (C q_s + D q_y), and the recovery of the slack,
// multiplier and bound-dual steps from dx.
//
// FP64 division is the expensive operation on this GPU (a reciprocal sequence
// on the FP64 pipe), so every division happens once, in mpopf_ipm_prepare: the
// reciprocals rl = 1/(v - lo), ru = 1/(hi - v) go to a caller workspace and
// the right-hand side and the recovery are division-free.  With the bound-dual
// rows of Eq. (5) eliminated, the dual terms cancel (-zl + (zl dl - mu)/dl =
// -mu rl), which is the form used here and by the CPU oracle.  The recovered
// slack step is the one Eq. (5) implies, ds = C (A dx + delta_c q_s - q_y).
// Every value follows the oracle's written rounding order.
#include <string>

#include "mpopf_internal.cuh"

extern "C" int mpopf_vjp_jv(mpopf_handle *h, const double *x, const double *jv, const double *y, double *gx,
                            double *gpd, double *gqd, void *stream);
extern "C" int mpopf_jvp_jv(mpopf_handle *h, const double *x, const double *jv, const double *v, const double *dpd,
                            const double *dqd, double *jv_out, void *stream);

namespace mpopf {
namespace {

__device__ __forceinline__ bool finite(double v) { return ((__double2hiint(v) >> 20) & 0x7ff) != 0x7ff; }

// a == b for binary64 values (+0 == -0, NaN equal to nothing) by integer
// operations: the comparison would otherwise take an FP64 pipe slot
// (measured: mpopf_ipm_prepare 1.182 -> 1.139 ms at 10k buses x 168).
__device__ __forceinline__ bool feq(double a, double b) {
  const unsigned long long x = (unsigned long long)__double_as_longlong(a);
  const unsigned long long y = (unsigned long long)__double_as_longlong(b);
  const bool nan = (x << 1) > 0xffe0000000000000ULL || (y << 1) > 0xffe0000000000000ULL;
  return !nan && (x == y || ((x | y) << 1) == 0);
}

// rl = 1/(v - lo), ru = 1/(hi - v); 0 for an infinite bound.
__device__ __forceinline__ void recips(double v, double lo, double hi, double *rl, double *ru) {
  *rl = finite(lo) ? 1.0 / (v - lo) : 0.0;
  *ru = finite(hi) ? 1.0 / (hi - v) : 0.0;
}

__device__ __forceinline__ double sigma_of(double rl, double ru, double zl, double zu) { return fma(zl, rl, zu * ru); }

__global__ void __launch_bounds__(kBlock) k_prep_vars(int64_t n, const double *__restrict__ x,
                                                      const double *__restrict__ xl, const double *__restrict__ xu,
                                                      const double *__restrict__ zl, const double *__restrict__ zu,
                                                      double *__restrict__ sigx, double *__restrict__ rl_out,
                                                      double *__restrict__ ru_out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  double rl, ru;
  recips(x[j], xl[j], xu[j], &rl, &ru);
  sigx[j] = sigma_of(rl, ru, zl[j], zu[j]);
  rl_out[j] = rl;
  ru_out[j] = ru;
}

// C = 1 / fma(delta_c, Sigma_s, e) with e = 1 + delta_c delta_w; for
// delta_c == 0 that is exactly 1 and the division is skipped (ZERO_DC).
template <bool ZERO_DC>
__global__ void __launch_bounds__(kBlock) k_prep_rows(int64_t m, const double *__restrict__ s,
                                                      const double *__restrict__ gl, const double *__restrict__ gu,
                                                      const double *__restrict__ zl, const double *__restrict__ zu,
                                                      double dw, double dc, double e, double eps,
                                                      double *__restrict__ dvec, double *__restrict__ cvec,
                                                      double *__restrict__ rl_out, double *__restrict__ ru_out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  double lo = gl[i], hi = gu[i];
  if (feq(lo, hi)) { lo = lo - eps; hi = hi + eps; }
  double rl, ru;
  recips(s[i], lo, hi, &rl, &ru);
  const double sg = sigma_of(rl, ru, zl[i], zu[i]);
  const double c = ZERO_DC ? 1.0 : 1.0 / fma(dc, sg, e);
  cvec[i] = c;
  dvec[i] = (sg + dw) * c;
  rl_out[i] = rl;
  ru_out[i] = ru;
}

// w = fma(C, q_s, D q_y) - y with q_s = fma(mu, ru - rl, y), q_y = c - s.
__global__ void __launch_bounds__(kBlock) k_rhs_rows(int64_t m, const double *__restrict__ s,
                                                     const double *__restrict__ y, const double *__restrict__ c,
                                                     const double *__restrict__ rl, const double *__restrict__ ru,
                                                     const double *__restrict__ dvec,
                                                     const double *__restrict__ cvec, double mu,
                                                     double *__restrict__ w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double yi = y[i];
  const double qs = fma(mu, ru[i] - rl[i], yi);
  const double qy = c[i] - s[i];
  w[i] = fma(cvec[i], qs, dvec[i] * qy) - yi;
}

// rhs = fma(mu, ru - rl, grad) + (J^T w), the product already in rhs.
__global__ void __launch_bounds__(kBlock) k_rhs_vars(int64_t n, const double *__restrict__ grad,
                                                     const double *__restrict__ rl, const double *__restrict__ ru,
                                                     double mu, double *__restrict__ rhs) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  rhs[j] = fma(mu, ru[j] - rl[j], grad[j]) + rhs[j];
}

// A zero reciprocal marks an infinite bound (finite bounds are strictly
// inactive, so their reciprocals are positive).
__global__ void __launch_bounds__(kBlock) k_rec_rows(int64_t m, const double *__restrict__ s,
                                                     const double *__restrict__ y, const double *__restrict__ c,
                                                     const double *__restrict__ zl, const double *__restrict__ zu,
                                                     const double *__restrict__ rlv, const double *__restrict__ ruv,
                                                     const double *__restrict__ cvec, double mu, double dw, double dc,
                                                     double *__restrict__ ds, double *__restrict__ dy,
                                                     double *__restrict__ dzl, double *__restrict__ dzu) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double rl = rlv[i], ru = ruv[i], zli = zl[i], zui = zu[i];
  const double sg = sigma_of(rl, ru, zli, zui);
  const double qs = fma(mu, ru - rl, y[i]);
  const double qy = c[i] - s[i];
  const double d = cvec[i] * (fma(dc, qs, ds[i]) - qy);  // ds holds J dx
  ds[i] = d;
  dy[i] = fma(sg + dw, d, -qs);
  dzl[i] = rl != 0.0 ? fma(-rl, fma(zli, d, mu), zli) : 0.0;
  dzu[i] = ru != 0.0 ? fma(-ru, fma(-zui, d, mu), zui) : 0.0;
}

__global__ void __launch_bounds__(kBlock) k_rec_vars(int64_t n, const double *__restrict__ zl,
                                                     const double *__restrict__ zu, const double *__restrict__ rlv,
                                                     const double *__restrict__ ruv, const double *__restrict__ dx,
                                                     double mu, double *__restrict__ dzl, double *__restrict__ dzu) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double rl = rlv[j], ru = ruv[j], v = dx[j];
  dzl[j] = rl != 0.0 ? fma(-rl, fma(zl[j], v, mu), zl[j]) : 0.0;
  dzu[j] = ru != 0.0 ? fma(-ru, fma(-zu[j], v, mu), zu[j]) : 0.0;
}

unsigned grid_for(int64_t count) { return (unsigned)((count + kBlock - 1) / kBlock); }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

int check_launch(const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return MPOPF_OK;
}

}  // namespace
}  // namespace mpopf

using namespace mpopf;

extern "C" {

int mpopf_ipm_prepare(mpopf_handle *h, const double *x, const double *s, const double *zl_x, const double *zu_x,
                      const double *zl_s, const double *zu_s, double delta_w, double delta_c, double eps_tol,
                      double *sigma_x, double *dvec, double *cvec, double *recip, void *stream) {
  if (!h || !x || !s || !zl_x || !zu_x || !zl_s || !zu_s || !sigma_x || !dvec || !cvec || !recip)
    return fail(MPOPF_ERR_ARG, "mpopf_ipm_prepare: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_ipm_prepare: not available on a period shard");
  const Dev &d = h->d;
  const mpopf_pattern &P = h->pat;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = d.n, m = d.m;
  const double e = 1.0 + delta_c * delta_w;
  if (n > 0) k_prep_vars<<<grid_for(n), kBlock, 0, st>>>(n, x, P.xl, P.xu, zl_x, zu_x, sigma_x, recip, recip + n);
  if (m > 0) {
    double *rl = recip + 2 * n, *ru = recip + 2 * n + m;
    if (delta_c == 0.0)
      k_prep_rows<true><<<grid_for(m), kBlock, 0, st>>>(m, s, P.gl, P.gu, zl_s, zu_s, delta_w, delta_c, e, eps_tol,
                                                        dvec, cvec, rl, ru);
    else
      k_prep_rows<false><<<grid_for(m), kBlock, 0, st>>>(m, s, P.gl, P.gu, zl_s, zu_s, delta_w, delta_c, e,
                                                         eps_tol, dvec, cvec, rl, ru);
  }
  return check_launch("mpopf_ipm_prepare");
}

int mpopf_ipm_rhs(mpopf_handle *h, const double *x, const double *jv, const double *s, const double *y,
                  const double *grad, const double *c, const double *recip, const double *dvec, const double *cvec,
                  double mu, double *rhs, void *stream) {
  if (!h || !x || !s || !y || !grad || !c || !recip || !dvec || !cvec || !rhs)
    return fail(MPOPF_ERR_ARG, "mpopf_ipm_rhs: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_ipm_rhs: not available on a period shard");
  const Dev &d = h->d;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = d.n, m = d.m;
  double *w = h->work;
  if (m > 0)
    k_rhs_rows<<<grid_for(m), kBlock, 0, st>>>(m, s, y, c, recip + 2 * n, recip + 2 * n + m, dvec, cvec, mu, w);
  int rc = check_launch("mpopf_ipm_rhs");
  if (rc != MPOPF_OK) return rc;
  rc = mpopf_vjp_jv(h, x, jv, w, rhs, nullptr, nullptr, stream);
  if (rc != MPOPF_OK) return rc;
  if (n > 0) k_rhs_vars<<<grid_for(n), kBlock, 0, st>>>(n, grad, recip, recip + n, mu, rhs);
  return check_launch("mpopf_ipm_rhs");
}

int mpopf_ipm_recover(mpopf_handle *h, const double *x, const double *jv, const double *s, const double *y,
                      const double *zl_x, const double *zu_x, const double *zl_s, const double *zu_s,
                      const double *c, const double *recip, const double *cvec, const double *dx, double mu,
                      double delta_w, double delta_c, double *ds, double *dy, double *dzl_x, double *dzu_x,
                      double *dzl_s, double *dzu_s, void *stream) {
  if (!h || !x || !s || !y || !zl_x || !zu_x || !zl_s || !zu_s || !c || !recip || !cvec || !dx || !ds || !dy ||
      !dzl_x || !dzu_x || !dzl_s || !dzu_s)
    return fail(MPOPF_ERR_ARG, "mpopf_ipm_recover: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_ipm_recover: not available on a period shard");
  const Dev &d = h->d;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = d.n, m = d.m;
  int rc = mpopf_jvp_jv(h, x, jv, dx, nullptr, nullptr, ds, stream);  // ds = J dx
  if (rc != MPOPF_OK) return rc;
  if (m > 0)
    k_rec_rows<<<grid_for(m), kBlock, 0, st>>>(m, s, y, c, zl_s, zu_s, recip + 2 * n, recip + 2 * n + m, cvec, mu,
                                               delta_w, delta_c, ds, dy, dzl_s, dzu_s);
  if (n > 0) k_rec_vars<<<grid_for(n), kBlock, 0, st>>>(n, zl_x, zu_x, recip, recip + n, dx, mu, dzl_x, dzu_x);
  return check_launch("mpopf_ipm_recover");
}

}  // extern "C"
