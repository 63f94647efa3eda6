// Interior-point algebra around the condensed matrix (Sec. III-B of the paper):
// the diagonal scalings Sigma_x, Sigma_s, C, D from the bounds and duals (with
// the relaxation of equality rows to [g - eps, g + eps]), the condensed
// right-hand side q_x + A^T (C q_s + D q_y), and the recovery of the slack,
// multiplier and bound-dual steps from dx.  Elementwise kernels plus the
// matrix-free J^T w / J v kernels; every value follows the same written order
// as the CPU oracle.  The recovered slack step is the one Eq. (5) implies,
// ds = C (A dx + delta_c q_s - q_y); the printed form with -A dx does not solve
// the printed block system.
#include <string>

#include "mpopf_internal.cuh"

extern "C" int mpopf_vjp(mpopf_handle *h, const double *x, const double *y, double *gx, double *gpd, double *gqd,
                         void *stream);
extern "C" int mpopf_jvp(mpopf_handle *h, const double *x, const double *v, const double *dpd, const double *dqd,
                         double *jv_out, void *stream);

namespace mpopf {
namespace {

__device__ __forceinline__ bool finite(double v) {
  return ((__double2hiint(v) >> 20) & 0x7ff) != 0x7ff;
}

struct Barrier {
  double sig, pzl, pzu, dl, du;
  bool has_l, has_u;
};

// Sigma = zl/(v - lo) + zu/(hi - v); pzl = fma(zl, v - lo, -mu), pzu = fma(zu, hi - v, -mu).
__device__ __forceinline__ Barrier barrier(double v, double lo, double hi, double zl, double zu, double mu) {
  Barrier b;
  b.has_l = finite(lo);
  b.has_u = finite(hi);
  b.pzl = b.pzu = b.dl = b.du = 0.0;
  double a = 0.0, c = 0.0;
  if (b.has_l) { b.dl = v - lo; a = zl / b.dl; b.pzl = fma(zl, b.dl, -mu); }
  if (b.has_u) { b.du = hi - v; c = zu / b.du; b.pzu = fma(zu, b.du, -mu); }
  b.sig = a + c;
  return b;
}

__device__ __forceinline__ void slack_bounds(double gl, double gu, double eps, double *sl, double *su) {
  if (gl == gu) { *sl = gl - eps; *su = gu + eps; } else { *sl = gl; *su = gu; }
}

__global__ void __launch_bounds__(kBlock) k_prep_vars(int64_t n, const double *__restrict__ x,
                                                      const double *__restrict__ xl, const double *__restrict__ xu,
                                                      const double *__restrict__ zl, const double *__restrict__ zu,
                                                      double *__restrict__ sigx) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  sigx[j] = barrier(x[j], xl[j], xu[j], zl[j], zu[j], 0.0).sig;
}

__global__ void __launch_bounds__(kBlock) k_prep_rows(int64_t m, const double *__restrict__ s,
                                                      const double *__restrict__ gl, const double *__restrict__ gu,
                                                      const double *__restrict__ zl, const double *__restrict__ zu,
                                                      double dw, double dc, double e, double eps,
                                                      double *__restrict__ dvec, double *__restrict__ cvec) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  double sl, su;
  slack_bounds(gl[i], gu[i], eps, &sl, &su);
  const double sg = barrier(s[i], sl, su, zl[i], zu[i], 0.0).sig;
  const double c = 1.0 / fma(dc, sg, e);
  cvec[i] = c;
  dvec[i] = (sg + dw) * c;
}

// q_s, q_y and the barrier terms of row i.
struct RowQ {
  double qs, qy, sig, cc;
  Barrier b;
};
__device__ __forceinline__ RowQ row_q(int64_t i, const double *s, const double *y, const double *gl, const double *gu,
                                      const double *zl, const double *zu, const double *c, double mu, double dc,
                                      double e, double eps) {
  RowQ r;
  double sl, su;
  slack_bounds(gl[i], gu[i], eps, &sl, &su);
  r.b = barrier(s[i], sl, su, zl[i], zu[i], mu);
  double qs = (zu[i] - zl[i]) + y[i];
  qs = qs + (r.b.has_l ? r.b.pzl / r.b.dl : 0.0);
  qs = qs - (r.b.has_u ? r.b.pzu / r.b.du : 0.0);
  r.qs = qs;
  r.qy = c[i] - s[i];
  r.sig = r.b.sig;
  r.cc = 1.0 / fma(dc, r.b.sig, e);
  return r;
}

__global__ void __launch_bounds__(kBlock) k_rhs_rows(int64_t m, const double *__restrict__ s,
                                                     const double *__restrict__ y, const double *__restrict__ gl,
                                                     const double *__restrict__ gu, const double *__restrict__ zl,
                                                     const double *__restrict__ zu, const double *__restrict__ c,
                                                     double mu, double dw, double dc, double e, double eps,
                                                     double *__restrict__ w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const RowQ r = row_q(i, s, y, gl, gu, zl, zu, c, mu, dc, e, eps);
  const double dd = (r.sig + dw) * r.cc;
  w[i] = fma(r.cc, r.qs, dd * r.qy) - y[i];
}

__global__ void __launch_bounds__(kBlock) k_rhs_vars(int64_t n, const double *__restrict__ x,
                                                     const double *__restrict__ xl, const double *__restrict__ xu,
                                                     const double *__restrict__ zl, const double *__restrict__ zu,
                                                     const double *__restrict__ grad, double mu,
                                                     double *__restrict__ rhs) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Barrier b = barrier(x[j], xl[j], xu[j], zl[j], zu[j], mu);
  double base = (grad[j] - zl[j]) + zu[j];
  base = base + (b.has_l ? b.pzl / b.dl : 0.0);
  base = base - (b.has_u ? b.pzu / b.du : 0.0);
  rhs[j] = base + rhs[j];  // rhs holds J^T w
}

__global__ void __launch_bounds__(kBlock) k_rec_rows(int64_t m, const double *__restrict__ s,
                                                     const double *__restrict__ y, const double *__restrict__ gl,
                                                     const double *__restrict__ gu, const double *__restrict__ zl,
                                                     const double *__restrict__ zu, const double *__restrict__ c,
                                                     double mu, double dw, double dc, double e, double eps,
                                                     double *__restrict__ ds, double *__restrict__ dy,
                                                     double *__restrict__ dzl, double *__restrict__ dzu) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const RowQ r = row_q(i, s, y, gl, gu, zl, zu, c, mu, dc, e, eps);
  const double d = r.cc * (fma(dc, r.qs, ds[i]) - r.qy);  // ds holds J dx
  ds[i] = d;
  dy[i] = fma(r.sig + dw, d, -r.qs);
  dzl[i] = r.b.has_l ? fma(-zl[i], d, r.b.pzl) / r.b.dl : 0.0;
  dzu[i] = r.b.has_u ? fma(zu[i], d, r.b.pzu) / r.b.du : 0.0;
}

__global__ void __launch_bounds__(kBlock) k_rec_vars(int64_t n, const double *__restrict__ x,
                                                     const double *__restrict__ xl, const double *__restrict__ xu,
                                                     const double *__restrict__ zl, const double *__restrict__ zu,
                                                     const double *__restrict__ dx, double mu,
                                                     double *__restrict__ dzl, double *__restrict__ dzu) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Barrier b = barrier(x[j], xl[j], xu[j], zl[j], zu[j], mu);
  dzl[j] = b.has_l ? fma(-zl[j], dx[j], b.pzl) / b.dl : 0.0;
  dzu[j] = b.has_u ? fma(zu[j], dx[j], b.pzu) / b.du : 0.0;
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
                      double *sigma_x, double *dvec, double *cvec, void *stream) {
  if (!h || !x || !s || !zl_x || !zu_x || !zl_s || !zu_s || !sigma_x || !dvec || !cvec)
    return fail(MPOPF_ERR_ARG, "mpopf_ipm_prepare: NULL argument");
  const Dev &d = h->d;
  const mpopf_pattern &P = h->pat;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double e = 1.0 + delta_c * delta_w;
  if (d.n > 0) k_prep_vars<<<grid_for(d.n), kBlock, 0, st>>>(d.n, x, P.xl, P.xu, zl_x, zu_x, sigma_x);
  if (d.m > 0)
    k_prep_rows<<<grid_for(d.m), kBlock, 0, st>>>(d.m, s, P.gl, P.gu, zl_s, zu_s, delta_w, delta_c, e, eps_tol, dvec,
                                                  cvec);
  return check_launch("mpopf_ipm_prepare");
}

int mpopf_ipm_rhs(mpopf_handle *h, const double *x, const double *s, const double *y, const double *zl_x,
                  const double *zu_x, const double *zl_s, const double *zu_s, const double *grad, const double *c,
                  double mu, double delta_w, double delta_c, double eps_tol, double *rhs, void *stream) {
  if (!h || !x || !s || !y || !zl_x || !zu_x || !zl_s || !zu_s || !grad || !c || !rhs)
    return fail(MPOPF_ERR_ARG, "mpopf_ipm_rhs: NULL argument");
  const Dev &d = h->d;
  const mpopf_pattern &P = h->pat;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double e = 1.0 + delta_c * delta_w;
  double *w = h->work;
  if (d.m > 0)
    k_rhs_rows<<<grid_for(d.m), kBlock, 0, st>>>(d.m, s, y, P.gl, P.gu, zl_s, zu_s, c, mu, delta_w, delta_c, e,
                                                 eps_tol, w);
  int rc = check_launch("mpopf_ipm_rhs");
  if (rc != MPOPF_OK) return rc;
  rc = mpopf_vjp(h, x, w, rhs, nullptr, nullptr, stream);
  if (rc != MPOPF_OK) return rc;
  if (d.n > 0) k_rhs_vars<<<grid_for(d.n), kBlock, 0, st>>>(d.n, x, P.xl, P.xu, zl_x, zu_x, grad, mu, rhs);
  return check_launch("mpopf_ipm_rhs");
}

int mpopf_ipm_recover(mpopf_handle *h, const double *x, const double *s, const double *y, const double *zl_x,
                      const double *zu_x, const double *zl_s, const double *zu_s, const double *c, const double *dx,
                      double mu, double delta_w, double delta_c, double eps_tol, double *ds, double *dy,
                      double *dzl_x, double *dzu_x, double *dzl_s, double *dzu_s, void *stream) {
  if (!h || !x || !s || !y || !zl_x || !zu_x || !zl_s || !zu_s || !c || !dx || !ds || !dy || !dzl_x || !dzu_x ||
      !dzl_s || !dzu_s)
    return fail(MPOPF_ERR_ARG, "mpopf_ipm_recover: NULL argument");
  const Dev &d = h->d;
  const mpopf_pattern &P = h->pat;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double e = 1.0 + delta_c * delta_w;
  int rc = mpopf_jvp(h, x, dx, nullptr, nullptr, ds, stream);  // ds = J dx
  if (rc != MPOPF_OK) return rc;
  if (d.m > 0)
    k_rec_rows<<<grid_for(d.m), kBlock, 0, st>>>(d.m, s, y, P.gl, P.gu, zl_s, zu_s, c, mu, delta_w, delta_c, e,
                                                 eps_tol, ds, dy, dzl_s, dzu_s);
  if (d.n > 0) k_rec_vars<<<grid_for(d.n), kBlock, 0, st>>>(d.n, x, P.xl, P.xu, zl_x, zu_x, dx, mu, dzl_x, dzu_x);
  return check_launch("mpopf_ipm_recover");
}

}  // extern "C"
