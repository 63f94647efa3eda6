// Matrix-free derivative products of libmpopf (sm_103a, FP64): J^T y with the
// load adjoint, J v with load tangents, and W v -- without materialising J or W.
//
// Same decomposition as the sweep: a branch x period kernel computes the branch
// element's local values (the flow terms and their derivatives, recomputed from
// x), writes the arc variables' results and one incidence record per branch end;
// a bus x period kernel sums its records in branch order (no atomics); a
// generator x period kernel handles pg/qg.  Every value follows the fixed
// rounding order of the definitions (element-local sums in the row order, then
// added in element order), so results are bitwise reproducible.
#include "mpopf_device.cuh"

namespace mpopf {
namespace {

// CTA size of the product kernels (per-element kernels; 48 registers or
// fewer): 128 measured J v 0.433 ms against 0.438 ms at 256 and 0.435 ms at 64
// (10k buses x 168); J^T y and W v within 0.3%.
#ifndef MPOPF_ADJ_BLOCK
#define MPOPF_ADJ_BLOCK 128
#endif
constexpr int kAdjBlock = MPOPF_ADJ_BLOCK;

// ---------------------------------------------------------------------------
// J^T y.  Branch element local sums over its rows K1..K7:
//   va_f: a1 y1, + a2 y2, + a3 y3, + a4 y4, + y5   (va_t: the exact negation)
//   vm_f: b_k y_k (k = 1..4);  vm_t: c_k y_k
//   p_f: fma(2pf, y6, y1);  q_f: fma(2qf, y6, y2);  p_t: fma(2pt, y7, y3);
//   q_t: fma(2qt, y7, y4); then the bus element adds -y8 (p) or -y9 (q).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjBlock) k_vjp_branch(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ y, double *__restrict__ gx) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t TL = (int64_t)d.T * L, tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const double vf = __ldg(x + d.x_vm + tN + f), vt = __ldg(x + d.x_vm + tN + to);
  const Flow F = flow_terms(d, l, __ldg(x + tN + f), __ldg(x + tN + to), vf, vt);
  const FlowJ J = flow_jac(d, l, F, vf, vt);
  const int64_t rk1 = d.T + tl;
  const double y1 = __ldg(y + rk1), y2 = __ldg(y + rk1 + TL), y3 = __ldg(y + rk1 + 2 * TL);
  const double y4 = __ldg(y + rk1 + 3 * TL), y5 = __ldg(y + rk1 + 4 * TL), y6 = __ldg(y + rk1 + 5 * TL);
  const double y7 = __ldg(y + rk1 + 6 * TL);
  const double Ld = fma(J.a4, y4, fma(J.a3, y3, fma(J.a2, y2, J.a1 * y1))) + y5;
  const double Lvf = fma(J.b4, y4, fma(J.b3, y3, fma(J.b2, y2, J.b1 * y1)));
  const double Lvt = fma(J.c4, y4, fma(J.c3, y3, fma(J.c2, y2, J.c1 * y1)));
  const double pf = __ldg(x + pb + l), pt = __ldg(x + pb + L + l);
  const double qf = __ldg(x + qb + l), qt = __ldg(x + qb + L + l);
  const int64_t r8f = d.c_k8 + tN + f, r8t = d.c_k8 + tN + to, d89 = d.c_k9 - d.c_k8;
  gx[pb + l] = fma(twice(pf), y6, y1) - __ldg(y + r8f);
  gx[qb + l] = fma(twice(qf), y6, y2) - __ldg(y + r8f + d89);
  gx[pb + L + l] = fma(twice(pt), y7, y3) - __ldg(y + r8t);
  gx[qb + L + l] = fma(twice(qt), y7, y4) - __ldg(y + r8t + d89);
  double *R = d.S + (int64_t)t * 2 * L * kRec;
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * kRec) = make_double2(Ld, Lvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * kRec) = make_double2(negx(Ld), Lvt);
}

__global__ void __launch_bounds__(kAdjBlock) k_vjp_bus(Dev d, const double *__restrict__ x,
                                                    const double *__restrict__ y, double *__restrict__ gx,
                                                    double *__restrict__ gpd, double *__restrict__ gqd) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int32_t s0 = __ldg(d.inc_ptr + pos), s1 = __ldg(d.inc_ptr + pos + 1);
  const double *R = d.S + (int64_t)t * 2 * d.L * kRec;
  // va: reference element first, then the incident branches in branch order.
  double ga = 0.0, gv = 0.0;
  bool has_a = false, has_v = false;
  if (n == d.ref) { ga = __ldg(y + t); has_a = true; }
  for (int32_t q = s0; q < s1; ++q) {
    const double2 r = __ldg(reinterpret_cast<const double2 *>(R + (int64_t)q * kRec));
    ga = has_a ? ga + r.x : r.x;
    gv = has_v ? gv + r.y : r.y;
    has_a = has_v = true;
  }
  // vm: then the bus element (rows K8, K9).
  const double vm = __ldg(x + d.x_vm + tn);
  const double y8 = __ldg(y + d.c_k8 + tn), y9 = __ldg(y + d.c_k9 + tn);
  const double Lbus = fma(__ldg(d.bus_p2bs + n) * vm, y9, (__ldg(d.bus_m2gs + n) * vm) * y8);
  gv = has_v ? gv + Lbus : Lbus;
  gx[tn] = ga;
  gx[d.x_vm + tn] = gv;
  if (gpd) {
    const int64_t ldb = (int64_t)t * d.D;
    for (int32_t e = __ldg(d.bload_ptr + n); e < __ldg(d.bload_ptr + n + 1); ++e) {
      const int32_t k = __ldg(d.bload_idx + e);
      gpd[ldb + k] = negx(y8);
      gqd[ldb + k] = negx(y9);
    }
  }
}

__global__ void __launch_bounds__(kAdjBlock) k_vjp_gen(Dev d, const double *__restrict__ y, double *__restrict__ gx) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= d.T * G) return;
  const int32_t t = tg / G, g = tg - t * G;
  const int64_t tn = (int64_t)t * d.N + __ldg(d.gen_bus + g);
  double a = __ldg(y + d.c_k8 + tn);  // bus element (K8, entry +1)
  const int64_t rr = d.c_k10 + (int64_t)(t - 1) * G + g;
  if (t >= 1) a = a + __ldg(y + rr);         // ramp row (t, g): +1
  if (t + 1 < d.T) a = a - __ldg(y + rr + G);  // ramp row (t + 1, g): -1
  gx[d.x_pg + tg] = a;
  double b = __ldg(y + d.c_k9 + tn);  // bus element (K9, entry +1)
  if (d.qramp) {
    const int64_t rq = d.c_k11 + (int64_t)(t - 1) * G + g;
    if (t >= 1) b = b + __ldg(y + rq);         // reactive ramp row (t, g): +1
    if (t + 1 < d.T) b = b - __ldg(y + rq + G);  // reactive ramp row (t + 1, g): -1
  }
  gx[d.x_qg + tg] = b;
}

// ---------------------------------------------------------------------------
// J v (+ load tangents): one row at a time in its J order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjBlock) k_jvp_branch(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ v, double *__restrict__ out) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t TL = (int64_t)d.T * L, tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const double vf = __ldg(x + d.x_vm + tN + f), vt = __ldg(x + d.x_vm + tN + to);
  const Flow F = flow_terms(d, l, __ldg(x + tN + f), __ldg(x + tN + to), vf, vt);
  const FlowJ J = flow_jac(d, l, F, vf, vt);
  const double uf = __ldg(v + tN + f), ut = __ldg(v + tN + to);
  const double wf = __ldg(v + d.x_vm + tN + f), wt = __ldg(v + d.x_vm + tN + to);
  const double vpf = __ldg(v + pb + l), vpt = __ldg(v + pb + L + l);
  const double vqf = __ldg(v + qb + l), vqt = __ldg(v + qb + L + l);
  const int64_t rk1 = d.T + tl;
  out[rk1] = fma(J.c1, wt, fma(J.b1, wf, fma(negx(J.a1), ut, fma(J.a1, uf, vpf))));
  out[rk1 + TL] = fma(J.c2, wt, fma(J.b2, wf, fma(negx(J.a2), ut, fma(J.a2, uf, vqf))));
  out[rk1 + 2 * TL] = fma(J.c3, wt, fma(J.b3, wf, fma(negx(J.a3), ut, fma(J.a3, uf, vpt))));
  out[rk1 + 3 * TL] = fma(J.c4, wt, fma(J.b4, wf, fma(negx(J.a4), ut, fma(J.a4, uf, vqt))));
  out[rk1 + 4 * TL] = uf - ut;
  const double pf = __ldg(x + pb + l), pt = __ldg(x + pb + L + l);
  const double qf = __ldg(x + qb + l), qt = __ldg(x + qb + L + l);
  out[rk1 + 5 * TL] = fma(twice(qf), vqf, twice(pf) * vpf);
  out[rk1 + 6 * TL] = fma(twice(qt), vqt, twice(pt) * vpt);
}

__global__ void __launch_bounds__(kAdjBlock) k_jvp_bus(Dev d, const double *__restrict__ x,
                                                    const double *__restrict__ v, const double *__restrict__ dpd,
                                                    const double *__restrict__ dqd, double *__restrict__ out) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int64_t L = d.L, G = d.G;
  if (n == d.ref) out[t] = __ldg(v + (int64_t)t * N + n);
  const double vm = __ldg(x + d.x_vm + tn), dvm = __ldg(v + d.x_vm + tn);
  double aP = (__ldg(d.bus_m2gs + n) * vm) * dvm, aQ = (__ldg(d.bus_p2bs + n) * vm) * dvm;
  const int64_t pgb = d.x_pg + (int64_t)t * G, qgb = d.x_qg + (int64_t)t * G;
  for (int32_t e = __ldg(d.bgen_ptr + n); e < __ldg(d.bgen_ptr + n + 1); ++e) {
    const int32_t g = __ldg(d.bgen_idx + e);
    aP = aP + __ldg(v + pgb + g);
    aQ = aQ + __ldg(v + qgb + g);
  }
  const int64_t pab = d.x_p + 2 * (int64_t)t * L, qab = d.x_q + 2 * (int64_t)t * L;
  for (int32_t e = __ldg(d.barc_ptr + n); e < __ldg(d.barc_ptr + n + 1); ++e) {
    const int32_t a = __ldg(d.barc_idx + e);
    aP = aP - __ldg(v + pab + a);
    aQ = aQ - __ldg(v + qab + a);
  }
  if (dpd) {
    const int64_t ldb = (int64_t)t * d.D;
    for (int32_t e = __ldg(d.bload_ptr + n); e < __ldg(d.bload_ptr + n + 1); ++e) {
      const int32_t k = __ldg(d.bload_idx + e);
      aP = aP - __ldg(dpd + ldb + k);
      aQ = aQ - __ldg(dqd + ldb + k);
    }
  }
  out[d.c_k8 + tn] = aP;
  out[d.c_k9 + tn] = aQ;
}

__global__ void __launch_bounds__(kAdjBlock) k_jvp_gen(Dev d, const double *__restrict__ v, double *__restrict__ out) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= (d.T - 1) * G) return;  // ramp rows (t, g), t = 1..T-1, row index (t - 1) G + g
  const int64_t cur = d.x_pg + G + tg;
  out[d.c_k10 + tg] = __ldg(v + cur) - __ldg(v + cur - G);
  if (d.qramp) {
    const int64_t qc = d.x_qg + G + tg;
    out[d.c_k11 + tg] = __ldg(v + qc) - __ldg(v + qc - G);
  }
}

// ---------------------------------------------------------------------------
// W v.  Branch element: its W entries in order (block (0,0)..(3,3), then the
// thermal diagonals), each entry (r, c, w) adding fma(w, v[c], .) to r and,
// off the diagonal, fma(w, v[r], .) to c.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjBlock) k_hvp_branch(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ lam, const double *__restrict__ v,
                                                       double *__restrict__ hv) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t TL = (int64_t)d.T * L, tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const double vf = __ldg(x + d.x_vm + tN + f), vt = __ldg(x + d.x_vm + tN + to);
  const Flow F = flow_terms(d, l, __ldg(x + tN + f), __ldg(x + tN + to), vf, vt);
  const int64_t rk1 = d.T + tl;
  const FlowW W = flow_hess(d, l, F, vf, vt, __ldg(lam + rk1), __ldg(lam + rk1 + TL), __ldg(lam + rk1 + 2 * TL),
                            __ldg(lam + rk1 + 3 * TL));
  const double uf = __ldg(v + tN + f), ut = __ldg(v + tN + to);
  const double wf = __ldg(v + d.x_vm + tN + f), wt = __ldg(v + d.x_vm + tN + to);
  const double nWdd = negx(W.Wdd), nWdvf = negx(W.Wdvf), nWdvt = negx(W.Wdvt), nAsum = negx(W.Asum);
  const double hf = fma(W.Wdvt, wt, fma(W.Wdvf, wf, fma(nWdd, ut, W.Wdd * uf)));
  const double ht = fma(nWdvt, wt, fma(nWdvf, wf, fma(W.Wdd, ut, nWdd * uf)));
  const double hvf = fma(nAsum, wt, fma(W.Wvfvf, wf, fma(nWdvf, ut, W.Wdvf * uf)));
  const double hvt = fma(W.Wvtvt, wt, fma(nAsum, wf, fma(nWdvt, ut, W.Wdvt * uf)));
  const double h6 = twice(__ldg(lam + rk1 + 5 * TL)), h7 = twice(__ldg(lam + rk1 + 6 * TL));
  hv[pb + l] = h6 * __ldg(v + pb + l);
  hv[qb + l] = h6 * __ldg(v + qb + l);
  hv[pb + L + l] = h7 * __ldg(v + pb + L + l);
  hv[qb + L + l] = h7 * __ldg(v + qb + L + l);
  double *R = d.S + (int64_t)t * 2 * L * kRec;
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * kRec) = make_double2(hf, hvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * kRec) = make_double2(ht, hvt);
}

__global__ void __launch_bounds__(kAdjBlock) k_hvp_bus(Dev d, const double *__restrict__ lam,
                                                    const double *__restrict__ v, double *__restrict__ hv) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int32_t s0 = __ldg(d.inc_ptr + pos), s1 = __ldg(d.inc_ptr + pos + 1);
  const double *R = d.S + (int64_t)t * 2 * d.L * kRec;
  double ha = 0.0, hm = 0.0;
  for (int32_t q = s0; q < s1; ++q) {
    const double2 r = __ldg(reinterpret_cast<const double2 *>(R + (int64_t)q * kRec));
    ha = (q == s0) ? r.x : ha + r.x;
    hm = (q == s0) ? r.y : hm + r.y;
  }
  const double dvm = __ldg(v + d.x_vm + tn);
  const double WP = __ldg(lam + d.c_k8 + tn) * __ldg(d.bus_m2gs + n);
  const double WQ = __ldg(lam + d.c_k9 + tn) * __ldg(d.bus_p2bs + n);
  const double Lbus = fma(WQ, dvm, WP * dvm);
  hv[tn] = ha;
  hv[d.x_vm + tn] = (s1 > s0) ? hm + Lbus : Lbus;
}

__global__ void __launch_bounds__(kAdjBlock) k_hvp_gen(Dev d, double sigma, const double *__restrict__ v,
                                                    double *__restrict__ hv) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= d.T * G) return;
  const int32_t g = tg % G;
  hv[d.x_pg + tg] = (sigma * __ldg(d.gen_c2x2 + g)) * __ldg(v + d.x_pg + tg);
  hv[d.x_qg + tg] = 0.0;
}

// ---------------------------------------------------------------------------
// The same two branch kernels reading J's values as the sweep wrote them
// (K1..K4 rows [1, a, -a, b, c], K5 [1, -1], K6/K7 [2p, 2q]) instead of
// recomputing the flow derivatives: identical sums in identical order, so the
// results equal those of k_vjp_branch / k_jvp_branch bit for bit when jv was
// evaluated at the same x.  Bus and generator kernels are shared.
// ---------------------------------------------------------------------------
struct StoredJ {
  double a1, b1, c1, na1, a2, b2, c2, na2, a3, b3, c3, na3, a4, b4, c4, na4, jp6, jq6, jp7, jq7;
};

__device__ __forceinline__ StoredJ stored_j(const Dev &d, const double *__restrict__ jv, int32_t tl) {
  const int64_t s5 = 5 * (int64_t)d.T * d.L;
  const double *j1 = jv + d.T + (int64_t)tl * 5;
  StoredJ J;
  J.a1 = __ldg(j1 + 1); J.na1 = __ldg(j1 + 2); J.b1 = __ldg(j1 + 3); J.c1 = __ldg(j1 + 4);
  J.a2 = __ldg(j1 + s5 + 1); J.na2 = __ldg(j1 + s5 + 2); J.b2 = __ldg(j1 + s5 + 3); J.c2 = __ldg(j1 + s5 + 4);
  J.a3 = __ldg(j1 + 2 * s5 + 1); J.na3 = __ldg(j1 + 2 * s5 + 2); J.b3 = __ldg(j1 + 2 * s5 + 3);
  J.c3 = __ldg(j1 + 2 * s5 + 4);
  J.a4 = __ldg(j1 + 3 * s5 + 1); J.na4 = __ldg(j1 + 3 * s5 + 2); J.b4 = __ldg(j1 + 3 * s5 + 3);
  J.c4 = __ldg(j1 + 3 * s5 + 4);
  // scalar loads: the K6/K7 blocks start at odd offsets when T is odd
  const double *j6 = jv + d.j_k6 + (int64_t)tl * 2, *j7 = jv + d.j_k7 + (int64_t)tl * 2;
  J.jp6 = __ldg(j6); J.jq6 = __ldg(j6 + 1); J.jp7 = __ldg(j7); J.jq7 = __ldg(j7 + 1);
  return J;
}

__global__ void __launch_bounds__(kAdjBlock) k_vjp_branch_jv(Dev d, const double *__restrict__ jv,
                                                          const double *__restrict__ y, double *__restrict__ gx) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t TL = (int64_t)d.T * L, tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const StoredJ J = stored_j(d, jv, tl);
  const int64_t rk1 = d.T + tl;
  const double y1 = __ldg(y + rk1), y2 = __ldg(y + rk1 + TL), y3 = __ldg(y + rk1 + 2 * TL);
  const double y4 = __ldg(y + rk1 + 3 * TL), y5 = __ldg(y + rk1 + 4 * TL), y6 = __ldg(y + rk1 + 5 * TL);
  const double y7 = __ldg(y + rk1 + 6 * TL);
  const double Ld = fma(J.a4, y4, fma(J.a3, y3, fma(J.a2, y2, J.a1 * y1))) + y5;
  const double Lvf = fma(J.b4, y4, fma(J.b3, y3, fma(J.b2, y2, J.b1 * y1)));
  const double Lvt = fma(J.c4, y4, fma(J.c3, y3, fma(J.c2, y2, J.c1 * y1)));
  const int64_t r8f = d.c_k8 + tN + f, r8t = d.c_k8 + tN + to, d89 = d.c_k9 - d.c_k8;
  gx[pb + l] = fma(J.jp6, y6, y1) - __ldg(y + r8f);
  gx[qb + l] = fma(J.jq6, y6, y2) - __ldg(y + r8f + d89);
  gx[pb + L + l] = fma(J.jp7, y7, y3) - __ldg(y + r8t);
  gx[qb + L + l] = fma(J.jq7, y7, y4) - __ldg(y + r8t + d89);
  double *R = d.S + (int64_t)t * 2 * L * kRec;
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * kRec) = make_double2(Ld, Lvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * kRec) = make_double2(negx(Ld), Lvt);
}

__global__ void __launch_bounds__(kAdjBlock) k_jvp_branch_jv(Dev d, const double *__restrict__ jv,
                                                          const double *__restrict__ v, double *__restrict__ out) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t TL = (int64_t)d.T * L, tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const StoredJ J = stored_j(d, jv, tl);
  const double uf = __ldg(v + tN + f), ut = __ldg(v + tN + to);
  const double wf = __ldg(v + d.x_vm + tN + f), wt = __ldg(v + d.x_vm + tN + to);
  const double vpf = __ldg(v + pb + l), vpt = __ldg(v + pb + L + l);
  const double vqf = __ldg(v + qb + l), vqt = __ldg(v + qb + L + l);
  const int64_t rk1 = d.T + tl;
  out[rk1] = fma(J.c1, wt, fma(J.b1, wf, fma(J.na1, ut, fma(J.a1, uf, vpf))));
  out[rk1 + TL] = fma(J.c2, wt, fma(J.b2, wf, fma(J.na2, ut, fma(J.a2, uf, vqf))));
  out[rk1 + 2 * TL] = fma(J.c3, wt, fma(J.b3, wf, fma(J.na3, ut, fma(J.a3, uf, vpt))));
  out[rk1 + 3 * TL] = fma(J.c4, wt, fma(J.b4, wf, fma(J.na4, ut, fma(J.a4, uf, vqt))));
  out[rk1 + 4 * TL] = uf - ut;
  out[rk1 + 5 * TL] = fma(J.jq6, vqf, J.jp6 * vpf);
  out[rk1 + 6 * TL] = fma(J.jq7, vqt, J.jp7 * vpt);
}

// Vectors per thread of the products for several vectors at one point.
#ifndef MPOPF_MANY_NV
#define MPOPF_MANY_NV 4
#endif
constexpr int kManyNV = MPOPF_MANY_NV;

// The products for nvec vectors at one point (the _many kernels; the single
// products' kernels above keep their own register allocation): a thread
// takes vectors blockIdx.y NV + i (i < NV, below nvec), vector j reading and
// writing the j-th of consecutive arrays of the single product's sizes, with
// its element's point-dependent values loaded (or recomputed) once for all of
// them.  Incidence records: one double2 per branch end, in a packed array of
// their own (vector j's T periods after the earlier vectors'); the templates
// also take NV = 0, which would be the single products' layout (the sweep's
// record array, kRec doubles apart).
template <int NV>
__host__ __device__ constexpr int rec_stride() {
  return NV ? 2 : kRec;
}
template <int NV>
__device__ __forceinline__ double *prod_rec(const Dev &d, int32_t t, int64_t j) {
  return d.S + ((NV ? j * d.T : 0) + t) * 2 * d.L * rec_stride<NV>();
}
template <int NV>
__host__ __device__ constexpr int vec_count() {
  return NV ? NV : 1;
}
// The thread's i-th vector, or -1 past the last one.
template <int NV>
__device__ __forceinline__ int64_t vec_index(int i, int32_t nvec) {
  if (!NV) return 0;
  const int64_t j = (int64_t)blockIdx.y * NV + i;
  return j < nvec ? j : -1;
}

// ---------------------------------------------------------------------------
// J^T y.  Branch element local sums over its rows K1..K7:
//   va_f: a1 y1, + a2 y2, + a3 y3, + a4 y4, + y5   (va_t: the exact negation)
//   vm_f: b_k y_k (k = 1..4);  vm_t: c_k y_k
//   p_f: fma(2pf, y6, y1);  q_f: fma(2qf, y6, y2);  p_t: fma(2pt, y7, y3);
//   q_t: fma(2qt, y7, y4); then the bus element adds -y8 (p) or -y9 (q).
// ---------------------------------------------------------------------------
// The branch rows' J values of an element (recomputed from x, or read from a
// stored J by the _jv kernels below).
struct BranchJ {
  double a1, b1, c1, a2, b2, c2, a3, b3, c3, a4, b4, c4, jp6, jq6, jp7, jq7;
};

// J^T y of one vector for a branch element with J values J.
template <int NV>
__device__ __forceinline__ void vjp_branch_vec(const Dev &d, const BranchJ &J, int32_t t, int32_t l, int32_t f,
                                               int32_t to, const double *__restrict__ y, double *__restrict__ gx,
                                               int64_t j) {
  const int32_t L = d.L;
  const int64_t TL = (int64_t)d.T * L, tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int64_t rk1 = d.T + (int64_t)t * L + l;
  const double y1 = __ldg(y + rk1), y2 = __ldg(y + rk1 + TL), y3 = __ldg(y + rk1 + 2 * TL);
  const double y4 = __ldg(y + rk1 + 3 * TL), y5 = __ldg(y + rk1 + 4 * TL), y6 = __ldg(y + rk1 + 5 * TL);
  const double y7 = __ldg(y + rk1 + 6 * TL);
  const double Ld = fma(J.a4, y4, fma(J.a3, y3, fma(J.a2, y2, J.a1 * y1))) + y5;
  const double Lvf = fma(J.b4, y4, fma(J.b3, y3, fma(J.b2, y2, J.b1 * y1)));
  const double Lvt = fma(J.c4, y4, fma(J.c3, y3, fma(J.c2, y2, J.c1 * y1)));
  const int64_t r8f = d.c_k8 + tN + f, r8t = d.c_k8 + tN + to, d89 = d.c_k9 - d.c_k8;
  gx[pb + l] = fma(J.jp6, y6, y1) - __ldg(y + r8f);
  gx[qb + l] = fma(J.jq6, y6, y2) - __ldg(y + r8f + d89);
  gx[pb + L + l] = fma(J.jp7, y7, y3) - __ldg(y + r8t);
  gx[qb + L + l] = fma(J.jq7, y7, y4) - __ldg(y + r8t + d89);
  double *R = prod_rec<NV>(d, t, j);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * rec_stride<NV>()) = make_double2(Ld, Lvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * rec_stride<NV>()) =
      make_double2(negx(Ld), Lvt);
}

// The branch J values recomputed from x (the sweep's formulas).
__device__ __forceinline__ BranchJ branch_j(const Dev &d, const double *__restrict__ x, int32_t t, int32_t l,
                                            int32_t f, int32_t to) {
  const int32_t L = d.L;
  const int64_t tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const double vf = __ldg(x + d.x_vm + tN + f), vt = __ldg(x + d.x_vm + tN + to);
  const Flow F = flow_terms(d, l, __ldg(x + tN + f), __ldg(x + tN + to), vf, vt);
  const FlowJ Jf = flow_jac(d, l, F, vf, vt);
  BranchJ J;
  J.a1 = Jf.a1; J.b1 = Jf.b1; J.c1 = Jf.c1;
  J.a2 = Jf.a2; J.b2 = Jf.b2; J.c2 = Jf.c2;
  J.a3 = Jf.a3; J.b3 = Jf.b3; J.c3 = Jf.c3;
  J.a4 = Jf.a4; J.b4 = Jf.b4; J.c4 = Jf.c4;
  J.jp6 = twice(__ldg(x + pb + l));
  J.jq6 = twice(__ldg(x + qb + l));
  J.jp7 = twice(__ldg(x + pb + L + l));
  J.jq7 = twice(__ldg(x + qb + L + l));
  return J;
}

// The branch J values as the sweep stored them (K1..K4 rows [1, a, -a, b, c],
// K6 / K7 [2p, 2q]).
__device__ __forceinline__ BranchJ stored_branch_j(const Dev &d, const double *__restrict__ jv, int32_t tl) {
  const int64_t s5 = 5 * (int64_t)d.T * d.L;
  const double *j1 = jv + d.T + (int64_t)tl * 5;
  BranchJ J;
  J.a1 = __ldg(j1 + 1); J.b1 = __ldg(j1 + 3); J.c1 = __ldg(j1 + 4);
  J.a2 = __ldg(j1 + s5 + 1); J.b2 = __ldg(j1 + s5 + 3); J.c2 = __ldg(j1 + s5 + 4);
  J.a3 = __ldg(j1 + 2 * s5 + 1); J.b3 = __ldg(j1 + 2 * s5 + 3); J.c3 = __ldg(j1 + 2 * s5 + 4);
  J.a4 = __ldg(j1 + 3 * s5 + 1); J.b4 = __ldg(j1 + 3 * s5 + 3); J.c4 = __ldg(j1 + 3 * s5 + 4);
  // scalar loads: the K6/K7 blocks start at odd offsets when T is odd
  const double *j6 = jv + d.j_k6 + (int64_t)tl * 2, *j7 = jv + d.j_k7 + (int64_t)tl * 2;
  J.jp6 = __ldg(j6); J.jq6 = __ldg(j6 + 1); J.jp7 = __ldg(j7); J.jq7 = __ldg(j7 + 1);
  return J;
}

// J^T y, branch x period; STORED: J's branch rows read from jv (separate
// instantiations, so that each form keeps its own register allocation).
template <int NV, bool STORED>
__global__ void __launch_bounds__(kAdjBlock) k_vjp_branch_many(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ jv, const double *__restrict__ y,
                                                       double *__restrict__ gx, int32_t nvec) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const BranchJ J = STORED ? stored_branch_j(d, jv, tl) : branch_j(d, x, t, l, f, to);
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    vjp_branch_vec<NV>(d, J, t, l, f, to, y + j * d.m, gx + j * d.n, j);
  }
}

template <int NV>
__global__ void __launch_bounds__(kAdjBlock) k_vjp_bus_many(Dev d, const double *__restrict__ x,
                                                    const double *__restrict__ y, double *__restrict__ gx,
                                                    double *__restrict__ gpd, double *__restrict__ gqd,
                                                    int32_t nvec) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int32_t s0 = __ldg(d.inc_ptr + pos), s1 = __ldg(d.inc_ptr + pos + 1);
  const double vm = __ldg(x + d.x_vm + tn);
  const double m2v = __ldg(d.bus_m2gs + n) * vm, p2v = __ldg(d.bus_p2bs + n) * vm;
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    const double *yj = y + j * d.m;
    const double *R = prod_rec<NV>(d, t, j);
    // va: reference element first, then the incident branches in branch order.
    double ga = 0.0, gv = 0.0;
    bool has_a = false, has_v = false;
    if (n == d.ref) { ga = __ldg(yj + t); has_a = true; }
    for (int32_t q = s0; q < s1; ++q) {
      const double2 r = __ldg(reinterpret_cast<const double2 *>(R + (int64_t)q * rec_stride<NV>()));
      ga = has_a ? ga + r.x : r.x;
      gv = has_v ? gv + r.y : r.y;
      has_a = has_v = true;
    }
    // vm: then the bus element (rows K8, K9).
    const double y8 = __ldg(yj + d.c_k8 + tn), y9 = __ldg(yj + d.c_k9 + tn);
    const double Lbus = fma(p2v, y9, m2v * y8);
    gv = has_v ? gv + Lbus : Lbus;
    double *gj = gx + j * d.n;
    gj[tn] = ga;
    gj[d.x_vm + tn] = gv;
    if (gpd) {
      const int64_t ldb = (int64_t)t * d.D + j * d.T * d.D;
      for (int32_t e = __ldg(d.bload_ptr + n); e < __ldg(d.bload_ptr + n + 1); ++e) {
        const int32_t k = __ldg(d.bload_idx + e);
        gpd[ldb + k] = negx(y8);
        gqd[ldb + k] = negx(y9);
      }
    }
  }
}

template <int NV>
__global__ void __launch_bounds__(kAdjBlock) k_vjp_gen_many(Dev d, const double *__restrict__ y, double *__restrict__ gx,
                                                    int32_t nvec) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= d.T * G) return;
  const int32_t t = tg / G, g = tg - t * G;
  const int64_t tn = (int64_t)t * d.N + __ldg(d.gen_bus + g);
  const int64_t rr = d.c_k10 + (int64_t)(t - 1) * G + g;
  const int64_t rq = d.c_k11 + (int64_t)(t - 1) * G + g;
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    const double *yj = y + j * d.m;
    double a = __ldg(yj + d.c_k8 + tn);           // bus element (K8, entry +1)
    if (t >= 1) a = a + __ldg(yj + rr);           // ramp row (t, g): +1
    if (t + 1 < d.T) a = a - __ldg(yj + rr + G);  // ramp row (t + 1, g): -1
    gx[j * d.n + d.x_pg + tg] = a;
    double b = __ldg(yj + d.c_k9 + tn);  // bus element (K9, entry +1)
    if (d.qramp) {
      if (t >= 1) b = b + __ldg(yj + rq);           // reactive ramp row (t, g): +1
      if (t + 1 < d.T) b = b - __ldg(yj + rq + G);  // reactive ramp row (t + 1, g): -1
    }
    gx[j * d.n + d.x_qg + tg] = b;
  }
}

// ---------------------------------------------------------------------------
// J v (+ load tangents): one row at a time in its J order.
// ---------------------------------------------------------------------------
template <int NV, bool STORED>
__global__ void __launch_bounds__(kAdjBlock) k_jvp_branch_many(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ jv, const double *__restrict__ v,
                                                       double *__restrict__ out, int32_t nvec) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t TL = (int64_t)d.T * L, tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const BranchJ J = STORED ? stored_branch_j(d, jv, tl) : branch_j(d, x, t, l, f, to);
  const int64_t rk1 = d.T + tl;
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    const double *vj = v + j * d.n;
    double *oj = out + j * d.m;
    const double uf = __ldg(vj + tN + f), ut = __ldg(vj + tN + to);
    const double wf = __ldg(vj + d.x_vm + tN + f), wt = __ldg(vj + d.x_vm + tN + to);
    const double vpf = __ldg(vj + pb + l), vpt = __ldg(vj + pb + L + l);
    const double vqf = __ldg(vj + qb + l), vqt = __ldg(vj + qb + L + l);
    oj[rk1] = fma(J.c1, wt, fma(J.b1, wf, fma(negx(J.a1), ut, fma(J.a1, uf, vpf))));
    oj[rk1 + TL] = fma(J.c2, wt, fma(J.b2, wf, fma(negx(J.a2), ut, fma(J.a2, uf, vqf))));
    oj[rk1 + 2 * TL] = fma(J.c3, wt, fma(J.b3, wf, fma(negx(J.a3), ut, fma(J.a3, uf, vpt))));
    oj[rk1 + 3 * TL] = fma(J.c4, wt, fma(J.b4, wf, fma(negx(J.a4), ut, fma(J.a4, uf, vqt))));
    oj[rk1 + 4 * TL] = uf - ut;
    oj[rk1 + 5 * TL] = fma(J.jq6, vqf, J.jp6 * vpf);
    oj[rk1 + 6 * TL] = fma(J.jq7, vqt, J.jp7 * vpt);
  }
}

template <int NV>
__global__ void __launch_bounds__(kAdjBlock) k_jvp_bus_many(Dev d, const double *__restrict__ x,
                                                    const double *__restrict__ v, const double *__restrict__ dpd,
                                                    const double *__restrict__ dqd, double *__restrict__ out,
                                                    int32_t nvec) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int64_t L = d.L, G = d.G;
  const double vm = __ldg(x + d.x_vm + tn);
  const double m2v = __ldg(d.bus_m2gs + n) * vm, p2v = __ldg(d.bus_p2bs + n) * vm;
  const int32_t g0 = __ldg(d.bgen_ptr + n), g1 = __ldg(d.bgen_ptr + n + 1);
  const int32_t a0 = __ldg(d.barc_ptr + n), a1 = __ldg(d.barc_ptr + n + 1);
  const int64_t pgb = d.x_pg + (int64_t)t * G, qgb = d.x_qg + (int64_t)t * G;
  const int64_t pab = d.x_p + 2 * (int64_t)t * L, qab = d.x_q + 2 * (int64_t)t * L;
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    const double *vj = v + j * d.n;
    double *oj = out + j * d.m;
    if (n == d.ref) oj[t] = __ldg(vj + (int64_t)t * N + n);
    const double dvm = __ldg(vj + d.x_vm + tn);
    double aP = m2v * dvm, aQ = p2v * dvm;
    for (int32_t e = g0; e < g1; ++e) {
      const int32_t g = __ldg(d.bgen_idx + e);
      aP = aP + __ldg(vj + pgb + g);
      aQ = aQ + __ldg(vj + qgb + g);
    }
    for (int32_t e = a0; e < a1; ++e) {
      const int32_t a = __ldg(d.barc_idx + e);
      aP = aP - __ldg(vj + pab + a);
      aQ = aQ - __ldg(vj + qab + a);
    }
    if (dpd) {
      const int64_t ldb = (int64_t)t * d.D + j * d.T * d.D;
      for (int32_t e = __ldg(d.bload_ptr + n); e < __ldg(d.bload_ptr + n + 1); ++e) {
        const int32_t k = __ldg(d.bload_idx + e);
        aP = aP - __ldg(dpd + ldb + k);
        aQ = aQ - __ldg(dqd + ldb + k);
      }
    }
    oj[d.c_k8 + tn] = aP;
    oj[d.c_k9 + tn] = aQ;
  }
}

template <int NV>
__global__ void __launch_bounds__(kAdjBlock) k_jvp_gen_many(Dev d, const double *__restrict__ v, double *__restrict__ out,
                                                    int32_t nvec) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= (d.T - 1) * G) return;  // ramp rows (t, g), t = 1..T-1, row index (t - 1) G + g
  const int64_t cur = d.x_pg + G + tg, qc = d.x_qg + G + tg;
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    const double *vj = v + j * d.n;
    out[j * d.m + d.c_k10 + tg] = __ldg(vj + cur) - __ldg(vj + cur - G);
    if (d.qramp) out[j * d.m + d.c_k11 + tg] = __ldg(vj + qc) - __ldg(vj + qc - G);
  }
}

// ---------------------------------------------------------------------------
// W v.  Branch element: its W entries in order (block (0,0)..(3,3), then the
// thermal diagonals), each entry (r, c, w) adding fma(w, v[c], .) to r and,
// off the diagonal, fma(w, v[r], .) to c.
// ---------------------------------------------------------------------------
// The branch element's W values: the block entries Wdd, Wdvf, Wdvt, Wvfvf,
// Wvtvt, their negations where the block holds them, -Asum, and the thermal
// diagonals h6, h7.
struct BranchW {
  double Wdd, nWdd, Wdvf, nWdvf, Wdvt, nWdvt, Wvfvf, Wvtvt, nAsum, h6, h7;
};

// Recomputed from (x, lam) (the sweep's formulas).
__device__ __forceinline__ BranchW branch_w(const Dev &d, const double *__restrict__ x,
                                            const double *__restrict__ lam, int32_t t, int32_t l, int32_t f,
                                            int32_t to) {
  const int64_t TL = (int64_t)d.T * d.L, tN = (int64_t)t * d.N;
  const double vf = __ldg(x + d.x_vm + tN + f), vt = __ldg(x + d.x_vm + tN + to);
  const Flow F = flow_terms(d, l, __ldg(x + tN + f), __ldg(x + tN + to), vf, vt);
  const int64_t rk1 = d.T + (int64_t)t * d.L + l;
  const FlowW W = flow_hess(d, l, F, vf, vt, __ldg(lam + rk1), __ldg(lam + rk1 + TL), __ldg(lam + rk1 + 2 * TL),
                            __ldg(lam + rk1 + 3 * TL));
  BranchW B;
  B.Wdd = W.Wdd; B.nWdd = negx(W.Wdd);
  B.Wdvf = W.Wdvf; B.nWdvf = negx(W.Wdvf);
  B.Wdvt = W.Wdvt; B.nWdvt = negx(W.Wdvt);
  B.Wvfvf = W.Wvfvf; B.Wvtvt = W.Wvtvt; B.nAsum = negx(W.Asum);
  B.h6 = twice(__ldg(lam + rk1 + 5 * TL));
  B.h7 = twice(__ldg(lam + rk1 + 6 * TL));
  return B;
}

// As the sweep stored them (hw [nnz_hess]: the element's ten block entries
// Wdd, -Wdd, Wdd, Wdvf, -Wdvf, Wvfvf, Wdvt, -Wdvt, -Asum, Wvtvt and the
// thermal diagonals h6, h6, h7, h7): the same values bit for bit.
__device__ __forceinline__ BranchW stored_branch_w(const Dev &d, const double *__restrict__ hw, int32_t tl) {
  const double *hb = hw + d.h_br + (int64_t)tl * 10;
  const double *th = hw + d.h_th + (int64_t)tl * 4;
  BranchW B;
  B.Wdd = __ldg(hb); B.nWdd = __ldg(hb + 1);
  B.Wdvf = __ldg(hb + 3); B.nWdvf = __ldg(hb + 4); B.Wvfvf = __ldg(hb + 5);
  B.Wdvt = __ldg(hb + 6); B.nWdvt = __ldg(hb + 7); B.nAsum = __ldg(hb + 8); B.Wvtvt = __ldg(hb + 9);
  B.h6 = __ldg(th); B.h7 = __ldg(th + 2);
  return B;
}

// W v, branch x period; STORED: the element's W values read from hw.
template <int NV, bool STORED>
__global__ void __launch_bounds__(kAdjBlock) k_hvp_branch_many(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ lam, const double *__restrict__ hw,
                                                       const double *__restrict__ v, double *__restrict__ hv,
                                                       int32_t nvec) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const BranchW W = STORED ? stored_branch_w(d, hw, tl) : branch_w(d, x, lam, t, l, f, to);
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    const double *vj = v + j * d.n;
    double *hj = hv + j * d.n;
    const double uf = __ldg(vj + tN + f), ut = __ldg(vj + tN + to);
    const double wf = __ldg(vj + d.x_vm + tN + f), wt = __ldg(vj + d.x_vm + tN + to);
    const double hf = fma(W.Wdvt, wt, fma(W.Wdvf, wf, fma(W.nWdd, ut, W.Wdd * uf)));
    const double ht = fma(W.nWdvt, wt, fma(W.nWdvf, wf, fma(W.Wdd, ut, W.nWdd * uf)));
    const double hvf = fma(W.nAsum, wt, fma(W.Wvfvf, wf, fma(W.nWdvf, ut, W.Wdvf * uf)));
    const double hvt = fma(W.Wvtvt, wt, fma(W.nAsum, wf, fma(W.nWdvt, ut, W.Wdvt * uf)));
    hj[pb + l] = W.h6 * __ldg(vj + pb + l);
    hj[qb + l] = W.h6 * __ldg(vj + qb + l);
    hj[pb + L + l] = W.h7 * __ldg(vj + pb + L + l);
    hj[qb + L + l] = W.h7 * __ldg(vj + qb + L + l);
    double *R = prod_rec<NV>(d, t, j);
    *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * rec_stride<NV>()) = make_double2(hf, hvf);
    *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * rec_stride<NV>()) =
        make_double2(ht, hvt);
  }
}

template <int NV>
__global__ void __launch_bounds__(kAdjBlock) k_hvp_bus_many(Dev d, const double *__restrict__ lam,
                                                    const double *__restrict__ v, double *__restrict__ hv,
                                                    int32_t nvec) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int32_t s0 = __ldg(d.inc_ptr + pos), s1 = __ldg(d.inc_ptr + pos + 1);
  const double WP = __ldg(lam + d.c_k8 + tn) * __ldg(d.bus_m2gs + n);
  const double WQ = __ldg(lam + d.c_k9 + tn) * __ldg(d.bus_p2bs + n);
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    const double *R = prod_rec<NV>(d, t, j);
    double ha = 0.0, hm = 0.0;
    for (int32_t q = s0; q < s1; ++q) {
      const double2 r = __ldg(reinterpret_cast<const double2 *>(R + (int64_t)q * rec_stride<NV>()));
      ha = (q == s0) ? r.x : ha + r.x;
      hm = (q == s0) ? r.y : hm + r.y;
    }
    const double dvm = __ldg(v + j * d.n + d.x_vm + tn);
    const double Lbus = fma(WQ, dvm, WP * dvm);
    double *hj = hv + j * d.n;
    hj[tn] = ha;
    hj[d.x_vm + tn] = (s1 > s0) ? hm + Lbus : Lbus;
  }
}

template <int NV>
__global__ void __launch_bounds__(kAdjBlock) k_hvp_gen_many(Dev d, double sigma, const double *__restrict__ v,
                                                    double *__restrict__ hv, int32_t nvec) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= d.T * G) return;
  const int32_t g = tg % G;
  const double w = sigma * __ldg(d.gen_c2x2 + g);
#pragma unroll
  for (int i = 0; i < vec_count<NV>(); ++i) {
    const int64_t j = vec_index<NV>(i, nvec);
    if (j < 0) break;
    hv[j * d.n + d.x_pg + tg] = w * __ldg(v + j * d.n + d.x_pg + tg);
    hv[j * d.n + d.x_qg + tg] = 0.0;
  }
}

unsigned grid_for(int64_t count) { return (unsigned)((count + kAdjBlock - 1) / kAdjBlock); }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

// The launches of the single products.
void launch_vjp1(const Dev &d, const double *x, const double *jv, const double *y, double *gx, double *gpd,
                 double *gqd, cudaStream_t s) {
  if (d.L > 0) {
    if (jv) k_vjp_branch_jv<<<grid_for((int64_t)d.T * d.L), kAdjBlock, 0, s>>>(d, jv, y, gx);
    else k_vjp_branch<<<grid_for((int64_t)d.T * d.L), kAdjBlock, 0, s>>>(d, x, y, gx);
  }
  k_vjp_bus<<<grid_for((int64_t)d.T * d.N), kAdjBlock, 0, s>>>(d, x, y, gx, gpd, d.D > 0 ? gqd : nullptr);
  if (d.G > 0) k_vjp_gen<<<grid_for((int64_t)d.T * d.G), kAdjBlock, 0, s>>>(d, y, gx);
}

void launch_jvp1(const Dev &d, const double *x, const double *jv, const double *v, const double *dpd,
                 const double *dqd, double *out, cudaStream_t s) {
  if (d.L > 0) {
    if (jv) k_jvp_branch_jv<<<grid_for((int64_t)d.T * d.L), kAdjBlock, 0, s>>>(d, jv, v, out);
    else k_jvp_branch<<<grid_for((int64_t)d.T * d.L), kAdjBlock, 0, s>>>(d, x, v, out);
  }
  k_jvp_bus<<<grid_for((int64_t)d.T * d.N), kAdjBlock, 0, s>>>(d, x, v, d.D > 0 ? dpd : nullptr, dqd, out);
  if (d.G > 0 && d.T > 1) k_jvp_gen<<<grid_for((int64_t)(d.T - 1) * d.G), kAdjBlock, 0, s>>>(d, v, out);
}

void launch_hvp1(const Dev &d, const double *x, const double *lam, double sigma, const double *v, double *hv,
                 cudaStream_t s) {
  if (d.L > 0) k_hvp_branch<<<grid_for((int64_t)d.T * d.L), kAdjBlock, 0, s>>>(d, x, lam, v, hv);
  k_hvp_bus<<<grid_for((int64_t)d.T * d.N), kAdjBlock, 0, s>>>(d, lam, v, hv);
  if (d.G > 0) k_hvp_gen<<<grid_for((int64_t)d.T * d.G), kAdjBlock, 0, s>>>(d, sigma, v, hv);
}

// The launches of the products for k vectors, NV per thread (grid y =
// ceil(k / NV)); d.S the packed records of the k vectors.
template <int NV>
void launch_vjp(const Dev &d, int32_t k, const double *x, const double *jv, const double *y, double *gx,
                double *gpd, double *gqd, cudaStream_t s) {
  static_assert(NV >= 1, "several vectors");
  const unsigned gy = (unsigned)((k + NV - 1) / NV);
  if (d.L > 0) {
    const dim3 g(grid_for((int64_t)d.T * d.L), gy);
    if (jv) k_vjp_branch_many<NV, true><<<g, kAdjBlock, 0, s>>>(d, x, jv, y, gx, k);
    else k_vjp_branch_many<NV, false><<<g, kAdjBlock, 0, s>>>(d, x, jv, y, gx, k);
  }
  k_vjp_bus_many<NV><<<dim3(grid_for((int64_t)d.T * d.N), gy), kAdjBlock, 0, s>>>(d, x, y, gx, gpd,
                                                                                  d.D > 0 ? gqd : nullptr, k);
  if (d.G > 0) k_vjp_gen_many<NV><<<dim3(grid_for((int64_t)d.T * d.G), gy), kAdjBlock, 0, s>>>(d, y, gx, k);
}

template <int NV>
void launch_jvp(const Dev &d, int32_t k, const double *x, const double *jv, const double *v, const double *dpd,
                const double *dqd, double *out, cudaStream_t s) {
  static_assert(NV >= 1, "several vectors");
  const unsigned gy = (unsigned)((k + NV - 1) / NV);
  if (d.L > 0) {
    const dim3 g(grid_for((int64_t)d.T * d.L), gy);
    if (jv) k_jvp_branch_many<NV, true><<<g, kAdjBlock, 0, s>>>(d, x, jv, v, out, k);
    else k_jvp_branch_many<NV, false><<<g, kAdjBlock, 0, s>>>(d, x, jv, v, out, k);
  }
  k_jvp_bus_many<NV><<<dim3(grid_for((int64_t)d.T * d.N), gy), kAdjBlock, 0, s>>>(
      d, x, v, d.D > 0 ? dpd : nullptr, dqd, out, k);
  if (d.G > 0 && d.T > 1)
    k_jvp_gen_many<NV><<<dim3(grid_for((int64_t)(d.T - 1) * d.G), gy), kAdjBlock, 0, s>>>(d, v, out, k);
}

template <int NV>
void launch_hvp(const Dev &d, int32_t k, const double *x, const double *lam, double sigma, const double *hw,
                const double *v, double *hv, cudaStream_t s) {
  static_assert(NV >= 1, "several vectors");
  const unsigned gy = (unsigned)((k + NV - 1) / NV);
  if (d.L > 0) {
    const dim3 g(grid_for((int64_t)d.T * d.L), gy);
    if (hw) k_hvp_branch_many<NV, true><<<g, kAdjBlock, 0, s>>>(d, x, lam, hw, v, hv, k);
    else k_hvp_branch_many<NV, false><<<g, kAdjBlock, 0, s>>>(d, x, lam, hw, v, hv, k);
  }
  k_hvp_bus_many<NV><<<dim3(grid_for((int64_t)d.T * d.N), gy), kAdjBlock, 0, s>>>(d, lam, v, hv, k);
  if (d.G > 0)
    k_hvp_gen_many<NV><<<dim3(grid_for((int64_t)d.T * d.G), gy), kAdjBlock, 0, s>>>(d, sigma, v, hv, k);
}

// The handle's descriptor with d.S pointing at the packed records of k
// vectors (2 L T double2 each) in the handle's scratch.
int many_dev(mpopf_handle *h, int32_t k, const char *who, cudaStream_t s, Dev *out) {
  if (k < 1 || k > 65535) return fail(MPOPF_ERR_ARG, std::string(who) + ": k outside [1, 65535]");
  const size_t rec = (size_t)2 * h->d.L * h->d.T * rec_stride<1>();
  const int rc = grow_points_scratch(h, (size_t)k * rec * sizeof(double), who, s);
  if (rc != MPOPF_OK) return rc;
  *out = h->d;
  out->S = h->pts;
  return MPOPF_OK;
}

int done(const char *who) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string(who) + ": " + cudaGetErrorString(e));
  return MPOPF_OK;
}

}  // namespace
}  // namespace mpopf

using namespace mpopf;

extern "C" {

int mpopf_vjp_jv(mpopf_handle *h, const double *x, const double *jv, const double *y, double *gx, double *gpd,
                 double *gqd, void *stream) {
  if (!h || !x || !y || !gx) return fail(MPOPF_ERR_ARG, "mpopf_vjp: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_vjp: not available on a period shard");
  if ((gpd == nullptr) != (gqd == nullptr)) return fail(MPOPF_ERR_ARG, "mpopf_vjp: give both gpd and gqd or neither");
  launch_vjp1(h->d, x, jv, y, gx, gpd, gqd, static_cast<cudaStream_t>(stream));
  return done("mpopf_vjp");
}

int mpopf_vjp(mpopf_handle *h, const double *x, const double *y, double *gx, double *gpd, double *gqd, void *stream) {
  return mpopf_vjp_jv(h, x, nullptr, y, gx, gpd, gqd, stream);
}

int mpopf_jvp_jv(mpopf_handle *h, const double *x, const double *jv, const double *v, const double *dpd,
                 const double *dqd, double *jv_out, void *stream) {
  if (!h || !x || !v || !jv_out) return fail(MPOPF_ERR_ARG, "mpopf_jvp: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_jvp: not available on a period shard");
  if ((dpd == nullptr) != (dqd == nullptr)) return fail(MPOPF_ERR_ARG, "mpopf_jvp: give both dpd and dqd or neither");
  launch_jvp1(h->d, x, jv, v, dpd, dqd, jv_out, static_cast<cudaStream_t>(stream));
  return done("mpopf_jvp");
}

int mpopf_jvp(mpopf_handle *h, const double *x, const double *v, const double *dpd, const double *dqd, double *jv_out,
              void *stream) {
  return mpopf_jvp_jv(h, x, nullptr, v, dpd, dqd, jv_out, stream);
}

int mpopf_hvp(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *v, double *hv,
              void *stream) {
  if (!h || !x || !lam || !v || !hv) return fail(MPOPF_ERR_ARG, "mpopf_hvp: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_hvp: not available on a period shard");
  launch_hvp1(h->d, x, lam, sigma, v, hv, static_cast<cudaStream_t>(stream));
  return done("mpopf_hvp");
}

int mpopf_vjp_many(mpopf_handle *h, int32_t k, const double *x, const double *jv, const double *y, double *gx,
                   double *gpd, double *gqd, void *stream) {
  if (!h || !x || !y || !gx) return fail(MPOPF_ERR_ARG, "mpopf_vjp_many: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_vjp_many: not available on a period shard");
  if ((gpd == nullptr) != (gqd == nullptr))
    return fail(MPOPF_ERR_ARG, "mpopf_vjp_many: give both gpd and gqd or neither");
  Dev d;
  const int rc = many_dev(h, k, "mpopf_vjp_many", static_cast<cudaStream_t>(stream), &d);
  if (rc != MPOPF_OK) return rc;
  launch_vjp<kManyNV>(d, k, x, jv, y, gx, gpd, gqd, static_cast<cudaStream_t>(stream));
  return done("mpopf_vjp_many");
}

int mpopf_jvp_many(mpopf_handle *h, int32_t k, const double *x, const double *jv, const double *v,
                   const double *dpd, const double *dqd, double *out, void *stream) {
  if (!h || !x || !v || !out) return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: not available on a period shard");
  if ((dpd == nullptr) != (dqd == nullptr))
    return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: give both dpd and dqd or neither");
  if (k < 1 || k > 65535) return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: k outside [1, 65535]");
  launch_jvp<kManyNV>(h->d, k, x, jv, v, dpd, dqd, out, static_cast<cudaStream_t>(stream));
  return done("mpopf_jvp_many");
}

int mpopf_hvp_many(mpopf_handle *h, int32_t k, const double *x, const double *lam, double sigma, const double *hw,
                   const double *v, double *hv, void *stream) {
  if (!h || !x || !lam || !v || !hv) return fail(MPOPF_ERR_ARG, "mpopf_hvp_many: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_hvp_many: not available on a period shard");
  Dev d;
  const int rc = many_dev(h, k, "mpopf_hvp_many", static_cast<cudaStream_t>(stream), &d);
  if (rc != MPOPF_OK) return rc;
  launch_hvp<kManyNV>(d, k, x, lam, sigma, hw, v, hv, static_cast<cudaStream_t>(stream));
  return done("mpopf_hvp_many");
}

}  // extern "C"
