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

// MANY: the kernels of the products for several vectors at one point (vector
// j = blockIdx.y reads and writes the j-th of consecutive arrays of the
// single product's sizes).  Incidence records: one double2 per branch end;
// a single product writes them into the sweep's record array (kRec doubles
// apart), several vectors into their own packed array (vector j's T periods
// after the earlier vectors').
template <bool MANY>
__device__ __forceinline__ double *prod_rec(const Dev &d, int32_t t) {
  return d.S + ((MANY ? (int64_t)blockIdx.y * d.T : 0) + t) * 2 * d.L * (MANY ? 2 : kRec);
}
template <bool MANY>
__host__ __device__ constexpr int rec_stride() {
  return MANY ? 2 : kRec;
}

// ---------------------------------------------------------------------------
// J^T y.  Branch element local sums over its rows K1..K7:
//   va_f: a1 y1, + a2 y2, + a3 y3, + a4 y4, + y5   (va_t: the exact negation)
//   vm_f: b_k y_k (k = 1..4);  vm_t: c_k y_k
//   p_f: fma(2pf, y6, y1);  q_f: fma(2qf, y6, y2);  p_t: fma(2pt, y7, y3);
//   q_t: fma(2qt, y7, y4); then the bus element adds -y8 (p) or -y9 (q).
// ---------------------------------------------------------------------------
template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_vjp_branch(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ y, double *__restrict__ gx) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  if (MANY) {
    y += (int64_t)blockIdx.y * d.m;
    gx += (int64_t)blockIdx.y * d.n;
  }
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
  double *R = prod_rec<MANY>(d, t);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * rec_stride<MANY>()) = make_double2(Ld, Lvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * rec_stride<MANY>()) =
      make_double2(negx(Ld), Lvt);
}

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_vjp_bus(Dev d, const double *__restrict__ x,
                                                    const double *__restrict__ y, double *__restrict__ gx,
                                                    double *__restrict__ gpd, double *__restrict__ gqd) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  if (MANY) {
    const int64_t j = blockIdx.y;
    y += j * d.m;
    gx += j * d.n;
    if (gpd) {
      gpd += j * d.T * d.D;
      gqd += j * d.T * d.D;
    }
  }
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int32_t s0 = __ldg(d.inc_ptr + pos), s1 = __ldg(d.inc_ptr + pos + 1);
  const double *R = prod_rec<MANY>(d, t);
  // va: reference element first, then the incident branches in branch order.
  double ga = 0.0, gv = 0.0;
  bool has_a = false, has_v = false;
  if (n == d.ref) { ga = __ldg(y + t); has_a = true; }
  for (int32_t q = s0; q < s1; ++q) {
    const double2 r = __ldg(reinterpret_cast<const double2 *>(R + (int64_t)q * rec_stride<MANY>()));
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

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_vjp_gen(Dev d, const double *__restrict__ y, double *__restrict__ gx) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= d.T * G) return;
  if (MANY) {
    y += (int64_t)blockIdx.y * d.m;
    gx += (int64_t)blockIdx.y * d.n;
  }
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
template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_jvp_branch(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ v, double *__restrict__ out) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  if (MANY) {
    v += (int64_t)blockIdx.y * d.n;
    out += (int64_t)blockIdx.y * d.m;
  }
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

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_jvp_bus(Dev d, const double *__restrict__ x,
                                                    const double *__restrict__ v, const double *__restrict__ dpd,
                                                    const double *__restrict__ dqd, double *__restrict__ out) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  if (MANY) {
    const int64_t j = blockIdx.y;
    v += j * d.n;
    out += j * d.m;
    if (dpd) {
      dpd += j * d.T * d.D;
      dqd += j * d.T * d.D;
    }
  }
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

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_jvp_gen(Dev d, const double *__restrict__ v, double *__restrict__ out) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= (d.T - 1) * G) return;  // ramp rows (t, g), t = 1..T-1, row index (t - 1) G + g
  if (MANY) {
    v += (int64_t)blockIdx.y * d.n;
    out += (int64_t)blockIdx.y * d.m;
  }
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
template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_hvp_branch(Dev d, const double *__restrict__ x,
                                                       const double *__restrict__ lam, const double *__restrict__ v,
                                                       double *__restrict__ hv) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  if (MANY) {
    v += (int64_t)blockIdx.y * d.n;
    hv += (int64_t)blockIdx.y * d.n;
  }
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
  double *R = prod_rec<MANY>(d, t);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * rec_stride<MANY>()) = make_double2(hf, hvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * rec_stride<MANY>()) = make_double2(ht, hvt);
}

// The branch element of W v with its W values as the sweep wrote them at the
// same (x, lam) (hw [nnz_hess]: the element's ten block entries Wdd, -Wdd,
// Wdd, Wdvf, -Wdvf, Wvfvf, Wdvt, -Wdvt, -Asum, Wvtvt and the thermal
// diagonals h6, h6, h7, h7) instead of recomputed: the same operands in the
// same order as k_hvp_branch, so the same results bit for bit.
template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_hvp_branch_hw(Dev d, const double *__restrict__ hw,
                                                          const double *__restrict__ v, double *__restrict__ hv) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  if (MANY) {
    v += (int64_t)blockIdx.y * d.n;
    hv += (int64_t)blockIdx.y * d.n;
  }
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  const int32_t f = __ldg(d.br_f + l), to = __ldg(d.br_t + l);
  const double *hb = hw + d.h_br + (int64_t)tl * 10;
  const double Wdd = __ldg(hb), nWdd = __ldg(hb + 1), Wdvf = __ldg(hb + 3), nWdvf = __ldg(hb + 4);
  const double Wvfvf = __ldg(hb + 5), Wdvt = __ldg(hb + 6), nWdvt = __ldg(hb + 7), nAsum = __ldg(hb + 8);
  const double Wvtvt = __ldg(hb + 9);
  const double uf = __ldg(v + tN + f), ut = __ldg(v + tN + to);
  const double wf = __ldg(v + d.x_vm + tN + f), wt = __ldg(v + d.x_vm + tN + to);
  const double hf = fma(Wdvt, wt, fma(Wdvf, wf, fma(nWdd, ut, Wdd * uf)));
  const double ht = fma(nWdvt, wt, fma(nWdvf, wf, fma(Wdd, ut, nWdd * uf)));
  const double hvf = fma(nAsum, wt, fma(Wvfvf, wf, fma(nWdvf, ut, Wdvf * uf)));
  const double hvt = fma(Wvtvt, wt, fma(nAsum, wf, fma(nWdvt, ut, Wdvt * uf)));
  const double *th = hw + d.h_th + (int64_t)tl * 4;
  const double h6 = __ldg(th), h7 = __ldg(th + 2);
  hv[pb + l] = h6 * __ldg(v + pb + l);
  hv[qb + l] = h6 * __ldg(v + qb + l);
  hv[pb + L + l] = h7 * __ldg(v + pb + L + l);
  hv[qb + L + l] = h7 * __ldg(v + qb + L + l);
  double *R = prod_rec<MANY>(d, t);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * rec_stride<MANY>()) = make_double2(hf, hvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * rec_stride<MANY>()) = make_double2(ht, hvt);
}

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_hvp_bus(Dev d, const double *__restrict__ lam,
                                                    const double *__restrict__ v, double *__restrict__ hv) {
  const int32_t N = d.N;
  const int32_t idx = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= d.T * N) return;
  if (MANY) {
    v += (int64_t)blockIdx.y * d.n;
    hv += (int64_t)blockIdx.y * d.n;
  }
  const int32_t t = idx / N, pos = idx - t * N;
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;
  const int32_t s0 = __ldg(d.inc_ptr + pos), s1 = __ldg(d.inc_ptr + pos + 1);
  const double *R = prod_rec<MANY>(d, t);
  double ha = 0.0, hm = 0.0;
  for (int32_t q = s0; q < s1; ++q) {
    const double2 r = __ldg(reinterpret_cast<const double2 *>(R + (int64_t)q * rec_stride<MANY>()));
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

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_hvp_gen(Dev d, double sigma, const double *__restrict__ v,
                                                    double *__restrict__ hv) {
  const int32_t G = d.G;
  const int32_t tg = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tg >= d.T * G) return;
  if (MANY) {
    v += (int64_t)blockIdx.y * d.n;
    hv += (int64_t)blockIdx.y * d.n;
  }
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

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_vjp_branch_jv(Dev d, const double *__restrict__ jv,
                                                          const double *__restrict__ y, double *__restrict__ gx) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  if (MANY) {
    y += (int64_t)blockIdx.y * d.m;
    gx += (int64_t)blockIdx.y * d.n;
  }
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
  double *R = prod_rec<MANY>(d, t);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + l) * rec_stride<MANY>()) = make_double2(Ld, Lvf);
  *reinterpret_cast<double2 *>(R + (int64_t)__ldg(d.br_slot + L + l) * rec_stride<MANY>()) =
      make_double2(negx(Ld), Lvt);
}

template <bool MANY>
__global__ void __launch_bounds__(kAdjBlock) k_jvp_branch_jv(Dev d, const double *__restrict__ jv,
                                                          const double *__restrict__ v, double *__restrict__ out) {
  const int32_t L = d.L;
  const int32_t tl = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= d.T * L) return;
  if (MANY) {
    v += (int64_t)blockIdx.y * d.n;
    out += (int64_t)blockIdx.y * d.m;
  }
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

unsigned grid_for(int64_t count) { return (unsigned)((count + kAdjBlock - 1) / kAdjBlock); }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

// The launches of each product; with MANY, k vectors (grid y) and d.S the
// packed records of the k vectors.
template <bool MANY>
void launch_vjp(const Dev &d, unsigned k, const double *x, const double *jv, const double *y, double *gx,
                double *gpd, double *gqd, cudaStream_t s) {
  if (d.L > 0) {
    const dim3 g(grid_for((int64_t)d.T * d.L), k);
    if (jv) k_vjp_branch_jv<MANY><<<g, kAdjBlock, 0, s>>>(d, jv, y, gx);
    else k_vjp_branch<MANY><<<g, kAdjBlock, 0, s>>>(d, x, y, gx);
  }
  k_vjp_bus<MANY><<<dim3(grid_for((int64_t)d.T * d.N), k), kAdjBlock, 0, s>>>(d, x, y, gx, gpd,
                                                                               d.D > 0 ? gqd : nullptr);
  if (d.G > 0) k_vjp_gen<MANY><<<dim3(grid_for((int64_t)d.T * d.G), k), kAdjBlock, 0, s>>>(d, y, gx);
}

template <bool MANY>
void launch_jvp(const Dev &d, unsigned k, const double *x, const double *jv, const double *v, const double *dpd,
                const double *dqd, double *out, cudaStream_t s) {
  if (d.L > 0) {
    const dim3 g(grid_for((int64_t)d.T * d.L), k);
    if (jv) k_jvp_branch_jv<MANY><<<g, kAdjBlock, 0, s>>>(d, jv, v, out);
    else k_jvp_branch<MANY><<<g, kAdjBlock, 0, s>>>(d, x, v, out);
  }
  k_jvp_bus<MANY><<<dim3(grid_for((int64_t)d.T * d.N), k), kAdjBlock, 0, s>>>(d, x, v, d.D > 0 ? dpd : nullptr,
                                                                               dqd, out);
  if (d.G > 0 && d.T > 1)
    k_jvp_gen<MANY><<<dim3(grid_for((int64_t)(d.T - 1) * d.G), k), kAdjBlock, 0, s>>>(d, v, out);
}

template <bool MANY>
void launch_hvp(const Dev &d, unsigned k, const double *x, const double *lam, double sigma, const double *hw,
                const double *v, double *hv, cudaStream_t s) {
  if (d.L > 0) {
    const dim3 g(grid_for((int64_t)d.T * d.L), k);
    if (hw) k_hvp_branch_hw<MANY><<<g, kAdjBlock, 0, s>>>(d, hw, v, hv);
    else k_hvp_branch<MANY><<<g, kAdjBlock, 0, s>>>(d, x, lam, v, hv);
  }
  k_hvp_bus<MANY><<<dim3(grid_for((int64_t)d.T * d.N), k), kAdjBlock, 0, s>>>(d, lam, v, hv);
  if (d.G > 0) k_hvp_gen<MANY><<<dim3(grid_for((int64_t)d.T * d.G), k), kAdjBlock, 0, s>>>(d, sigma, v, hv);
}

// The handle's descriptor with d.S pointing at the packed records of k
// vectors (2 L T double2 each) in the handle's scratch.
int many_dev(mpopf_handle *h, int32_t k, const char *who, Dev *out) {
  if (k < 1 || k > 65535) return fail(MPOPF_ERR_ARG, std::string(who) + ": k outside [1, 65535]");
  const size_t rec = (size_t)2 * h->d.L * h->d.T * rec_stride<true>();
  const int rc = grow_points_scratch(h, (size_t)k * rec * sizeof(double), who);
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
  launch_vjp<false>(h->d, 1, x, jv, y, gx, gpd, gqd, static_cast<cudaStream_t>(stream));
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
  launch_jvp<false>(h->d, 1, x, jv, v, dpd, dqd, jv_out, static_cast<cudaStream_t>(stream));
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
  launch_hvp<false>(h->d, 1, x, lam, sigma, nullptr, v, hv, static_cast<cudaStream_t>(stream));
  return done("mpopf_hvp");
}

int mpopf_vjp_many(mpopf_handle *h, int32_t k, const double *x, const double *jv, const double *y, double *gx,
                   double *gpd, double *gqd, void *stream) {
  if (!h || !x || !y || !gx) return fail(MPOPF_ERR_ARG, "mpopf_vjp_many: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_vjp_many: not available on a period shard");
  if ((gpd == nullptr) != (gqd == nullptr))
    return fail(MPOPF_ERR_ARG, "mpopf_vjp_many: give both gpd and gqd or neither");
  Dev d;
  const int rc = many_dev(h, k, "mpopf_vjp_many", &d);
  if (rc != MPOPF_OK) return rc;
  launch_vjp<true>(d, (unsigned)k, x, jv, y, gx, gpd, gqd, static_cast<cudaStream_t>(stream));
  return done("mpopf_vjp_many");
}

int mpopf_jvp_many(mpopf_handle *h, int32_t k, const double *x, const double *jv, const double *v,
                   const double *dpd, const double *dqd, double *out, void *stream) {
  if (!h || !x || !v || !out) return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: not available on a period shard");
  if ((dpd == nullptr) != (dqd == nullptr))
    return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: give both dpd and dqd or neither");
  if (k < 1 || k > 65535) return fail(MPOPF_ERR_ARG, "mpopf_jvp_many: k outside [1, 65535]");
  launch_jvp<true>(h->d, (unsigned)k, x, jv, v, dpd, dqd, out, static_cast<cudaStream_t>(stream));
  return done("mpopf_jvp_many");
}

int mpopf_hvp_many(mpopf_handle *h, int32_t k, const double *x, const double *lam, double sigma, const double *hw,
                   const double *v, double *hv, void *stream) {
  if (!h || !x || !lam || !v || !hv) return fail(MPOPF_ERR_ARG, "mpopf_hvp_many: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_hvp_many: not available on a period shard");
  Dev d;
  const int rc = many_dev(h, k, "mpopf_hvp_many", &d);
  if (rc != MPOPF_OK) return rc;
  launch_hvp<true>(d, (unsigned)k, x, lam, sigma, hw, v, hv, static_cast<cudaStream_t>(stream));
  return done("mpopf_hvp_many");
}

}  // extern "C"
