// Plain FP64 CPU oracle for the multi-period AC OPF callbacks and the condensed
// KKT assembly of arXiv 2405.14032.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
// this file; only the tests, the smoke check and the benchmark's CPU-baseline
// leg do.  It shares no code with the CUDA library.
//
// What it computes (passages of the paper):
//   * the model, Eq. (1): quadratic generator cost (1a), active/reactive bus
//     balance with shunts (1b, 1c), the four branch-flow definitions of the
//     pi-model (1d, 1e; the paper prints only the mutual term), apparent-power
//     thermal limits in squared form at both ends (1f), angle-difference limits
//     (1j), the reference angle (implied by Table II's counts) and P ramping
//     between consecutive periods (1k);
//   * the standard-form NLP of Eq. (3): objective, gradient, constraints c(x),
//     Jacobian values on a COO pattern analysed once (Sec. III-A), the
//     Lagrangian Hessian W = sigma grad^2 f + sum_i lambda_i grad^2 c_i (Eq. 4)
//     on a lower-triangular COO pattern;
//   * the condensed matrix M = W + delta_w I + Sigma_x + J^T D J (Sec. III-B),
//     lower CSR including the full diagonal;
//   * matrix-free J^T y (plus the load adjoint), J v and W v.
//
// Reading of the paper where it is silent (the full list is in the design
// notes): row/variable layout, COO orders, pi-model flows, squared thermal
// rows, gen-positive balance, quadratic cost, and a fixed rounding order.
//
// Rounding order.  Every quantity is defined by one fixed sequence of IEEE
// binary64 operations (each correctly rounded; fma = fused multiply-add with
// one rounding).  The sequences are written out below in the order the
// definitions are stated; the compiler is told not to contract or reorder
// (-ffp-contract=off, no fast-math).  sin/cos of the angle difference use
// Cody-Waite argument reduction and economised polynomials (sincos_cw below), so
// the value is a fixed function of its argument on every platform.
//
// Condensed-matrix order.  M is assembled element by element, the way the SIMD
// abstraction of Eq. (2) writes the model as a sum of pattern instances: an
// element is one instance (objective term of generator g at t, reference row
// at t, branch l at t, bus n at t, ramp row of g at t).  Each element's local
// block is  W entries of the element (COO order), then for each of its J rows
// in ascending order, for each local pair (p >= q in the row's J order) the
// term fma(D_i * J_ip, J_iq, .).  M_jk = (Sigma_x[j] + delta_w if j == k), then
// plus each element's local value in element order (objective, reference,
// branch, bus, ramp; within a kind period-major, then component).
//
// Parity unpinned: none.  Every function here is pinned by tests/test_oracle_*
// (closed forms, identities, complex-step and finite differences, counts of
// Table II, brute force on tiny cases).
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>
#include <algorithm>

namespace {

using cplx = std::complex<double>;

inline double fmaS(double a, double b, double c) { return std::fma(a, b, c); }
inline cplx fmaS(const cplx& a, const cplx& b, const cplx& c) { return a * b + c; }
inline double realpart(double a) { return a; }
inline double realpart(const cplx& a) { return a.real(); }

// ---------------------------------------------------------------------------
// sin and cos: Cody-Waite reduction by pi/2 (Cody & Waite, "Software Manual
// for the Elementary Functions", 1980) in three parts, then on |r| <= pi/4
//   sin r = r + r^3 P(s),  cos r = 1 + s Q(s),  s = r^2,  Horner in s,
// where P (degree 5) and Q (degree 6) are the Taylor series of (sin r - r)/r^3
// through s^7 and of (cos r - 1)/r^2 through s^8, economised by Chebyshev
// polynomials (Lanczos's telescoping: the top term c_n s^n is replaced by
// c_n (s^n - T*_n(s) / lead(T*_n)), T*_n(s) = T_n(16 s / 5 - 1), the shifted
// Chebyshev polynomial on [0, 5/8] >= [0, (pi/4)^2]) in exact rational
// arithmetic, each coefficient then rounded to nearest binary64.  Truncation
// and economisation change sin by < 2e-17 and cos by < 1e-18 on the interval.
// |x| <= RN(pi/4) skips the reduction (k = 0, r = x).  |x| >= 2^30 or
// non-finite falls back to the C library (outside the range a voltage-angle
// difference takes).
// ---------------------------------------------------------------------------
const double kQuarterPi = 0x1.921fb54442d18p-1;   // RN(pi/4)
const double kTwoOverPi = 0x1.45f306dc9c883p-1;   // RN(2/pi)
const double kPio2_1 = 0x1.921fb54442d18p+0;      // RN(pi/2)
const double kPio2_2 = 0x1.1a62633145c07p-54;     // RN(pi/2 - P1)
const double kPio2_3 = -0x1.f1976b7ed8fbcp-110;   // RN(pi/2 - P1 - P2)
// P(s) = kP0 + kP1 s + ... + kP5 s^5 (Taylor: -1/3!, 1/5!, -1/7!, ...)
const double kP0 = -0x1.5555555555555p-3, kP1 = 0x1.1111111110b56p-7, kP2 = -0x1.a01a019e6dedep-13,
             kP3 = 0x1.71de377a84b02p-19, kP4 = -0x1.ae5fedfda2660p-26, kP5 = 0x1.5e00b6cff8290p-33;
// Q(s) = kQ0 + kQ1 s + ... + kQ6 s^6 (Taylor: -1/2!, 1/4!, -1/6!, ...)
const double kQ0 = -0x1.0000000000000p-1, kQ1 = 0x1.5555555555550p-5, kQ2 = -0x1.6c16c16c15c7dp-10,
             kQ3 = 0x1.a01a019dc2b7ep-16, kQ4 = -0x1.27e4f8ca561dfp-22, kQ5 = 0x1.1eea6a6fdd11ap-29,
             kQ6 = -0x1.8fedb35736fa4p-37;

template <class S>
void sincos_cw(const S& x, S* sn, S* cs) {
  const double ax = std::fabs(realpart(x));
  if (!(ax < 1073741824.0)) {  // 2^30, NaN, Inf
    *sn = std::sin(x);
    *cs = std::cos(x);
    return;
  }
  S r = x;
  long long q = 0;
  if (!(ax <= kQuarterPi)) {
    const double k = std::rint(realpart(x) * kTwoOverPi);
    r = fmaS(S(-k), S(kPio2_1), x);
    r = fmaS(S(-k), S(kPio2_2), r);
    r = fmaS(S(-k), S(kPio2_3), r);
    q = static_cast<long long>(k) & 3;
  }
  const S r2 = r * r;
  S p = S(kP5);
  p = fmaS(p, r2, S(kP4));
  p = fmaS(p, r2, S(kP3));
  p = fmaS(p, r2, S(kP2));
  p = fmaS(p, r2, S(kP1));
  p = fmaS(p, r2, S(kP0));
  const S r3 = r2 * r;
  const S s = fmaS(r3, p, r);
  S c = S(kQ6);
  c = fmaS(c, r2, S(kQ5));
  c = fmaS(c, r2, S(kQ4));
  c = fmaS(c, r2, S(kQ3));
  c = fmaS(c, r2, S(kQ2));
  c = fmaS(c, r2, S(kQ1));
  c = fmaS(c, r2, S(kQ0));
  const S co = fmaS(r2, c, S(1.0));
  switch (q) {
    case 0: *sn = s; *cs = co; break;
    case 1: *sn = co; *cs = -s; break;
    case 2: *sn = -s; *cs = -co; break;
    default: *sn = -co; *cs = s; break;
  }
}

// ---------------------------------------------------------------------------
// Model: network, horizon, loads, layout.
// ---------------------------------------------------------------------------
struct Model {
  int64_t N, L, G, D, ref, T;
  std::vector<double> gs, bs, vmin, vmax;
  std::vector<int32_t> f, t;
  std::vector<double> br_r, br_x, br_b, tap, shift, smax, angmin, angmax;
  std::vector<int32_t> gbus;
  std::vector<double> c2, c1, c0, pmin, pmax, qmin, qmax, ramp;
  bool has_qramp;             // reactive ramp rows K11 present
  std::vector<double> qramp;  // [G] reactive ramp limits (if has_qramp)
  std::vector<int32_t> lbus;
  std::vector<double> pd, qd;  // [T][D]
  // pi-model admittance terms per branch (Y_ff = gff + j bff, ...)
  std::vector<double> gff, bff, gft, bft, gtf, btf, gtt, btt;
  // incidence lists, ascending
  std::vector<std::vector<int64_t>> bus_gens, bus_arcs, bus_loads;
  int64_t n, m;
  std::vector<int64_t> jrp;  // start of each row's J entries in the COO arrays [m + 1]
};

// Variables: kind-major, then period, then component.
inline int64_t v_va(const Model& M, int64_t t, int64_t i) { return t * M.N + i; }
inline int64_t v_vm(const Model& M, int64_t t, int64_t i) { return M.T * M.N + t * M.N + i; }
inline int64_t v_pg(const Model& M, int64_t t, int64_t g) { return 2 * M.T * M.N + t * M.G + g; }
inline int64_t v_qg(const Model& M, int64_t t, int64_t g) { return 2 * M.T * M.N + M.T * M.G + t * M.G + g; }
inline int64_t v_p(const Model& M, int64_t t, int64_t a) { return 2 * M.T * M.N + 2 * M.T * M.G + t * 2 * M.L + a; }
inline int64_t v_q(const Model& M, int64_t t, int64_t a) {
  return 2 * M.T * M.N + 2 * M.T * M.G + 2 * M.T * M.L + t * 2 * M.L + a;
}
// Variable kind (0 va, 1 vm, 2 pg, 3 qg, 4 p, 5 q) and period of index j.
void var_decode(const Model& M, int64_t j, int* kind, int64_t* t, int64_t* comp) {
  const int64_t cnt[6] = {M.N, M.N, M.G, M.G, 2 * M.L, 2 * M.L};
  for (int k = 0; k < 6; ++k) {
    const int64_t block = M.T * cnt[k];
    if (j < block) { *kind = k; *t = j / cnt[k]; *comp = j % cnt[k]; return; }
    j -= block;
  }
  *kind = -1; *t = -1; *comp = -1;
}

// Constraint rows: K0 ref (t); K1..K7 per branch (t*L + l); K8, K9 per bus;
// K10 ramp ((t-1)*G + g, t >= 1); K11 reactive ramp (same indexing, optional).
inline int64_t r_k0(const Model&, int64_t t) { return t; }
inline int64_t r_br(const Model& M, int k, int64_t t, int64_t l) { return M.T + (k - 1) * M.T * M.L + t * M.L + l; }
inline int64_t r_k8(const Model& M, int64_t t, int64_t n) { return M.T + 7 * M.T * M.L + t * M.N + n; }
inline int64_t r_k9(const Model& M, int64_t t, int64_t n) { return M.T + 7 * M.T * M.L + M.T * M.N + t * M.N + n; }
inline int64_t r_k10(const Model& M, int64_t t, int64_t g) { return M.T + 7 * M.T * M.L + 2 * M.T * M.N + (t - 1) * M.G + g; }
inline int64_t r_k11(const Model& M, int64_t t, int64_t g) { return r_k10(M, M.T, 0) + (t - 1) * M.G + g; }

// Row kind (0..10), period, component.
void row_decode(const Model& M, int64_t i, int* kind, int64_t* t, int64_t* comp) {
  if (i < M.T) { *kind = 0; *t = i; *comp = 0; return; }
  i -= M.T;
  if (i < 7 * M.T * M.L) { *kind = 1 + (int)(i / (M.T * M.L)); i %= (M.T * M.L); *t = i / M.L; *comp = i % M.L; return; }
  i -= 7 * M.T * M.L;
  if (i < 2 * M.T * M.N) { *kind = 8 + (int)(i / (M.T * M.N)); i %= (M.T * M.N); *t = i / M.N; *comp = i % M.N; return; }
  i -= 2 * M.T * M.N;
  *kind = 10;
  if (i >= (M.T - 1) * M.G) { *kind = 11; i -= (M.T - 1) * M.G; }
  *t = 1 + i / M.G; *comp = i % M.G;
}

// Number of J entries of row i (its J order, see row_eval).
int64_t row_len(const Model& M, int64_t i) {
  int kind; int64_t t, comp;
  row_decode(M, i, &kind, &t, &comp);
  if (kind == 0) return 1;
  if (kind >= 1 && kind <= 4) return 5;
  if (kind >= 5 && kind <= 7) return 2;
  if (kind == 8 || kind == 9) return 1 + (int64_t)M.bus_gens[comp].size() + (int64_t)M.bus_arcs[comp].size();
  return 2;
}

// Rows of periods [t0, t1) as ascending index ranges [first, last).
std::vector<std::pair<int64_t, int64_t>> window_rows(const Model& M, int64_t t0, int64_t t1) {
  std::vector<std::pair<int64_t, int64_t>> r;
  r.push_back({r_k0(M, t0), r_k0(M, t1)});
  for (int k = 1; k <= 7; ++k) r.push_back({r_br(M, k, t0, 0), r_br(M, k, t1, 0)});
  r.push_back({r_k8(M, t0, 0), r_k8(M, t1, 0)});
  r.push_back({r_k9(M, t0, 0), r_k9(M, t1, 0)});
  const int64_t a = std::max<int64_t>(t0, 1), b = std::max<int64_t>(t1, 1);
  r.push_back({r_k10(M, a, 0), r_k10(M, b, 0)});
  if (M.has_qramp) r.push_back({r_k11(M, a, 0), r_k11(M, b, 0)});
  return r;
}

// Variables of periods [t0, t1) as ascending index ranges.
std::vector<std::pair<int64_t, int64_t>> window_vars(const Model& M, int64_t t0, int64_t t1) {
  return {{v_va(M, t0, 0), v_va(M, t1, 0)}, {v_vm(M, t0, 0), v_vm(M, t1, 0)}, {v_pg(M, t0, 0), v_pg(M, t1, 0)},
          {v_qg(M, t0, 0), v_qg(M, t1, 0)}, {v_p(M, t0, 0), v_p(M, t1, 0)}, {v_q(M, t0, 0), v_q(M, t1, 0)}};
}

// pi-model terms of a branch (textbook: series admittance y = 1/(r + jx),
// line charging b, off-nominal tap tau and phase shift phi):
//   Y_ff = (y + j b/2)/tau^2, Y_ft = -y/(tau e^{-j phi}), Y_tf = -y/(tau e^{j phi}),
//   Y_tt = y + j b/2.
void branch_terms(Model& M) {
  M.gff.resize(M.L); M.bff.resize(M.L); M.gft.resize(M.L); M.bft.resize(M.L);
  M.gtf.resize(M.L); M.btf.resize(M.L); M.gtt.resize(M.L); M.btt.resize(M.L);
  for (int64_t l = 0; l < M.L; ++l) {
    const double r = M.br_r[l], x = M.br_x[l], bc = M.br_b[l];
    const double den = r * r + x * x;
    const double g = r / den;
    const double b = -x / den;
    const double tau = M.tap[l], tau2 = tau * tau;
    const double cph = std::cos(M.shift[l]), sph = std::sin(M.shift[l]);
    M.gff[l] = g / tau2;
    M.bff[l] = (b + 0.5 * bc) / tau2;
    M.gft[l] = -(g * cph - b * sph) / tau;
    M.bft[l] = -(g * sph + b * cph) / tau;
    M.gtf[l] = -(g * cph + b * sph) / tau;
    M.btf[l] = -(b * cph - g * sph) / tau;
    M.gtt[l] = g;
    M.btt[l] = b + 0.5 * bc;
  }
}

// ---------------------------------------------------------------------------
// Branch quantities at one period, in the fixed rounding order.
// ---------------------------------------------------------------------------
template <class S>
struct BranchQ {
  S dth, A1, A2, A3, A4;
  S vtA1, vtA2, vfA3, vfA4, uA1, uA2, uA3, uA4;
  S Pfr, Qfr, Pto, Qto;
  S dPfr_vf, dQfr_vf, dPto_vt, dQto_vt;
  S vfA1, vfA2, vtA3, vtA4;
};

template <class S>
BranchQ<S> branch_q(const Model& M, const S* x, int64_t t, int64_t l) {
  const int64_t f = M.f[l], to = M.t[l];
  const S thf = x[v_va(M, t, f)], tht = x[v_va(M, t, to)];
  const S vf = x[v_vm(M, t, f)], vt = x[v_vm(M, t, to)];
  const double gff = M.gff[l], bff = M.bff[l], gft = M.gft[l], bft = M.bft[l];
  const double gtf = M.gtf[l], btf = M.btf[l], gtt = M.gtt[l], btt = M.btt[l];
  BranchQ<S> q;
  q.dth = thf - tht;
  S sn, cs;
  sincos_cw(q.dth, &sn, &cs);
  const S vf2 = vf * vf, vt2 = vt * vt;
  // A1 = gft C + bft S, A2 = gft S - bft C, A3 = gtf C - btf S, A4 = -gtf S - btf C
  q.A1 = fmaS(S(gft), cs, S(bft) * sn);
  q.A2 = fmaS(S(gft), sn, -(S(bft) * cs));
  q.A3 = fmaS(S(gtf), cs, -(S(btf) * sn));
  q.A4 = fmaS(S(-gtf), sn, -(S(btf) * cs));
  q.vtA1 = vt * q.A1;
  q.vtA2 = vt * q.A2;
  q.vfA3 = vf * q.A3;
  q.vfA4 = vf * q.A4;
  q.uA1 = vf * q.vtA1;
  q.uA2 = vf * q.vtA2;
  q.uA3 = vt * q.vfA3;
  q.uA4 = vt * q.vfA4;
  // Flows: P_fr = gff vf^2 + vf vt A1, Q_fr = -bff vf^2 + vf vt A2,
  //        P_to = gtt vt^2 + vf vt A3, Q_to = -btt vt^2 + vf vt A4.
  q.Pfr = fmaS(S(gff), vf2, q.uA1);
  q.Qfr = fmaS(S(-bff), vf2, q.uA2);
  q.Pto = fmaS(S(gtt), vt2, q.uA3);
  q.Qto = fmaS(S(-btt), vt2, q.uA4);
  // Derivatives in the own-end voltage: 2 g_self v_self + v_other A.
  q.dPfr_vf = fmaS(S(2.0 * gff), vf, q.vtA1);
  q.dQfr_vf = fmaS(S(-(2.0 * bff)), vf, q.vtA2);
  q.dPto_vt = fmaS(S(2.0 * gtt), vt, q.vfA3);
  q.dQto_vt = fmaS(S(-(2.0 * btt)), vt, q.vfA4);
  // Derivatives in the other-end voltage.
  q.vfA1 = vf * q.A1;
  q.vfA2 = vf * q.A2;
  q.vtA3 = vt * q.A3;
  q.vtA4 = vt * q.A4;
  return q;
}

// ---------------------------------------------------------------------------
// One constraint row: value and Jacobian entries (columns in the row's J order).
// ---------------------------------------------------------------------------
template <class S>
void row_eval(const Model& M, const S* x, int64_t i, std::vector<int64_t>* cols, std::vector<S>* vals, S* cval) {
  int kind; int64_t t, comp;
  row_decode(M, i, &kind, &t, &comp);
  cols->clear(); vals->clear();
  auto push = [&](int64_t c, S v) { cols->push_back(c); vals->push_back(v); };
  if (kind == 0) {
    *cval = x[v_va(M, t, M.ref)];
    push(v_va(M, t, M.ref), S(1.0));
    return;
  }
  if (kind >= 1 && kind <= 7) {
    const int64_t l = comp, f = M.f[l], to = M.t[l];
    const int64_t jthf = v_va(M, t, f), jtht = v_va(M, t, to), jvf = v_vm(M, t, f), jvt = v_vm(M, t, to);
    const int64_t jpf = v_p(M, t, l), jqf = v_q(M, t, l), jpt = v_p(M, t, M.L + l), jqt = v_q(M, t, M.L + l);
    if (kind == 5) {
      *cval = x[jthf] - x[jtht];
      push(jthf, S(1.0)); push(jtht, S(-1.0));
      return;
    }
    if (kind == 6 || kind == 7) {
      const int64_t jp = kind == 6 ? jpf : jpt, jq = kind == 6 ? jqf : jqt;
      const S p = x[jp], qq = x[jq];
      const double smax2 = M.smax[l] * M.smax[l];
      *cval = fmaS(p, p, fmaS(qq, qq, S(-smax2)));
      push(jp, S(2.0) * p); push(jq, S(2.0) * qq);
      return;
    }
    const BranchQ<S> q = branch_q(M, x, t, l);
    if (kind == 1) {
      *cval = x[jpf] - q.Pfr;
      push(jpf, S(1.0)); push(jthf, q.uA2); push(jtht, -q.uA2); push(jvf, -q.dPfr_vf); push(jvt, -q.vfA1);
    } else if (kind == 2) {
      *cval = x[jqf] - q.Qfr;
      push(jqf, S(1.0)); push(jthf, -q.uA1); push(jtht, q.uA1); push(jvf, -q.dQfr_vf); push(jvt, -q.vfA2);
    } else if (kind == 3) {
      *cval = x[jpt] - q.Pto;
      push(jpt, S(1.0)); push(jthf, -q.uA4); push(jtht, q.uA4); push(jvf, -q.vtA3); push(jvt, -q.dPto_vt);
    } else {
      *cval = x[jqt] - q.Qto;
      push(jqt, S(1.0)); push(jthf, q.uA3); push(jtht, -q.uA3); push(jvf, -q.vtA4); push(jvt, -q.dQto_vt);
    }
    return;
  }
  if (kind == 8 || kind == 9) {
    const int64_t n = comp;
    const bool P = kind == 8;
    const S vm = x[v_vm(M, t, n)];
    const S vm2 = vm * vm;
    S acc = S(0.0);
    for (int64_t g : M.bus_gens[n]) acc = acc + x[P ? v_pg(M, t, g) : v_qg(M, t, g)];
    for (int64_t a : M.bus_arcs[n]) acc = acc - x[P ? v_p(M, t, a) : v_q(M, t, a)];
    acc = fmaS(S(P ? -M.gs[n] : M.bs[n]), vm2, acc);
    for (int64_t d : M.bus_loads[n]) acc = acc - S(P ? M.pd[t * M.D + d] : M.qd[t * M.D + d]);
    *cval = acc;
    const double k2 = P ? -(2.0 * M.gs[n]) : 2.0 * M.bs[n];
    push(v_vm(M, t, n), S(k2) * vm);
    for (int64_t g : M.bus_gens[n]) push(P ? v_pg(M, t, g) : v_qg(M, t, g), S(1.0));
    for (int64_t a : M.bus_arcs[n]) push(P ? v_p(M, t, a) : v_q(M, t, a), S(-1.0));
    return;
  }
  // kind 10: ramp of pg; kind 11: ramp of qg
  const int64_t g = comp;
  const int64_t jt = kind == 10 ? v_pg(M, t, g) : v_qg(M, t, g), jp = kind == 10 ? v_pg(M, t - 1, g) : v_qg(M, t - 1, g);
  *cval = x[jt] - x[jp];
  push(jt, S(1.0)); push(jp, S(-1.0));
}

// ---------------------------------------------------------------------------
// Elements (pattern instances) and their W entries.
// ---------------------------------------------------------------------------
enum ElemKind { E_OBJ = 0, E_REF = 1, E_BR = 2, E_BUS = 3, E_RAMP = 4, E_QRAMP = 5 };
struct HEnt { int64_t r, c; double v; };

inline void lower_push(std::vector<HEnt>* out, int64_t a, int64_t b, double v) {
  out->push_back(HEnt{std::max(a, b), std::min(a, b), v});
}

// W entries of one element in COO order; lam may be NULL to get the pattern
// only (values then 0).
void elem_hess(const Model& M, const double* x, const double* lam, double sigma, int kind, int64_t t,
               int64_t comp, std::vector<HEnt>* out) {
  out->clear();
  if (kind == E_OBJ) {
    const int64_t g = comp;
    const double v = lam ? sigma * (2.0 * M.c2[g]) : 0.0;
    lower_push(out, v_pg(M, t, g), v_pg(M, t, g), v);
    return;
  }
  if (kind == E_BR) {
    const int64_t l = comp, f = M.f[l], to = M.t[l];
    const int64_t u[4] = {v_va(M, t, f), v_va(M, t, to), v_vm(M, t, f), v_vm(M, t, to)};
    double w[10] = {0};
    if (lam) {
      const BranchQ<double> q = branch_q(M, x, t, l);
      const double l1 = lam[r_br(M, 1, t, l)], l2 = lam[r_br(M, 2, t, l)];
      const double l3 = lam[r_br(M, 3, t, l)], l4 = lam[r_br(M, 4, t, l)];
      const double vf = x[u[2]], vt = x[u[3]];
      // W = sum_k lambda_k grad^2 c_k with c_k = arc_k - E_k (E_k the flow).
      const double Asum = std::fma(l4, q.A4, std::fma(l3, q.A3, std::fma(l2, q.A2, l1 * q.A1)));
      const double Bsum = std::fma(l4, q.A3, std::fma(-l3, q.A4, std::fma(-l2, q.A1, l1 * q.A2)));
      const double Wdd = vf * (vt * Asum);
      const double Wdvf = vt * Bsum;
      const double Wdvt = vf * Bsum;
      const double Wvfvf = std::fma(l2, 2.0 * M.bff[l], -(l1 * (2.0 * M.gff[l])));
      const double Wvtvt = std::fma(l4, 2.0 * M.btt[l], -(l3 * (2.0 * M.gtt[l])));
      const double Wvfvt = -Asum;
      const double vals[10] = {Wdd, -Wdd, Wdd, Wdvf, -Wdvf, Wvfvf, Wdvt, -Wdvt, Wvfvt, Wvtvt};
      std::memcpy(w, vals, sizeof w);
    }
    const int pa[10] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
    const int pb[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
    for (int e = 0; e < 10; ++e) lower_push(out, u[pa[e]], u[pb[e]], w[e]);
    return;
  }
  if (kind == E_BUS) {
    const int64_t nb = comp;
    const int64_t j = v_vm(M, t, nb);
    const double wp = lam ? lam[r_k8(M, t, nb)] * -(2.0 * M.gs[nb]) : 0.0;
    const double wq = lam ? lam[r_k9(M, t, nb)] * (2.0 * M.bs[nb]) : 0.0;
    lower_push(out, j, j, wp);
    lower_push(out, j, j, wq);
    return;
  }
}

// Thermal W entries of a branch element (Hessian group 3): from p, from q, to p, to q.
void elem_hess_thermal(const Model& M, const double* lam, int64_t t, int64_t l, std::vector<HEnt>* out) {
  const double h6 = lam ? 2.0 * lam[r_br(M, 6, t, l)] : 0.0;
  const double h7 = lam ? 2.0 * lam[r_br(M, 7, t, l)] : 0.0;
  lower_push(out, v_p(M, t, l), v_p(M, t, l), h6);
  lower_push(out, v_q(M, t, l), v_q(M, t, l), h6);
  lower_push(out, v_p(M, t, M.L + l), v_p(M, t, M.L + l), h7);
  lower_push(out, v_q(M, t, M.L + l), v_q(M, t, M.L + l), h7);
}

// All W entries of an element, in COO order.
void elem_w(const Model& M, const double* x, const double* lam, double sigma, int kind, int64_t t, int64_t comp,
            std::vector<HEnt>* out) {
  elem_hess(M, x, lam, sigma, kind, t, comp, out);
  if (kind == E_BR) elem_hess_thermal(M, lam, t, comp, out);
}

// J rows of an element, ascending.
void elem_rows(const Model& M, int kind, int64_t t, int64_t comp, std::vector<int64_t>* rows) {
  rows->clear();
  if (kind == E_REF) rows->push_back(r_k0(M, t));
  if (kind == E_BR) for (int k = 1; k <= 7; ++k) rows->push_back(r_br(M, k, t, comp));
  if (kind == E_BUS) { rows->push_back(r_k8(M, t, comp)); rows->push_back(r_k9(M, t, comp)); }
  if (kind == E_RAMP) rows->push_back(r_k10(M, t, comp));
  if (kind == E_QRAMP) rows->push_back(r_k11(M, t, comp));
}

int64_t elem_count(const Model& M, int kind) {
  switch (kind) {
    case E_OBJ: return M.G;
    case E_REF: return 1;
    case E_BR: return M.L;
    case E_BUS: return M.N;
    default: return M.G;
  }
}

// Visit every element whose period touches [t0, t1), in canonical order.
// Ramp elements of period t touch pg at t and t-1, so t = t1 is included.
template <class F>
void for_elements(const Model& M, int64_t t0, int64_t t1, F fn) {
  for (int kind = E_OBJ; kind <= E_QRAMP; ++kind) {
    if (kind == E_QRAMP && !M.has_qramp) break;
    int64_t ta = t0, tb = t1;
    if (kind == E_RAMP || kind == E_QRAMP) { ta = std::max<int64_t>(t0, 1); tb = std::min<int64_t>(t1 + 1, M.T); }
    for (int64_t t = ta; t < tb; ++t)
      for (int64_t c = 0; c < elem_count(M, kind); ++c) fn(kind, t, c);
  }
}

bool var_in_window(const Model& M, int64_t j, int64_t t0, int64_t t1) {
  int kind; int64_t t, comp;
  var_decode(M, j, &kind, &t, &comp);
  return t >= t0 && t < t1;
}

}  // namespace

// ===========================================================================
// C interface (ctypes).
// ===========================================================================
extern "C" {

void* orc_new(const int64_t* dims /* N, L, G, D, ref, T */,
              const double* bus /* [4][N]: gs, bs, vmin, vmax */,
              const int32_t* br_ft /* [2][L] */, const double* br /* [8][L]: r, x, b, tap, shift, smax, angmin, angmax */,
              const int32_t* gen_bus, const double* gen /* [8][G]: c2, c1, c0, pmin, pmax, qmin, qmax, ramp */,
              const int32_t* load_bus, const double* pd, const double* qd,
              const double* qramp /* [G] reactive ramp limits, or NULL for none */) {
  Model* M = new Model();
  M->N = dims[0]; M->L = dims[1]; M->G = dims[2]; M->D = dims[3]; M->ref = dims[4]; M->T = dims[5];
  const int64_t N = M->N, L = M->L, G = M->G, D = M->D, T = M->T;
  auto cp = [](const double* p, int64_t n) { return std::vector<double>(p, p + n); };
  M->gs = cp(bus, N); M->bs = cp(bus + N, N); M->vmin = cp(bus + 2 * N, N); M->vmax = cp(bus + 3 * N, N);
  M->f.assign(br_ft, br_ft + L); M->t.assign(br_ft + L, br_ft + 2 * L);
  M->br_r = cp(br, L); M->br_x = cp(br + L, L); M->br_b = cp(br + 2 * L, L); M->tap = cp(br + 3 * L, L);
  M->shift = cp(br + 4 * L, L); M->smax = cp(br + 5 * L, L); M->angmin = cp(br + 6 * L, L); M->angmax = cp(br + 7 * L, L);
  M->gbus.assign(gen_bus, gen_bus + G);
  M->c2 = cp(gen, G); M->c1 = cp(gen + G, G); M->c0 = cp(gen + 2 * G, G); M->pmin = cp(gen + 3 * G, G);
  M->pmax = cp(gen + 4 * G, G); M->qmin = cp(gen + 5 * G, G); M->qmax = cp(gen + 6 * G, G); M->ramp = cp(gen + 7 * G, G);
  M->has_qramp = qramp != nullptr;
  if (M->has_qramp) M->qramp = cp(qramp, G);
  M->lbus.assign(load_bus, load_bus + D);
  M->pd = cp(pd, T * D); M->qd = cp(qd, T * D);
  branch_terms(*M);
  M->bus_gens.assign(N, {}); M->bus_arcs.assign(N, {}); M->bus_loads.assign(N, {});
  for (int64_t g = 0; g < G; ++g) M->bus_gens[M->gbus[g]].push_back(g);
  for (int64_t a = 0; a < 2 * L; ++a) M->bus_arcs[a < L ? M->f[a] : M->t[a - L]].push_back(a);
  for (int64_t d = 0; d < D; ++d) M->bus_loads[M->lbus[d]].push_back(d);
  M->n = T * (2 * N + 2 * G + 4 * L);
  M->m = T * (1 + 7 * L + 2 * N) + G * (T - 1) * (M->has_qramp ? 2 : 1);
  M->jrp.assign(M->m + 1, 0);
  for (int64_t i = 0; i < M->m; ++i) M->jrp[i + 1] = M->jrp[i] + row_len(*M, i);
  return M;
}

void orc_free(void* h) { delete static_cast<Model*>(h); }

// n, m, nnz of J, nnz of W (H).
void orc_sizes(void* h, int64_t* out) {
  const Model& M = *static_cast<Model*>(h);
  out[0] = M.n; out[1] = M.m; out[2] = M.jrp[M.m];
  out[3] = M.T * (M.G + 10 * M.L + 4 * M.L + 2 * M.N);
}

// Variable bounds x^flat, x^sharp and row bounds of Eq. (3).
void orc_bounds(void* h, double* xl, double* xu, double* gl, double* gu) {
  const Model& M = *static_cast<Model*>(h);
  const double inf = INFINITY;
  for (int64_t t = 0; t < M.T; ++t) {
    for (int64_t i = 0; i < M.N; ++i) {
      xl[v_va(M, t, i)] = -inf; xu[v_va(M, t, i)] = inf;
      xl[v_vm(M, t, i)] = M.vmin[i]; xu[v_vm(M, t, i)] = M.vmax[i];
    }
    for (int64_t g = 0; g < M.G; ++g) {
      xl[v_pg(M, t, g)] = M.pmin[g]; xu[v_pg(M, t, g)] = M.pmax[g];
      xl[v_qg(M, t, g)] = M.qmin[g]; xu[v_qg(M, t, g)] = M.qmax[g];
    }
    for (int64_t a = 0; a < 2 * M.L; ++a) {
      xl[v_p(M, t, a)] = -inf; xu[v_p(M, t, a)] = inf;
      xl[v_q(M, t, a)] = -inf; xu[v_q(M, t, a)] = inf;
    }
  }
  for (int64_t i = 0; i < M.m; ++i) {
    int kind; int64_t t, comp;
    row_decode(M, i, &kind, &t, &comp);
    double lo = 0.0, hi = 0.0;
    if (kind == 5) { lo = M.angmin[comp]; hi = M.angmax[comp]; }
    if (kind == 6 || kind == 7) { lo = -inf; hi = 0.0; }
    if (kind == 10) { lo = -M.ramp[comp]; hi = M.ramp[comp]; }
    if (kind == 11) { lo = -M.qramp[comp]; hi = M.qramp[comp]; }
    gl[i] = lo; gu[i] = hi;
  }
}

// J pattern: rows ascending, entries of a row in its J order.
void orc_jac_pattern(void* h, int32_t* rows, int32_t* cols) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<double> x(M.n, 1.0);
  std::vector<int64_t> c; std::vector<double> v; double cv;
  int64_t k = 0;
  for (int64_t i = 0; i < M.m; ++i) {
    row_eval<double>(M, x.data(), i, &c, &v, &cv);
    for (size_t e = 0; e < c.size(); ++e) { rows[k] = (int32_t)i; cols[k] = (int32_t)c[e]; ++k; }
  }
}

// W pattern: objective (t, g), branch blocks (t, l), thermal (t, l), shunt (t, n).
void orc_hess_pattern(void* h, int32_t* rows, int32_t* cols) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<HEnt> e;
  int64_t k = 0;
  auto emit = [&]() { for (auto& q : e) { rows[k] = (int32_t)q.r; cols[k] = (int32_t)q.c; ++k; } };
  for (int64_t t = 0; t < M.T; ++t) for (int64_t g = 0; g < M.G; ++g) { elem_hess(M, nullptr, nullptr, 0, E_OBJ, t, g, &e); emit(); }
  for (int64_t t = 0; t < M.T; ++t) for (int64_t l = 0; l < M.L; ++l) { elem_hess(M, nullptr, nullptr, 0, E_BR, t, l, &e); emit(); }
  for (int64_t t = 0; t < M.T; ++t) for (int64_t l = 0; l < M.L; ++l) { e.clear(); elem_hess_thermal(M, nullptr, t, l, &e); emit(); }
  for (int64_t t = 0; t < M.T; ++t) for (int64_t n = 0; n < M.N; ++n) { elem_hess(M, nullptr, nullptr, 0, E_BUS, t, n, &e); emit(); }
}

// Offsets of the J entries of each row (int64 [m + 1]) — positions in the COO arrays.
void orc_jac_rowptr(void* h, int64_t* rp) {
  const Model& M = *static_cast<Model*>(h);
  for (int64_t i = 0; i <= M.m; ++i) rp[i] = M.jrp[i];
}

// Objective, gradient, constraints, J values and W values restricted to the
// periods [t0, t1): f sums the objective terms of those periods; g, c and J
// cover variables and rows of those periods (ramp row (t, g) belongs to t);
// W covers elements of those periods.  Entries outside the window are left
// untouched.  Any output pointer may be NULL.
void orc_eval(void* h, int64_t t0, int64_t t1, const double* x, const double* lam, double sigma,
              double* fobj, double* grad, double* c, double* jv, double* hv) {
  const Model& M = *static_cast<Model*>(h);
  if (fobj) {
    double acc = 0.0;
    for (int64_t t = t0; t < t1; ++t)
      for (int64_t g = 0; g < M.G; ++g) {
        const double pg = x[v_pg(M, t, g)];
        acc = acc + std::fma(std::fma(M.c2[g], pg, M.c1[g]), pg, M.c0[g]);
      }
    *fobj = acc;
  }
  if (grad) {
    for (const auto& rg : window_vars(M, t0, t1))
      for (int64_t j = rg.first; j < rg.second; ++j) {
        int kind; int64_t t, comp;
        var_decode(M, j, &kind, &t, &comp);
        grad[j] = kind == 2 ? std::fma(2.0 * M.c2[comp], x[j], M.c1[comp]) : 0.0;
      }
  }
  if (c || jv) {
    std::vector<int64_t> cols; std::vector<double> vals; double cv;
    for (const auto& rg : window_rows(M, t0, t1))
      for (int64_t i = rg.first; i < rg.second; ++i) {
        row_eval<double>(M, x, i, &cols, &vals, &cv);
        if (c) c[i] = cv;
        if (jv) for (size_t e = 0; e < vals.size(); ++e) jv[M.jrp[i] + e] = vals[e];
      }
  }
  if (hv) {
    std::vector<HEnt> e;
    const int64_t off_br = M.T * M.G, off_th = off_br + 10 * M.T * M.L, off_sh = off_th + 4 * M.T * M.L;
    for (int64_t t = t0; t < t1; ++t) {
      for (int64_t g = 0; g < M.G; ++g) {
        elem_hess(M, x, lam, sigma, E_OBJ, t, g, &e);
        hv[t * M.G + g] = e[0].v;
      }
      for (int64_t l = 0; l < M.L; ++l) {
        elem_hess(M, x, lam, sigma, E_BR, t, l, &e);
        for (int k = 0; k < 10; ++k) hv[off_br + (t * M.L + l) * 10 + k] = e[k].v;
        e.clear();
        elem_hess_thermal(M, lam, t, l, &e);
        for (int k = 0; k < 4; ++k) hv[off_th + (t * M.L + l) * 4 + k] = e[k].v;
      }
      for (int64_t n = 0; n < M.N; ++n) {
        elem_hess(M, x, lam, sigma, E_BUS, t, n, &e);
        hv[off_sh + (t * M.N + n) * 2] = e[0].v;
        hv[off_sh + (t * M.N + n) * 2 + 1] = e[1].v;
      }
    }
  }
}

}  // extern "C"

namespace {
// Rows of the condensed matrix for the variables of a window of periods:
// global row index and length of each row, then the columns (ascending) and
// values of every row in turn.
struct KktRows {
  std::vector<int64_t> rows, rowlen;
  std::vector<int32_t> cols;
  std::vector<double> vals;
};

// Local block of one element: (key, value) pairs, each key once, values
// accumulated in the stated order.
struct Local {
  std::vector<std::pair<std::pair<int64_t, int64_t>, double>> e;
  double& at(int64_t r, int64_t c) {
    for (auto& kv : e)
      if (kv.first.first == r && kv.first.second == c) return kv.second;
    e.push_back({{r, c}, 0.0});
    return e.back().second;
  }
};

void kkt_compute(const Model& M, int64_t t0, int64_t t1, const double* x, const double* lam, double sigma,
                 const double* sigx, const double* dvec, double delta_w, KktRows* out) {
  // Contributions in the order they are added: diagonal terms first, then
  // every element's local values in element order.  A stable sort by key
  // keeps that order within each key; each key is then summed left to right.
  std::vector<std::pair<std::pair<int64_t, int64_t>, double>> contrib;
  std::vector<int64_t> wrows;
  for (const auto& rg : window_vars(M, t0, t1))
    for (int64_t j = rg.first; j < rg.second; ++j) {
      wrows.push_back(j);
      contrib.push_back({{j, j}, sigx[j] + delta_w});
    }
  std::vector<HEnt> we;
  std::vector<int64_t> erows, cols_i;
  std::vector<double> vals_i;
  double cv;
  Local loc;
  for_elements(M, t0, t1, [&](int kind, int64_t t, int64_t comp) {
    loc.e.clear();
    elem_w(M, x, lam, sigma, kind, t, comp, &we);
    for (const HEnt& e : we) {
      double& slot = loc.at(e.r, e.c);
      slot = slot + e.v;
    }
    elem_rows(M, kind, t, comp, &erows);
    for (int64_t i : erows) {
      row_eval<double>(M, x, i, &cols_i, &vals_i, &cv);
      const double Di = dvec[i];
      for (size_t p = 0; p < cols_i.size(); ++p) {
        const double w = Di * vals_i[p];
        for (size_t q = 0; q <= p; ++q) {
          double& slot = loc.at(std::max(cols_i[p], cols_i[q]), std::min(cols_i[p], cols_i[q]));
          slot = std::fma(w, vals_i[q], slot);
        }
      }
    }
    for (const auto& kv : loc.e)
      if (var_in_window(M, kv.first.first, t0, t1)) contrib.push_back(kv);
  });
  std::stable_sort(contrib.begin(), contrib.end(),
                   [](const auto& a, const auto& b) { return a.first < b.first; });
  out->rows.clear(); out->rowlen.clear(); out->cols.clear(); out->vals.clear();
  size_t k = 0;
  while (k < contrib.size()) {
    const auto key = contrib[k].first;
    double acc = 0.0;
    for (; k < contrib.size() && contrib[k].first == key; ++k) acc = acc + contrib[k].second;
    if (out->rows.empty() || out->rows.back() != key.first) {
      out->rows.push_back(key.first);
      out->rowlen.push_back(0);
    }
    out->rowlen.back() += 1;
    out->cols.push_back((int32_t)key.second);
    out->vals.push_back(acc);
  }
}
}  // namespace

// Condensed matrix rows for the variables of periods [t0, t1), in global row
// order, in two explicit steps: orc_kkt_new computes them into a result object
// that the caller owns; orc_kkt_sizes reports its row and entry counts;
// orc_kkt_copy writes the global row index and length of each row and the
// columns and values of all rows; orc_kkt_free releases it.
extern "C" void* orc_kkt_new(void* h, int64_t t0, int64_t t1, const double* x, const double* lam, double sigma,
                             const double* sigx, const double* dvec, double delta_w) {
  const Model& M = *static_cast<Model*>(h);
  KktRows* out = new KktRows();
  kkt_compute(M, t0, t1, x, lam, sigma, sigx, dvec, delta_w, out);
  return out;
}

// sizes[0] = number of rows, sizes[1] = number of entries.
extern "C" void orc_kkt_sizes(const void* res, int64_t* sizes) {
  const KktRows& R = *static_cast<const KktRows*>(res);
  sizes[0] = (int64_t)R.rows.size();
  sizes[1] = (int64_t)R.cols.size();
}

extern "C" void orc_kkt_copy(const void* res, int64_t* rows_out, int64_t* rowlen, int32_t* cols, double* vals) {
  const KktRows& R = *static_cast<const KktRows*>(res);
  for (size_t r = 0; r < R.rows.size(); ++r) { rows_out[r] = R.rows[r]; rowlen[r] = R.rowlen[r]; }
  std::memcpy(cols, R.cols.data(), R.cols.size() * sizeof(int32_t));
  std::memcpy(vals, R.vals.data(), R.vals.size() * sizeof(double));
}

extern "C" void orc_kkt_free(void* res) { delete static_cast<KktRows*>(res); }

extern "C" {

// Number of window rows of orc_kkt.
int64_t orc_window_rows(void* h, int64_t t0, int64_t t1) {
  const Model& M = *static_cast<Model*>(h);
  return (t1 - t0) * (2 * M.N + 2 * M.G + 4 * M.L);
}

// J^T y for the variables of periods [t0, t1), element by element: each
// element's local sum over its rows ascending, fma(J_ij, y_i, .), then added
// into gx in element order.  gpd/gqd (may be NULL): the load adjoint
// (dc/dPd)^T y = -y at the P-balance row of the load's bus (Q likewise).
void orc_vjp(void* h, int64_t t0, int64_t t1, const double* x, const double* y, double* gx, double* gpd, double* gqd) {
  const Model& M = *static_cast<Model*>(h);
  for (const auto& rg : window_vars(M, t0, t1))
    for (int64_t j = rg.first; j < rg.second; ++j) gx[j] = 0.0;
  std::vector<int64_t> erows, cols_i;
  std::vector<double> vals_i;
  double cv;
  for_elements(M, t0, t1, [&](int kind, int64_t t, int64_t comp) {
    std::map<int64_t, double> loc;
    elem_rows(M, kind, t, comp, &erows);
    for (int64_t i : erows) {
      row_eval<double>(M, x, i, &cols_i, &vals_i, &cv);
      for (size_t p = 0; p < cols_i.size(); ++p) {
        double& slot = loc[cols_i[p]];
        slot = std::fma(vals_i[p], y[i], slot);
      }
    }
    for (const auto& kv : loc) if (var_in_window(M, kv.first, t0, t1)) gx[kv.first] += kv.second;
  });
  for (int64_t t = t0; t < t1; ++t)
    for (int64_t d = 0; d < M.D; ++d) {
      if (gpd) gpd[t * M.D + d] = -y[r_k8(M, t, M.lbus[d])];
      if (gqd) gqd[t * M.D + d] = -y[r_k9(M, t, M.lbus[d])];
    }
}

// W v for the variables of periods [t0, t1), element by element: for each W
// entry (r, c, w) of the element in COO order, loc[r] = fma(w, v[c], loc[r])
// and, off the diagonal, loc[c] = fma(w, v[r], loc[c]); then added into hv in
// element order.
void orc_hvp(void* h, int64_t t0, int64_t t1, const double* x, const double* lam, double sigma, const double* v,
             double* hv) {
  const Model& M = *static_cast<Model*>(h);
  for (const auto& rg : window_vars(M, t0, t1))
    for (int64_t j = rg.first; j < rg.second; ++j) hv[j] = 0.0;
  std::vector<HEnt> we;
  for_elements(M, t0, t1, [&](int kind, int64_t t, int64_t comp) {
    std::map<int64_t, double> loc;
    elem_w(M, x, lam, sigma, kind, t, comp, &we);
    for (const HEnt& e : we) {
      double& a = loc[e.r];
      a = std::fma(e.v, v[e.c], a);
      if (e.r != e.c) {
        double& b = loc[e.c];
        b = std::fma(e.v, v[e.r], b);
      }
    }
    for (const auto& kv : loc) if (var_in_window(M, kv.first, t0, t1)) hv[kv.first] += kv.second;
  });
}

// J v for the rows of periods [t0, t1): acc = fma(J_ip, v[col_p], acc) over
// the row's J order.  With load tangents dpd/dqd ([T][D], may be NULL) the
// balance rows also get the load term: dc/dPd = -1, so acc = acc - dpd[t][d]
// for the loads of the bus in ascending order (the tangent of c(x, Pd, Qd)).
void orc_jvp(void* h, int64_t t0, int64_t t1, const double* x, const double* v, const double* dpd,
             const double* dqd, double* out) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<int64_t> cols; std::vector<double> vals; double cv;
  for (const auto& rg : window_rows(M, t0, t1))
    for (int64_t i = rg.first; i < rg.second; ++i) {
      row_eval<double>(M, x, i, &cols, &vals, &cv);
      double acc = 0.0;
      for (size_t p = 0; p < cols.size(); ++p) acc = std::fma(vals[p], v[cols[p]], acc);
      int kind; int64_t t, comp;
      row_decode(M, i, &kind, &t, &comp);
      const double* dl = kind == 8 ? dpd : kind == 9 ? dqd : nullptr;
      if (dl)
        for (int64_t d : M.bus_loads[comp]) acc = acc - dl[t * M.D + d];
      out[i] = acc;
    }
}

// ---------------------------------------------------------------------------
// Interior-point algebra around the condensed matrix (Sec. III-B).
// Bounds: x in [xl, xu] (Eq. 1g-1i), slacks s in [sl, su] with sl = gl, su = gu
// for inequality rows and the relaxation gl - eps, gu + eps for equality rows
// (gl == gu; the paper relaxes g(x) = 0 to s in [-eps, eps]).  An infinite
// bound contributes nothing (its dual is taken as 0).
// For v in {x, s} with distances dl = v - vl, du = vu - v to its finite bounds:
//   rl = 1/dl, ru = 1/du                      (0 for an infinite bound)
//   Sigma = fma(zl, rl, zu ru)
//   C = 1 / fma(delta_c, Sigma_s, 1 + delta_c delta_w),  D = (Sigma_s + delta_w) C
// Eliminating the bound-dual rows of Eq. 5 (complementarity zl dl - mu) from
// the dual rows, the dual terms cancel: -zl + (zl dl - mu)/dl = -mu rl, so
//   q_x = fma(mu, ru - rl, grad) - J^T y,   q_s = fma(mu, ru - rl, y),
//   q_y = c - s,
//   rhs = fma(mu, ru_x - rl_x, grad) + J^T w,  w = fma(C, q_s, D q_y) - y
//     (J^T y of q_x and J^T (C q_s + D q_y) merged into one product),
//   ds = C (fma(delta_c, q_s, J dx) - q_y)   (eliminating rows 2-3 of Eq. 5)
//   dy = fma(Sigma_s + delta_w, ds, -q_s)
//   dzl = fma(-rl, fma(zl, dv, mu), zl)  = ((zl dl - mu) - zl dv) / dl
//   dzu = fma(-ru, fma(-zu, dv, mu), zu) = ((zu du - mu) + zu dv) / du
// ---------------------------------------------------------------------------
namespace {
struct Recip {
  double rl, ru;
  bool has_l, has_u;
};
Recip recips(double v, double lo, double hi) {
  Recip r{0.0, 0.0, std::isfinite(lo), std::isfinite(hi)};
  if (r.has_l) r.rl = 1.0 / (v - lo);
  if (r.has_u) r.ru = 1.0 / (hi - v);
  return r;
}
double sigma_of(const Recip& r, double zl, double zu) { return std::fma(zl, r.rl, zu * r.ru); }
void slack_bounds(double gl, double gu, double eps, double* sl, double* su) {
  if (gl == gu) { *sl = gl - eps; *su = gu + eps; } else { *sl = gl; *su = gu; }
}
}  // namespace

extern "C" {

// Sigma_x [n]; D, C [m]; if not NULL: Sigma_s [m] and the reciprocals
// recip [2n + 2m] = rl_x [n], ru_x [n], rl_s [m], ru_s [m].
void orc_ipm_prepare(void* h, const double* x, const double* s, const double* zlx, const double* zux, const double* zls,
                     const double* zus, double delta_w, double delta_c, double eps, double* sigx, double* dvec,
                     double* cvec, double* sigs, double* recip) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<double> xl(M.n), xu(M.n), gl(M.m), gu(M.m);
  orc_bounds(h, xl.data(), xu.data(), gl.data(), gu.data());
  for (int64_t j = 0; j < M.n; ++j) {
    const Recip r = recips(x[j], xl[j], xu[j]);
    sigx[j] = sigma_of(r, zlx[j], zux[j]);
    if (recip) { recip[j] = r.rl; recip[M.n + j] = r.ru; }
  }
  const double e = 1.0 + delta_c * delta_w;
  for (int64_t i = 0; i < M.m; ++i) {
    double sl, su;
    slack_bounds(gl[i], gu[i], eps, &sl, &su);
    const Recip r = recips(s[i], sl, su);
    const double sg = sigma_of(r, zls[i], zus[i]);
    const double c = 1.0 / std::fma(delta_c, sg, e);
    cvec[i] = c;
    dvec[i] = (sg + delta_w) * c;
    if (sigs) sigs[i] = sg;
    if (recip) { recip[2 * M.n + i] = r.rl; recip[2 * M.n + M.m + i] = r.ru; }
  }
}

// Condensed right-hand side rhs [n]; w [m] (if not NULL) is the row vector of
// the merged transposed product.
void orc_ipm_rhs(void* h, const double* x, const double* s, const double* y, const double* zlx, const double* zux,
                 const double* zls, const double* zus, const double* grad, const double* c, double mu,
                 double delta_w, double delta_c, double eps, double* rhs, double* w_out) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<double> xl(M.n), xu(M.n), gl(M.m), gu(M.m), w(M.m), jt(M.n);
  orc_bounds(h, xl.data(), xu.data(), gl.data(), gu.data());
  const double e = 1.0 + delta_c * delta_w;
  for (int64_t i = 0; i < M.m; ++i) {
    double sl, su;
    slack_bounds(gl[i], gu[i], eps, &sl, &su);
    const Recip r = recips(s[i], sl, su);
    const double sg = sigma_of(r, zls[i], zus[i]);
    const double cc = 1.0 / std::fma(delta_c, sg, e);
    const double dd = (sg + delta_w) * cc;
    const double qs = std::fma(mu, r.ru - r.rl, y[i]);
    const double qy = c[i] - s[i];
    w[i] = std::fma(cc, qs, dd * qy) - y[i];
  }
  orc_vjp(h, 0, M.T, x, w.data(), jt.data(), nullptr, nullptr);
  for (int64_t j = 0; j < M.n; ++j) {
    const Recip r = recips(x[j], xl[j], xu[j]);
    rhs[j] = std::fma(mu, r.ru - r.rl, grad[j]) + jt[j];
  }
  if (w_out) for (int64_t i = 0; i < M.m; ++i) w_out[i] = w[i];
}

// Step recovery from dx [n]: ds, dy, dzl_s, dzu_s [m]; dzl_x, dzu_x [n].
void orc_ipm_recover(void* h, const double* x, const double* s, const double* y, const double* zlx, const double* zux,
                     const double* zls, const double* zus, const double* c, const double* dx, double mu,
                     double delta_w, double delta_c, double eps, double* ds, double* dy, double* dzlx,
                     double* dzux, double* dzls, double* dzus) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<double> xl(M.n), xu(M.n), gl(M.m), gu(M.m), jdx(M.m);
  orc_bounds(h, xl.data(), xu.data(), gl.data(), gu.data());
  orc_jvp(h, 0, M.T, x, dx, nullptr, nullptr, jdx.data());
  const double e = 1.0 + delta_c * delta_w;
  for (int64_t i = 0; i < M.m; ++i) {
    double sl, su;
    slack_bounds(gl[i], gu[i], eps, &sl, &su);
    const Recip r = recips(s[i], sl, su);
    const double sg = sigma_of(r, zls[i], zus[i]);
    const double cc = 1.0 / std::fma(delta_c, sg, e);
    const double qs = std::fma(mu, r.ru - r.rl, y[i]);
    const double qy = c[i] - s[i];
    const double d = cc * (std::fma(delta_c, qs, jdx[i]) - qy);
    ds[i] = d;
    dy[i] = std::fma(sg + delta_w, d, -qs);
    dzls[i] = r.has_l ? std::fma(-r.rl, std::fma(zls[i], d, mu), zls[i]) : 0.0;
    dzus[i] = r.has_u ? std::fma(-r.ru, std::fma(-zus[i], d, mu), zus[i]) : 0.0;
  }
  for (int64_t j = 0; j < M.n; ++j) {
    const Recip r = recips(x[j], xl[j], xu[j]);
    dzlx[j] = r.has_l ? std::fma(-r.rl, std::fma(zlx[j], dx[j], mu), zlx[j]) : 0.0;
    dzux[j] = r.has_u ? std::fma(-r.ru, std::fma(-zux[j], dx[j], mu), zux[j]) : 0.0;
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// COO -> CSC compression of J and of the lower-triangle W (Sec. III-A: the
// COO matrices may be compressed to CSC).  Plain definition: entries ordered
// by (column, row); entries with the same (row, column) (only W has them) are
// one CSC entry whose value is their sum, added in COO order starting from the
// first.  which = 0: J (m x n), which = 1: W (n x n, lower triangle).
// ---------------------------------------------------------------------------
namespace {
struct CooEntry {
  int32_t col, row;
  int64_t e;
};
std::vector<CooEntry> coo_sorted(void* h, int32_t which) {
  int64_t sz[4];
  orc_sizes(h, sz);
  const int64_t nnz = which == 0 ? sz[2] : sz[3];
  std::vector<int32_t> r(nnz), c(nnz);
  if (which == 0) orc_jac_pattern(h, r.data(), c.data());
  else orc_hess_pattern(h, r.data(), c.data());
  std::vector<CooEntry> v(nnz);
  for (int64_t e = 0; e < nnz; ++e) v[e] = CooEntry{c[e], r[e], e};
  std::sort(v.begin(), v.end(), [](const CooEntry& a, const CooEntry& b) {
    if (a.col != b.col) return a.col < b.col;
    if (a.row != b.row) return a.row < b.row;
    return a.e < b.e;
  });
  return v;
}
}  // namespace

extern "C" {
int64_t orc_csc_nnz(void* h, int32_t which) {
  const std::vector<CooEntry> v = coo_sorted(h, which);
  int64_t k = 0;
  for (size_t p = 0; p < v.size(); ++p)
    if (p == 0 || v[p].col != v[p - 1].col || v[p].row != v[p - 1].row) ++k;
  return k;
}

// colptr [ncols + 1], rowidx [orc_csc_nnz]; vals (if coo != NULL) [orc_csc_nnz].
void orc_csc(void* h, int32_t which, const double* coo, int64_t* colptr, int32_t* rowidx, double* vals) {
  const Model& M = *static_cast<Model*>(h);
  const std::vector<CooEntry> v = coo_sorted(h, which);
  for (int64_t j = 0; j <= M.n; ++j) colptr[j] = 0;
  int64_t k = -1;
  for (size_t p = 0; p < v.size(); ++p) {
    const bool fresh = p == 0 || v[p].col != v[p - 1].col || v[p].row != v[p - 1].row;
    if (fresh) {
      ++k;
      rowidx[k] = v[p].row;
      colptr[v[p].col + 1] += 1;
      if (coo) vals[k] = coo[v[p].e];
    } else if (coo) {
      vals[k] = vals[k] + coo[v[p].e];
    }
  }
  for (int64_t j = 0; j < M.n; ++j) colptr[j + 1] += colptr[j];
}
}  // extern "C"

// The canonical sin/cos (for pins against the C library).
void orc_sincos(const double* x, int64_t n, double* s, double* c) {
  for (int64_t i = 0; i < n; ++i) sincos_cw(x[i], &s[i], &c[i]);
}

// Gradient of the Lagrangian sigma grad f + J^T lam (plain sums, row order),
// at a real point, and its complex-step directional derivative
// Im(gradL(x + i h dx)) / h, which is W dx exactly up to rounding.
void orc_gradlag(void* h, const double* x, const double* lam, double sigma, double* out) {
  const Model& M = *static_cast<Model*>(h);
  for (int64_t j = 0; j < M.n; ++j) out[j] = 0.0;
  for (int64_t t = 0; t < M.T; ++t)
    for (int64_t g = 0; g < M.G; ++g) {
      const int64_t j = v_pg(M, t, g);
      out[j] += sigma * (2.0 * M.c2[g] * x[j] + M.c1[g]);
    }
  std::vector<int64_t> cols; std::vector<double> vals; double cv;
  for (int64_t i = 0; i < M.m; ++i) {
    row_eval<double>(M, x, i, &cols, &vals, &cv);
    for (size_t p = 0; p < cols.size(); ++p) out[cols[p]] += vals[p] * lam[i];
  }
}

void orc_gradlag_cstep(void* h, const double* x, const double* lam, double sigma, const double* dx, double hstep,
                       double* out) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<cplx> xc(M.n), acc(M.n, cplx(0.0, 0.0));
  for (int64_t j = 0; j < M.n; ++j) xc[j] = cplx(x[j], hstep * dx[j]);
  for (int64_t t = 0; t < M.T; ++t)
    for (int64_t g = 0; g < M.G; ++g) {
      const int64_t j = v_pg(M, t, g);
      acc[j] += sigma * (2.0 * M.c2[g] * xc[j] + M.c1[g]);
    }
  std::vector<int64_t> cols; std::vector<cplx> vals; cplx cv;
  for (int64_t i = 0; i < M.m; ++i) {
    row_eval<cplx>(M, xc.data(), i, &cols, &vals, &cv);
    for (size_t p = 0; p < cols.size(); ++p) acc[cols[p]] += vals[p] * lam[i];
  }
  for (int64_t j = 0; j < M.n; ++j) out[j] = acc[j].imag() / hstep;
}

}  // extern "C"

// ===========================================================================
// Textbook constraint evaluation for the pins: plain expressions, C-library
// sin/cos, no fma, written independently of the rounding-order code above.
// Templated so that a complex step gives exact directional derivatives.
// ===========================================================================
namespace {
template <class S>
void cons_textbook(const Model& M, const S* x, S* c) {
  for (int64_t t = 0; t < M.T; ++t) {
    c[r_k0(M, t)] = x[v_va(M, t, M.ref)];
    for (int64_t l = 0; l < M.L; ++l) {
      const int64_t f = M.f[l], to = M.t[l];
      const S thf = x[v_va(M, t, f)], tht = x[v_va(M, t, to)];
      const S vf = x[v_vm(M, t, f)], vt = x[v_vm(M, t, to)];
      const S d = thf - tht;
      const S cd = std::cos(d), sd = std::sin(d);
      const S Pfr = M.gff[l] * vf * vf + vf * vt * (M.gft[l] * cd + M.bft[l] * sd);
      const S Qfr = -M.bff[l] * vf * vf + vf * vt * (M.gft[l] * sd - M.bft[l] * cd);
      const S Pto = M.gtt[l] * vt * vt + vf * vt * (M.gtf[l] * cd - M.btf[l] * sd);
      const S Qto = -M.btt[l] * vt * vt + vf * vt * (-M.gtf[l] * sd - M.btf[l] * cd);
      const S pf = x[v_p(M, t, l)], qf = x[v_q(M, t, l)], pt = x[v_p(M, t, M.L + l)], qt = x[v_q(M, t, M.L + l)];
      c[r_br(M, 1, t, l)] = pf - Pfr;
      c[r_br(M, 2, t, l)] = qf - Qfr;
      c[r_br(M, 3, t, l)] = pt - Pto;
      c[r_br(M, 4, t, l)] = qt - Qto;
      c[r_br(M, 5, t, l)] = thf - tht;
      c[r_br(M, 6, t, l)] = pf * pf + qf * qf - M.smax[l] * M.smax[l];
      c[r_br(M, 7, t, l)] = pt * pt + qt * qt - M.smax[l] * M.smax[l];
    }
    for (int64_t n = 0; n < M.N; ++n) {
      S P = 0.0, Q = 0.0;
      for (int64_t g : M.bus_gens[n]) { P += x[v_pg(M, t, g)]; Q += x[v_qg(M, t, g)]; }
      for (int64_t a : M.bus_arcs[n]) { P -= x[v_p(M, t, a)]; Q -= x[v_q(M, t, a)]; }
      const S vm = x[v_vm(M, t, n)];
      P -= M.gs[n] * vm * vm;
      Q += M.bs[n] * vm * vm;
      for (int64_t d : M.bus_loads[n]) { P -= M.pd[t * M.D + d]; Q -= M.qd[t * M.D + d]; }
      c[r_k8(M, t, n)] = P;
      c[r_k9(M, t, n)] = Q;
    }
    if (t >= 1)
      for (int64_t g = 0; g < M.G; ++g) c[r_k10(M, t, g)] = x[v_pg(M, t, g)] - x[v_pg(M, t - 1, g)];
    if (t >= 1 && M.has_qramp)
      for (int64_t g = 0; g < M.G; ++g) c[r_k11(M, t, g)] = x[v_qg(M, t, g)] - x[v_qg(M, t - 1, g)];
  }
}
}  // namespace

extern "C" {
void orc_cons_textbook(void* h, const double* x, double* c) {
  const Model& M = *static_cast<Model*>(h);
  cons_textbook<double>(M, x, c);
}

// Directional derivative of the textbook c(x) by complex step: Im c(x + i h dx) / h.
void orc_cons_cstep(void* h, const double* x, const double* dx, double hstep, double* dc) {
  const Model& M = *static_cast<Model*>(h);
  std::vector<cplx> xc(M.n), cc(M.m);
  for (int64_t j = 0; j < M.n; ++j) xc[j] = cplx(x[j], hstep * dx[j]);
  cons_textbook<cplx>(M, xc.data(), cc.data());
  for (int64_t i = 0; i < M.m; ++i) dc[i] = cc[i].imag() / hstep;
}

// Textbook objective sum_{t,g} c2 pg^2 + c1 pg + c0 (plain expression).
double orc_obj_textbook(void* h, const double* x) {
  const Model& M = *static_cast<Model*>(h);
  double acc = 0.0;
  for (int64_t t = 0; t < M.T; ++t)
    for (int64_t g = 0; g < M.G; ++g) {
      const double pg = x[v_pg(M, t, g)];
      acc += M.c2[g] * pg * pg + M.c1[g] * pg + M.c0[g];
    }
  return acc;
}

// pi-model terms (for closed-form pins): out[8][L] = gff, bff, gft, bft, gtf, btf, gtt, btt.
void orc_branch_terms(void* h, double* out) {
  const Model& M = *static_cast<Model*>(h);
  for (int64_t l = 0; l < M.L; ++l) {
    out[0 * M.L + l] = M.gff[l]; out[1 * M.L + l] = M.bff[l]; out[2 * M.L + l] = M.gft[l]; out[3 * M.L + l] = M.bft[l];
    out[4 * M.L + l] = M.gtf[l]; out[5 * M.L + l] = M.btf[l]; out[6 * M.L + l] = M.gtt[l]; out[7 * M.L + l] = M.btt[l];
  }
}
}  // extern "C"
