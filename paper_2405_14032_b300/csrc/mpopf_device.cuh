// Device helpers shared by the evaluation and adjoint kernels of libmpopf:
// the fixed-rounding-order sin/cos, integer sign flip and doubling, and the
// branch flow terms with their first and second derivatives.
#pragma once
#include "mpopf_internal.cuh"

namespace mpopf {

// ---------------------------------------------------------------------------
// sin and cos of the angle difference: Cody & Waite reduction by pi/2 in three
// parts (Software Manual for the Elementary Functions, 1980), then, with
// s = r^2, sin r = r + r^3 P(s) and cos r = 1 + s Q(s), Horner in s.  P (degree
// 5) and Q (degree 6) are the Taylor series of (sin r - r)/r^3 through s^7 and
// of (cos r - 1)/r^2 through s^8, economised by Chebyshev polynomials
// (Lanczos's telescoping: each top term c_n s^n traded for the lower terms of
// c_n T*_n(s) / lead(T*_n), T*_n(s) = T_n(16 s / 5 - 1) on [0, 5/8], which
// covers |r| <= pi/4) in exact rational arithmetic, then rounded to nearest:
// 15 FP64 instructions for both values (19 for the plain Taylor series through
// r^17 and r^18), the polynomials within 2e-17 of sin and 1e-18 of cos.
// |x| <= RN(pi/4) needs no reduction.  Outside |x| < 2^30 (and for NaN/Inf) the
// CUDA library is used.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sincos_cw(double x, double *sn, double *cs) {
  const unsigned long long ax = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
  if (ax >= 0x41D0000000000000ULL) {  // |x| >= 2^30, Inf, NaN
    sincos(x, sn, cs);
    return;
  }
  double r = x;
  int q = 0;
  if (ax > 0x3FE921FB54442D18ULL) {  // |x| > RN(pi/4)
    const double k = rint(x * 0x1.45f306dc9c883p-1);
    r = fma(-k, 0x1.921fb54442d18p+0, x);
    r = fma(-k, 0x1.1a62633145c07p-54, r);
    r = fma(-k, -0x1.f1976b7ed8fbcp-110, r);
    q = (int)(__double2ll_rz(k) & 3);
  }
  const double r2 = r * r;
  double p = 0x1.5e00b6cff8290p-33;
  p = fma(p, r2, -0x1.ae5fedfda2660p-26);
  p = fma(p, r2, 0x1.71de377a84b02p-19);
  p = fma(p, r2, -0x1.a01a019e6dedep-13);
  p = fma(p, r2, 0x1.1111111110b56p-7);
  p = fma(p, r2, -0x1.5555555555555p-3);
  const double r3 = r2 * r;
  const double s = fma(r3, p, r);
  double c = -0x1.8fedb35736fa4p-37;
  c = fma(c, r2, 0x1.1eea6a6fdd11ap-29);
  c = fma(c, r2, -0x1.27e4f8ca561dfp-22);
  c = fma(c, r2, 0x1.a01a019dc2b7ep-16);
  c = fma(c, r2, -0x1.6c16c16c15c7dp-10);
  c = fma(c, r2, 0x1.5555555555550p-5);
  c = fma(c, r2, -0x1.0000000000000p-1);
  const double co = fma(r2, c, 1.0);
  if (q == 0) { *sn = s; *cs = co; }
  else if (q == 1) { *sn = co; *cs = -s; }
  else if (q == 2) { *sn = -s; *cs = -co; }
  else { *sn = -co; *cs = s; }
}

// -x by flipping the sign bit with an integer operation (exact; keeps the
// scarce FP64 pipe free).
__device__ __forceinline__ double negx(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// 2x exactly with integer operations only (no branch, no FP64 instruction):
// exponent + 1 for normal results, a one-bit left shift of the magnitude for
// zero and subnormal inputs, infinity on overflow, Inf and NaN unchanged.
__device__ __forceinline__ double twice(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
  const int sign = hi & (int)0x80000000;
  int rh = hi + 0x100000, rl = lo;
  const int sub_h = sign | ((hi & 0x7fffffff) << 1) | (int)((unsigned)lo >> 31);
  rh = (e == 0u) ? sub_h : rh;
  rl = (e == 0u) ? (int)((unsigned)lo << 1) : rl;
  rh = (e == 2046u) ? (sign | 0x7ff00000) : rh;
  rl = (e == 2046u) ? 0 : rl;
  rh = (e == 2047u) ? hi : rh;
  rl = (e == 2047u) ? lo : rl;
  return __hiloint2double(rh, rl);
}

// Flow terms of branch l at one period (pi-model, Eq. 1d/1e read as the full
// four-flow form): A1 = gft C + bft S, A2 = gft S - bft C, A3 = gtf C - btf S,
// A4 = -gtf S - btf C with C, S = cos, sin(va_f - va_t); vtA1 = vt A1, ...;
// uA1 = vf (vt A1), uA2 = vf (vt A2), uA3 = vt (vf A3), uA4 = vt (vf A4).
struct Flow {
  double dth, A1, A2, A3, A4, vtA1, vtA2, vfA3, vfA4, uA1, uA2, uA3, uA4;
};

__device__ __forceinline__ Flow flow_terms(const Dev &d, int32_t l, double thf, double tht, double vf, double vt) {
  const int64_t L = d.L;
  const double *bc = d.bc;
  const double gft = __ldg(bc + (int64_t)BC_GFT * L + l), bft = __ldg(bc + (int64_t)BC_BFT * L + l);
  const double gtf = __ldg(bc + (int64_t)BC_GTF * L + l), btf = __ldg(bc + (int64_t)BC_BTF * L + l);
  Flow F;
  F.dth = thf - tht;
  double sn, cs;
  sincos_cw(F.dth, &sn, &cs);
  const double bS = bft * sn, bC = bft * cs;
  F.A1 = fma(gft, cs, bS);
  F.A2 = fma(gft, sn, -bC);
  if (__ldg(d.br_sym + l)) {  // btf == bft: the products are the same
    F.A3 = fma(gtf, cs, -bS);
    F.A4 = fma(-gtf, sn, -bC);
  } else {
    F.A3 = fma(gtf, cs, -(btf * sn));
    F.A4 = fma(-gtf, sn, -(btf * cs));
  }
  F.vtA1 = vt * F.A1;
  F.vtA2 = vt * F.A2;
  F.vfA3 = vf * F.A3;
  F.vfA4 = vf * F.A4;
  F.uA1 = vf * F.vtA1;
  F.uA2 = vf * F.vtA2;
  F.uA3 = vt * F.vfA3;
  F.uA4 = vt * F.vfA4;
  return F;
}

// J entries of the four flow rows over (va_f, va_t, vm_f, vm_t): [a, -a, b, c]
// (the arc variable's entry is 1).  -fma(a, b, c) == fma(-a, b, -c) and
// -(a b) == (-a) b exactly.
struct FlowJ {
  double a1, b1, c1, a2, b2, c2, a3, b3, c3, a4, b4, c4;
};

__device__ __forceinline__ FlowJ flow_jac(const Dev &d, int32_t l, const Flow &F, double vf, double vt) {
  const int64_t L = d.L;
  const double *bc = d.bc;
  const double g2ff = __ldg(bc + (int64_t)BC_G2FF * L + l), b2ff = __ldg(bc + (int64_t)BC_B2FF * L + l);
  const double g2tt = __ldg(bc + (int64_t)BC_G2TT * L + l), b2tt = __ldg(bc + (int64_t)BC_B2TT * L + l);
  FlowJ J;
  J.a1 = F.uA2; J.b1 = fma(-g2ff, vf, -F.vtA1); J.c1 = (-vf) * F.A1;
  J.a2 = negx(F.uA1); J.b2 = fma(b2ff, vf, -F.vtA2); J.c2 = (-vf) * F.A2;
  J.a3 = negx(F.uA4); J.b3 = (-vt) * F.A3; J.c3 = fma(-g2tt, vt, -F.vfA3);
  J.a4 = F.uA3; J.b4 = (-vt) * F.A4; J.c4 = fma(b2tt, vt, -F.vfA4);
  return J;
}

// W block of a branch (sum over the four flow rows, c_k = arc_k - E_k):
// Asum = sum lambda_k A_k, Bsum = l1 A2 - l2 A1 - l3 A4 + l4 A3 (fixed order),
// W_dd = vf (vt Asum), W_dvf = vt Bsum, W_dvt = vf Bsum,
// W_vfvf = l2 2bff - l1 2gff, W_vtvt = l4 2btt - l3 2gtt, W_vfvt = -Asum.
struct FlowW {
  double Asum, Wdd, Wdvf, Wdvt, Wvfvf, Wvtvt;
};

__device__ __forceinline__ FlowW flow_hess(const Dev &d, int32_t l, const Flow &F, double vf, double vt, double l1,
                                           double l2, double l3, double l4) {
  const int64_t L = d.L;
  const double *bc = d.bc;
  const double g2ff = __ldg(bc + (int64_t)BC_G2FF * L + l), b2ff = __ldg(bc + (int64_t)BC_B2FF * L + l);
  const double g2tt = __ldg(bc + (int64_t)BC_G2TT * L + l), b2tt = __ldg(bc + (int64_t)BC_B2TT * L + l);
  FlowW W;
  W.Asum = fma(l4, F.A4, fma(l3, F.A3, fma(l2, F.A2, l1 * F.A1)));
  const double Bsum = fma(l4, F.A3, fma(-l3, F.A4, fma(-l2, F.A1, l1 * F.A2)));
  W.Wdd = vf * (vt * W.Asum);
  W.Wdvf = vt * Bsum;
  W.Wdvt = vf * Bsum;
  W.Wvfvf = fma(l2, b2ff, -(l1 * g2ff));
  W.Wvtvt = fma(l4, b2tt, -(l3 * g2tt));
  return W;
}

}  // namespace mpopf
