// Evaluation kernels of libmpopf (sm_103a, FP64).
//
// One thread per component x period instance (the SIMD abstraction of Eq. 2):
//   k_branch  (t, l): flows, rows K1..K7, their J entries, the branch block of W,
//                     the thermal W entries, the four M rows of the branch's
//                     arcs, and the six distinct values of the branch element's
//                     bus-variable block of M (to the scratch buffer S);
//   k_bus     (t, n): balance rows K8/K9, the reference row, shunt W entries,
//                     and the va/vm rows of M, summing the incident branches'
//                     values from S in a fixed order (no atomics);
//   k_gen     (t, g): objective terms, gradient, objective W entry, ramp rows
//                     and the pg/qg rows of M;
//   k_fsum           : the objective's fixed-order tree reduction;
//   k_batch          : all of the above for many instances, one persistent launch.
// An evaluation runs k_branch and k_bus on the caller's stream and k_gen with
// k_fsum on the handle's side stream (forked after k_branch, joined at the end).
// Every value follows one fixed sequence of binary64 operations (explicit fma
// where the definition has one; the build disables contraction), so results
// are bitwise reproducible from run to run.
#include <algorithm>
#include <cstring>

#include "mpopf_device.cuh"

namespace mpopf {
namespace {

template <unsigned MASK>
__device__ __forceinline__ unsigned eff(unsigned rt) { return MASK ? MASK : rt; }

// Branch kernel launch shape: threads per CTA and resident CTAs per SM (the
// register cap, 80, follows from them).  At that cap, 64-thread CTAs (12 per
// SM) measured 0.830 ms at 10k buses x 168 against 0.831 ms for 96 x 8,
// 0.833 ms for 128 x 6, 0.839 ms for 192 x 4, 0.857 ms for 256 x 3, 1.051 ms
// for 384 x 2 and 0.863 ms for 32 x 24; small instances gain most (10k buses
// x 1: 33.5 -> 27.3 us per sweep).
#ifndef MPOPF_BRANCH_MINB
#define MPOPF_BRANCH_MINB 12
#endif
#ifndef MPOPF_BRANCH_BLOCK
#define MPOPF_BRANCH_BLOCK 64
#endif
// Bus kernel CTA size (48 registers, so 1280 resident threads per SM whatever
// the size): 128 measured 0.258 ms against 0.261 ms for 256 at 10k buses x 168,
// and 26.3 against 27.3 us per sweep at 10k buses x 1.
#ifndef MPOPF_BUS_BLOCK
#define MPOPF_BUS_BLOCK 128
#endif
// Loads of values another CTA wrote in the same launch go through L2 (the
// persistent batch kernel); separate launches may use the read-only path.
template <bool COH>
__device__ __forceinline__ double2 ld_rec(const double *p) {
  return COH ? __ldcg(reinterpret_cast<const double2 *>(p)) : __ldg(reinterpret_cast<const double2 *>(p));
}
template <bool COH>
__device__ __forceinline__ double ld_part(const double *p) {
  return COH ? __ldcg(p) : *p;
}

// Waits (griddepcontrol.wait) until the grids this launch depends on
// programmatically have completed and their writes are visible; returns at
// once for a launch without such a dependency.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Records a CUDA event pair around one launch when profiling is on.
struct Timed {
  Prof *p;
  cudaStream_t s;
  int slot;
  Timed(Prof *prof, cudaStream_t st, int kind) : p(prof), s(st), slot(-1) {
    if (p && p->next < p->cap) {
      slot = p->next++;
      p->kind[slot] = kind;
      cudaEventRecord(p->ev[2 * slot], s);
    }
  }
  ~Timed() {
    if (slot >= 0) cudaEventRecord(p->ev[2 * slot + 1], s);
  }
};

// Output staging of one warp (k_branch, k_batch).  The J rows of the four
// flow constraints and the W blocks of 32 consecutive branch elements are
// contiguous ranges of the outputs, but each lane writes its own short piece
// of them (5 or 10 entries): one L2 request per lane and store.  Staged, the
// lanes write their pieces to a per-warp buffer in shared memory (in output
// order) and the range goes out whole: in k_branch as coalesced warp stores
// (one request per 128-byte line); in the persistent batch kernel as one
// bulk copy (cp.async.bulk, shared to global, issued by one lane) when the
// destination is 16-byte aligned, which measured faster there and slower in
// k_branch.
// Without the bulk copy, one pad word per 32 spreads the lanes' pieces over
// the shared-memory banks; the bulk copy needs the range unpadded.
constexpr int kStageCap = 320;                            // doubles per warp
constexpr int kStagePitch = kStageCap + kStageCap / 32;  // with the pad words
template <bool BULK>
__device__ __forceinline__ int spad(int p) { return BULK ? p : p + (p >> 5); }
template <bool BULK>
__device__ __forceinline__ void warp_flush(double *__restrict__ g, double *s, int n, int lane) {
  if (BULK && (reinterpret_cast<uintptr_t>(g) & 15) == 0) {  // uniform over the warp
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the lanes' writes, to the copy engine
    __syncwarp();
    if (lane == 0) {
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                   :: "l"(g), "r"((unsigned)__cvta_generic_to_shared(s)), "r"(n * 8) : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // buffer free again
    }
    __syncwarp();
    return;
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) g[i] = s[spad<BULK>(i)];
  __syncwarp();
}
// Lane 0's bulk copies have completed their writes (before the warp exits).
__device__ __forceinline__ void bulk_done(int lane) {
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// SYM: every branch of the model is symmetric (the per-branch test is known).
// PTS: the element belongs to point blockIdx.y of a sweep over several points,
// whose incidence records follow the earlier points' (T periods each).
// BW: the bus-end products D8 (m2gs vm) and D9 (p2bs vm) come from d.bw,
// formed by k_bw with the same operations (the element waits for that grid
// before its first read of them).
template <unsigned MASK, bool BULK = false, bool SYM = false, bool PTS = false, bool BW = false>
__device__ __forceinline__ void branch_body(const Dev &d, int32_t tl, unsigned rt, const double *__restrict__ x,
                                            const double *__restrict__ lam, const double *__restrict__ sx,
                                            const double *__restrict__ dv, double dw, double *__restrict__ grad,
                                            double *__restrict__ c, double *__restrict__ jv,
                                            double *__restrict__ hv, double *__restrict__ kv,
                                            double *stage = nullptr) {
  // stage: the warp's staging buffer when all 32 lanes hold elements, else null
  const unsigned mk = eff<MASK>(rt);
  const int lane = (int)(threadIdx.x & 31);
  const int32_t L = d.L;
  if (tl >= d.T * L) return;
  const int32_t t = tl / L, l = tl - t * L;
  const int64_t TL = (int64_t)d.T * L;
  const int64_t tN = (int64_t)t * d.N;
  const int64_t pb = d.x_p + 2 * (int64_t)t * L, qb = d.x_q + 2 * (int64_t)t * L;
  if (mk & MPOPF_OUT_GRAD) {
    grad[pb + l] = 0.0;
    grad[pb + L + l] = 0.0;
    grad[qb + l] = 0.0;
    grad[qb + L + l] = 0.0;
  }
  if (!(mk & (MPOPF_OUT_CONS | MPOPF_OUT_JAC | MPOPF_OUT_HESS | MPOPF_OUT_KKT))) return;

  // per-branch integers in 16-byte loads (quads, structure of arrays)
  const int4 ends = __ldg(d.brp + (int64_t)BRP_ENDS * L + l);
  const int32_t f = ends.x, to = ends.y;
  const double thf = __ldg(x + tN + f), tht = __ldg(x + tN + to);
  const double vf = __ldg(x + d.x_vm + tN + f), vt = __ldg(x + d.x_vm + tN + to);
  const double *bc = d.bc;
  const double gft = __ldg(bc + (int64_t)BC_GFT * L + l), bft = __ldg(bc + (int64_t)BC_BFT * L + l);
  const double gtf = __ldg(bc + (int64_t)BC_GTF * L + l), btf = __ldg(bc + (int64_t)BC_BTF * L + l);

  // Flow terms.
  const double dth = thf - tht;
  double sn, cs;
  sincos_cw(dth, &sn, &cs);
  const double bS = bft * sn, bC = bft * cs;
  const double A1 = fma(gft, cs, bS);
  const double A2 = fma(gft, sn, -bC);
  double A3, A4;
  if (SYM || __ldg(d.br_sym + l)) {  // btf == bft: the products are the same
    A3 = fma(gtf, cs, -bS);
    A4 = fma(-gtf, sn, -bC);
  } else {
    A3 = fma(gtf, cs, -(btf * sn));
    A4 = fma(-gtf, sn, -(btf * cs));
  }
  const double vtA1 = vt * A1, vtA2 = vt * A2, vfA3 = vf * A3, vfA4 = vf * A4;
  const double uA1 = vf * vtA1, uA2 = vf * vtA2, uA3 = vt * vfA3, uA4 = vt * vfA4;

  const double pf = __ldg(x + pb + l), pt = __ldg(x + pb + L + l);
  const double qf = __ldg(x + qb + l), qt = __ldg(x + qb + L + l);
  const int64_t rk1 = d.T + tl;  // row of K1; K_k at rk1 + (k-1) T L

  if (mk & MPOPF_OUT_CONS) {
    const double gff = __ldg(bc + (int64_t)BC_GFF * L + l), bff = __ldg(bc + (int64_t)BC_BFF * L + l);
    const double gtt = __ldg(bc + (int64_t)BC_GTT * L + l), btt = __ldg(bc + (int64_t)BC_BTT * L + l);
    const double smax2 = __ldg(bc + (int64_t)BC_SMAX2 * L + l);
    const double vf2 = vf * vf, vt2 = vt * vt;
    c[rk1] = pf - fma(gff, vf2, uA1);
    c[rk1 + TL] = qf - fma(-bff, vf2, uA2);
    c[rk1 + 2 * TL] = pt - fma(gtt, vt2, uA3);
    c[rk1 + 3 * TL] = qt - fma(-btt, vt2, uA4);
    c[rk1 + 4 * TL] = dth;
    c[rk1 + 5 * TL] = fma(pf, pf, fma(qf, qf, -smax2));
    c[rk1 + 6 * TL] = fma(pt, pt, fma(qt, qt, -smax2));
  }
  if (!(mk & (MPOPF_OUT_JAC | MPOPF_OUT_HESS | MPOPF_OUT_KKT))) return;

  const double g2ff = __ldg(bc + (int64_t)BC_G2FF * L + l), b2ff = __ldg(bc + (int64_t)BC_B2FF * L + l);
  const double g2tt = __ldg(bc + (int64_t)BC_G2TT * L + l), b2tt = __ldg(bc + (int64_t)BC_B2TT * L + l);
  // J entries of the flow rows over (va_f, va_t, vm_f, vm_t): [a, -a, b, c].
  // (-fma(a, b, c) == fma(-a, b, -c) and -(a b) == (-a) b exactly.)
  const double a1 = uA2, na1 = negx(uA2), b1 = fma(-g2ff, vf, -vtA1), c1 = (-vf) * A1;
  const double a2 = negx(uA1), na2 = uA1, b2 = fma(b2ff, vf, -vtA2), c2 = (-vf) * A2;
  const double a3 = negx(uA4), na3 = uA4, b3 = (-vt) * A3, c3 = fma(-g2tt, vt, -vfA3);
  const double a4 = uA3, na4 = negx(uA3), b4 = (-vt) * A4, c4 = fma(b2tt, vt, -vfA4);
  const double jp6 = twice(pf), jq6 = twice(qf), jp7 = twice(pt), jq7 = twice(qt);

  if (mk & MPOPF_OUT_JAC) {
    const int64_t s5 = 5 * TL;
    if (stage) {
      double *g = jv + d.T + (int64_t)(tl - lane) * 5;
      auto put5 = [&](double *gk, double v1, double v2, double v3, double v4) {
        stage[spad<BULK>(5 * lane)] = 1.0; stage[spad<BULK>(5 * lane + 1)] = v1;
        stage[spad<BULK>(5 * lane + 2)] = v2; stage[spad<BULK>(5 * lane + 3)] = v3;
        stage[spad<BULK>(5 * lane + 4)] = v4;
        warp_flush<BULK>(gk, stage, 160, lane);
      };
      put5(g, a1, na1, b1, c1);
      put5(g + s5, a2, na2, b2, c2);
      put5(g + 2 * s5, a3, na3, b3, c3);
      put5(g + 3 * s5, a4, na4, b4, c4);
    } else {
      double *j1 = jv + d.T + (int64_t)tl * 5;
      j1[0] = 1.0; j1[1] = a1; j1[2] = na1; j1[3] = b1; j1[4] = c1;
      j1[s5 + 0] = 1.0; j1[s5 + 1] = a2; j1[s5 + 2] = na2; j1[s5 + 3] = b2; j1[s5 + 4] = c2;
      j1[2 * s5 + 0] = 1.0; j1[2 * s5 + 1] = a3; j1[2 * s5 + 2] = na3; j1[2 * s5 + 3] = b3; j1[2 * s5 + 4] = c3;
      j1[3 * s5 + 0] = 1.0; j1[3 * s5 + 1] = a4; j1[3 * s5 + 2] = na4; j1[3 * s5 + 3] = b4; j1[3 * s5 + 4] = c4;
    }
    double *j5 = jv + d.j_k5 + (int64_t)tl * 2;
    j5[0] = 1.0; j5[1] = -1.0;
    double *j6 = jv + d.j_k6 + (int64_t)tl * 2;
    j6[0] = jp6; j6[1] = jq6;
    double *j7 = jv + d.j_k7 + (int64_t)tl * 2;
    j7[0] = jp7; j7[1] = jq7;
  }
  if (!(mk & (MPOPF_OUT_HESS | MPOPF_OUT_KKT))) return;

  // W: branch block (sum over the four flow rows) and thermal entries.
  const double l1 = __ldg(lam + rk1), l2 = __ldg(lam + rk1 + TL), l3 = __ldg(lam + rk1 + 2 * TL);
  const double l4 = __ldg(lam + rk1 + 3 * TL), l6 = __ldg(lam + rk1 + 5 * TL), l7 = __ldg(lam + rk1 + 6 * TL);
  const double Asum = fma(l4, A4, fma(l3, A3, fma(l2, A2, l1 * A1)));
  const double Bsum = fma(l4, A3, fma(-l3, A4, fma(-l2, A1, l1 * A2)));
  const double Wdd = vf * (vt * Asum);
  const double Wdvf = vt * Bsum, Wdvt = vf * Bsum;
  const double Wvfvf = fma(l2, b2ff, -(l1 * g2ff));
  const double Wvtvt = fma(l4, b2tt, -(l3 * g2tt));
  const double h6 = twice(l6), h7 = twice(l7);
  const double nAsum = negx(Asum);
  if (mk & MPOPF_OUT_HESS) {
    if (stage) {
      const int b = 10 * lane;
      stage[spad<BULK>(b)] = Wdd; stage[spad<BULK>(b + 1)] = negx(Wdd); stage[spad<BULK>(b + 2)] = Wdd;
      stage[spad<BULK>(b + 3)] = Wdvf; stage[spad<BULK>(b + 4)] = negx(Wdvf); stage[spad<BULK>(b + 5)] = Wvfvf;
      stage[spad<BULK>(b + 6)] = Wdvt; stage[spad<BULK>(b + 7)] = negx(Wdvt); stage[spad<BULK>(b + 8)] = nAsum;
      stage[spad<BULK>(b + 9)] = Wvtvt;
      warp_flush<BULK>(hv + d.h_br + (int64_t)(tl - lane) * 10, stage, 320, lane);
      const int e = 4 * lane;
      stage[spad<BULK>(e)] = h6; stage[spad<BULK>(e + 1)] = h6; stage[spad<BULK>(e + 2)] = h7;
      stage[spad<BULK>(e + 3)] = h7;
      warp_flush<BULK>(hv + d.h_th + (int64_t)(tl - lane) * 4, stage, 128, lane);
    } else {
      double *hb = hv + d.h_br + (int64_t)tl * 10;
      hb[0] = Wdd; hb[1] = negx(Wdd); hb[2] = Wdd; hb[3] = Wdvf; hb[4] = negx(Wdvf);
      hb[5] = Wvfvf; hb[6] = Wdvt; hb[7] = negx(Wdvt); hb[8] = nAsum; hb[9] = Wvtvt;
      double *ht = hv + d.h_th + (int64_t)tl * 4;
      ht[0] = h6; ht[1] = h6; ht[2] = h7; ht[3] = h7;
    }
  }
  if (!(mk & MPOPF_OUT_KKT)) return;

  // Condensed matrix: the branch element's local block.
  const double D1 = __ldg(dv + rk1), D2 = __ldg(dv + rk1 + TL), D3 = __ldg(dv + rk1 + 2 * TL);
  const double D4 = __ldg(dv + rk1 + 3 * TL), D5 = __ldg(dv + rk1 + 4 * TL), D6 = __ldg(dv + rk1 + 5 * TL);
  const double D7 = __ldg(dv + rk1 + 6 * TL);
  const double w11 = D1 * a1, w31 = D1 * b1, w41 = D1 * c1;
  const double w12 = D2 * a2, w32 = D2 * b2, w42 = D2 * c2;
  const double w13 = D3 * a3, w33 = D3 * b3, w43 = D3 * c3;
  const double w14 = D4 * a4, w34 = D4 * b4, w44 = D4 * c4;
  double Sdd = fma(w14, a4, fma(w13, a3, fma(w12, a2, fma(w11, a1, Wdd))));
  Sdd = Sdd + D5;
  const double Svfd = fma(w34, a4, fma(w33, a3, fma(w32, a2, fma(w31, a1, Wdvf))));
  const double Svtd = fma(w44, a4, fma(w43, a3, fma(w42, a2, fma(w41, a1, Wdvt))));
  const double Svfvf = fma(w34, b4, fma(w33, b3, fma(w32, b2, fma(w31, b1, Wvfvf))));
  const double Svtvf = fma(w44, b4, fma(w43, b3, fma(w42, b2, fma(w41, b1, nAsum))));
  const double Svtvt = fma(w44, c4, fma(w43, c3, fma(w42, c2, fma(w41, c1, Wvtvt))));
  {
    // incidence records of both ends (bus-major, read by k_bus)
    double *R = d.S + (int64_t)t * 2 * L * kRec;
    if (PTS) R += (int64_t)blockIdx.y * d.T * 2 * L * kRec;
    double2 *recf = reinterpret_cast<double2 *>(R + (int64_t)ends.z * kRec);
    recf[0] = make_double2(Sdd, Svfd);
    recf[1] = make_double2(Svfvf, Svtvf);
    recf[2] = make_double2(pf, qf);
    double2 *rect = reinterpret_cast<double2 *>(R + (int64_t)ends.w * kRec);
    rect[0] = make_double2(Sdd, negx(Svtd));
    rect[1] = make_double2(Svtvt, Svtvf);
    rect[2] = make_double2(pt, qt);
  }
  // Arc-variable diagonals and the (q, p) pair of each end.
  const double t6p = D6 * jp6, t6q = D6 * jq6, t7p = D7 * jp7, t7q = D7 * jq7;
  const double Lpp_f = fma(t6p, jp6, h6 + D1);
  const double Lqq_f = fma(t6q, jq6, h6 + D2);
  const double Lqp_f = t6q * jp6;
  const double Lpp_t = fma(t7p, jp7, h7 + D3);
  const double Lqq_t = fma(t7q, jq7, h7 + D4);
  const double Lqp_t = t7q * jp7;
  // Bus elements at both ends: their (arc, vm) and (arc, arc) entries.
  const int64_t r8f = d.c_k8 + tN + f, r8t = d.c_k8 + tN + to;
  const double D8f = __ldg(dv + r8f), D9f = __ldg(dv + r8f + (d.c_k9 - d.c_k8));
  const double D8t = __ldg(dv + r8t), D9t = __ldg(dv + r8t + (d.c_k9 - d.c_k8));
  double w8f, w9f, w8t, w9t;
  if (BW) {
    grid_dependency_wait();
    const int64_t TN = (int64_t)d.T * d.N;
    const double *bw = d.bw;
    if (PTS) bw += (int64_t)blockIdx.y * 2 * TN;
    w8f = __ldcg(bw + tN + f);
    w9f = __ldcg(bw + TN + tN + f);
    w8t = __ldcg(bw + tN + to);
    w9t = __ldcg(bw + TN + tN + to);
  } else {
    w8f = D8f * (__ldg(d.bus_m2gs + f) * vf);
    w9f = D9f * (__ldg(d.bus_p2bs + f) * vf);
    w8t = D8t * (__ldg(d.bus_m2gs + to) * vt);
    w9t = D9t * (__ldg(d.bus_p2bs + to) * vt);
  }
  const double sxpf = __ldg(sx + pb + l), sxpt = __ldg(sx + pb + L + l);
  const double sxqf = __ldg(sx + qb + l), sxqt = __ldg(sx + qb + L + l);
  const bool flo = f < to;
  const int4 rank = __ldg(d.brp + (int64_t)BRP_RANK * L + l);
  const int32_t rf = rank.x, rt2 = rank.y, kf = rank.z, kt = rank.w;
  // Writes one arc row at kv[start ..]: [va lo, va hi, vm lo, vm hi], ngen x gval, [qp], nrank x aval, diag.
  // The rows of 32 consecutive arcs of one kind and period are consecutive
  // rows of M (contiguous in kv); a warp whose rows are contiguous and fit the
  // buffer stages them, any other writes them directly.
  // Writes one arc row at kv[start ..]: [va lo, va hi, vm lo, vm hi], ngen x gval, [qp], nrank x aval, diag.
  auto arc_row = [&](int64_t start, double vaf, double vat, double vmf, double vmt, int32_t ngen, double gval,
                     bool has_qp, double qp, int32_t nrank, double aval, double diag) {
    kv[start] = flo ? vaf : vat;
    kv[start + 1] = flo ? vat : vaf;
    kv[start + 2] = flo ? vmf : vmt;
    kv[start + 3] = flo ? vmt : vmf;
    int k = 4;
    for (int32_t e = 0; e < ngen; ++e) kv[start + k++] = gval;
    if (has_qp) kv[start + k++] = qp;
    for (int32_t e = 0; e < nrank; ++e) kv[start + k++] = aval;
    kv[start + k] = diag;
  };
  const int64_t mp = d.m_p + (int64_t)t * d.mb_p, mq = d.m_q + (int64_t)t * d.mb_q;
  const int4 mrow = __ldg(d.brp + (int64_t)BRP_MROW * L + l);
  arc_row(mp + mrow.x, w11, negx(w11), w31 - w8f, w41, kf, negx(D8f), false, 0.0, rf, D8f,
          ((sxpf + dw) + Lpp_f) + D8f);
  arc_row(mq + mrow.z, w12, negx(w12), w32 - w9f, w42, kf, negx(D9f), true, Lqp_f, rf, D9f,
          ((sxqf + dw) + Lqq_f) + D9f);
  arc_row(mp + mrow.y, w13, negx(w13), w33, w43 - w8t, kt, negx(D8t), false, 0.0, rt2, D8t,
          ((sxpt + dw) + Lpp_t) + D8t);
  arc_row(mq + mrow.w, w14, negx(w14), w34, w44 - w9t, kt, negx(D9t), true, Lqp_t, rt2, D9t,
          ((sxqt + dw) + Lqq_t) + D9t);
}

// Elements [first, end) of the branch x period range (t L + l).
// The point offsets of a sweep over several points: point j = blockIdx.y
// reads and writes the j-th of consecutive arrays of the single-point sizes.
#define MPOPF_POINT_OFFSETS(d)                                        \
  do {                                                                \
    const int64_t j_ = blockIdx.y;                                    \
    x += j_ * (d).n;                                                  \
    sx += j_ * (d).n;                                                 \
    dv += j_ * (d).m;                                                 \
    grad += j_ * (d).n;                                               \
    c += j_ * (d).m;                                                  \
    jv += j_ * (d).nnz_jac;                                           \
    hv += j_ * (d).nnz_hess;                                          \
    kv += j_ * (d).nnz_kkt;                                           \
  } while (0)

template <unsigned MASK, bool SYM, bool PTS = false, bool BW = false>
__global__ void __launch_bounds__(MPOPF_BRANCH_BLOCK, MPOPF_BRANCH_MINB)
    k_branch(Dev d, unsigned rt, const double *__restrict__ x, const double *__restrict__ lam,
             const double *__restrict__ sx, const double *__restrict__ dv, double dw, double *__restrict__ grad,
             double *__restrict__ c, double *__restrict__ jv, double *__restrict__ hv, double *__restrict__ kv,
             int32_t first, int32_t end) {
  // a bus launch behind this one (programmatic dependent launch) may be
  // scheduled once every CTA of this grid has started; it waits for this
  // grid's completion before it reads the records
  asm volatile("griddepcontrol.launch_dependents;");
  const int32_t tl = first + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (tl >= end) return;
  if (PTS) {
    MPOPF_POINT_OFFSETS(d);
    lam += (int64_t)blockIdx.y * d.m;
  }
  __shared__ __align__(16) double s_stage[MPOPF_BRANCH_BLOCK / 32][kStagePitch];
  const bool full = tl - (int32_t)(threadIdx.x & 31) + 31 < end;  // uniform over the warp
  branch_body<MASK, false, SYM, PTS, BW>(d, tl, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv,
                                         full ? s_stage[threadIdx.x >> 5] : nullptr);
}

// The branch kernel over elements [first, end) on stream s; the instantiation
// without the per-branch symmetry test when every branch is symmetric
// (measured 0.798 against 0.810 ms at 10k buses x 168; the same values).
// With PTS, `points` points (grid y).
template <unsigned MASK, bool PTS = false>
void launch_branch(const Dev &d, unsigned rt, const double *x, const double *lam, const double *sx,
                   const double *dv, double dw, double *grad, double *c, double *jv, double *hv, double *kv,
                   int32_t first, int32_t end, cudaStream_t s, unsigned points = 1) {
  const dim3 grid((unsigned)(((int64_t)end - first + MPOPF_BRANCH_BLOCK - 1) / MPOPF_BRANCH_BLOCK), PTS ? points : 1);
  if (d.all_sym)
    k_branch<MASK, true, PTS><<<grid, MPOPF_BRANCH_BLOCK, 0, s>>>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv,
                                                                   first, end);
  else
    k_branch<MASK, false, PTS><<<grid, MPOPF_BRANCH_BLOCK, 0, s>>>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv,
                                                                    first, end);
}

// The bus-end products of the arc rows of M, once per bus and period of
// [first, end) (t N + n): w8 = D8 (m2gs vm) and w9 = D9 (p2bs vm), the
// operations the branch kernel would otherwise do at each end of each
// branch.  A grid-stride loop over a grid of at most a few CTAs per SM, so
// that every CTA is resident at once and the branch kernel behind it (a
// programmatic dependent launch) starts at once.
// With PTS, point blockIdx.y of a sweep over several points (its x, D and
// products follow the earlier points').
template <bool PTS = false>
__global__ void __launch_bounds__(kBlock) k_bw(Dev d, const double *__restrict__ x, const double *__restrict__ dv,
                                               int32_t first, int32_t end) {
  asm volatile("griddepcontrol.launch_dependents;");
  const int64_t TN = (int64_t)d.T * d.N;
  if (PTS) {
    x += (int64_t)blockIdx.y * d.n;
    dv += (int64_t)blockIdx.y * d.m;
    d.bw += (int64_t)blockIdx.y * 2 * TN;
  }
  for (int32_t i = first + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); i < end;
       i += (int32_t)(gridDim.x * blockDim.x)) {
    const int32_t n = i % d.N;
    const double vm = __ldg(x + d.x_vm + i);
    d.bw[i] = __ldg(dv + d.c_k8 + i) * (__ldg(d.bus_m2gs + n) * vm);
    d.bw[TN + i] = __ldg(dv + d.c_k9 + i) * (__ldg(d.bus_p2bs + n) * vm);
  }
}

// The bus-end products, then the branch kernel reading them (a programmatic
// dependent launch when `pdl`), for a full sweep over elements [first, end).
template <unsigned MASK>
cudaError_t launch_branch_bw(const Dev &d, unsigned rt, const double *x, const double *lam, const double *sx,
                             const double *dv, double dw, double *grad, double *c, double *jv, double *hv,
                             double *kv, cudaStream_t s, bool pdl, Prof *prof, int32_t sms) {
  const int32_t bf = d.w0 * d.N, be = d.w1 * d.N;
  const unsigned g = (unsigned)std::min<int64_t>(((int64_t)be - bf + kBlock - 1) / kBlock, 4 * (int64_t)sms);
  k_bw<<<g, kBlock, 0, s>>>(d, x, dv, bf, be);
  Timed tm(prof, s, KIND_BRANCH);
  const int32_t first = d.w0 * d.L, end = d.w1 * d.L;
  const unsigned grid = (unsigned)(((int64_t)end - first + MPOPF_BRANCH_BLOCK - 1) / MPOPF_BRANCH_BLOCK);
  void (*kern)(Dev, unsigned, const double *, const double *, const double *, const double *, double, double *,
               double *, double *, double *, double *, int32_t, int32_t) =
      d.all_sym ? k_branch<MASK, true, false, true> : k_branch<MASK, false, false, true>;
  if (!pdl) {
    kern<<<grid, MPOPF_BRANCH_BLOCK, 0, s>>>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, first, end);
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(MPOPF_BRANCH_BLOCK);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, first, end);
}

// ---------------------------------------------------------------------------
// Bus x period.
// ---------------------------------------------------------------------------

// PART: 0 everything; 1 the balance rows, their J rows, the shunt W entries,
// the gradient zeros and the reference row; 2 the va / vm rows of M (the two
// halves of a split schedule, run side by side).
// PTS: as in branch_body.
template <unsigned MASK, bool COH, bool WAIT = false, int PART = 0, bool PTS = false>
__device__ __forceinline__ void bus_body(const Dev &d, int32_t idx, unsigned rt, const double *__restrict__ x,
                                         const double *__restrict__ lam, const double *__restrict__ sx,
                                         const double *__restrict__ dv, double dw, double *__restrict__ grad,
                                         double *__restrict__ c, double *__restrict__ jv, double *__restrict__ hv,
                                         double *__restrict__ kv) {
  const unsigned mk = eff<MASK>(rt);
  const int32_t N = d.N;
  if (idx >= d.T * N) return;
  const int32_t t = idx / N;
  const int32_t pos = idx - t * N;  // position in the processing order
  const int32_t n = __ldg(d.bus_order + pos);
  const int32_t tn = t * N + n;  // (period, bus) position of every per-bus array
  const int64_t tN = (int64_t)t * N;
  const int64_t L = d.L, G = d.G;
  if (PART != 2 && (mk & MPOPF_OUT_GRAD)) {
    grad[tn] = 0.0;
    grad[d.x_vm + tn] = 0.0;
  }
  if (PART != 2 && n == d.ref) {
    if (mk & MPOPF_OUT_CONS) c[t] = __ldg(x + tN + n);
    if (mk & MPOPF_OUT_JAC) jv[t] = 1.0;
  }
  if (!(mk & (MPOPF_OUT_CONS | MPOPF_OUT_JAC | MPOPF_OUT_HESS | MPOPF_OUT_KKT))) return;
  const double vm = __ldg(x + d.x_vm + tn);
  const int32_t g0 = __ldg(d.bgen_ptr + n), g1 = __ldg(d.bgen_ptr + n + 1);
  const int32_t s0 = __ldg(d.inc_ptr + pos), s1 = __ldg(d.inc_ptr + pos + 1);  // incidence slots
  const double m2gs = __ldg(d.bus_m2gs + n), p2bs = __ldg(d.bus_p2bs + n);
  // Incidence records of this bus (written by k_branch when M is assembled).
  const double *R = d.S + (int64_t)t * 2 * L * kRec;
  if (PTS) R += (int64_t)blockIdx.y * d.T * 2 * L * kRec;
  const bool have_rec = mk & MPOPF_OUT_KKT;
  // a bus launch that may start before the branch launch has finished waits
  // here, before its first read of the records
  if (WAIT && have_rec) grid_dependency_wait();
  if (PART != 2 && (mk & MPOPF_OUT_CONS)) {
    const double vm2 = vm * vm;
    double aP = 0.0, aQ = 0.0;
    const int64_t pgb = d.x_pg + (int64_t)t * G, qgb = d.x_qg + (int64_t)t * G;
    for (int32_t e = g0; e < g1; ++e) {
      const int32_t g = __ldg(d.bgen_idx + e);
      aP = aP + __ldg(x + pgb + g);
      aQ = aQ + __ldg(x + qgb + g);
    }
    // Arc flows in ascending arc index: from ends (branch order), then to ends.
    if (have_rec) {
      // unrolled so that the record loads of several arcs are in flight
      // together (measured: 0.264 -> 0.253 ms at 10k buses x 168; the adds
      // keep their order)
#pragma unroll 4
      for (int32_t e = s0; e < s1; ++e) {
        const int32_t q = __ldg(d.arc_perm + e);
        const double2 pq = ld_rec<COH>(R + (int64_t)q * kRec + 4);
        aP = aP - pq.x;
        aQ = aQ - pq.y;
      }
    } else {
      const int64_t pab = d.x_p + 2 * (int64_t)t * L, qab = d.x_q + 2 * (int64_t)t * L;
      for (int32_t e = __ldg(d.barc_ptr + n); e < __ldg(d.barc_ptr + n + 1); ++e) {
        const int32_t a = __ldg(d.barc_idx + e);
        aP = aP - __ldg(x + pab + a);
        aQ = aQ - __ldg(x + qab + a);
      }
    }
    aP = fma(__ldg(d.bus_mgs + n), vm2, aP);
    aQ = fma(__ldg(d.bus_bs + n), vm2, aQ);
    const int64_t ldb = (int64_t)t * d.D;
    for (int32_t e = __ldg(d.bload_ptr + n); e < __ldg(d.bload_ptr + n + 1); ++e) {
      const int32_t k = __ldg(d.bload_idx + e);
      aP = aP - __ldg(d.pd + ldb + k);
      aQ = aQ - __ldg(d.qd + ldb + k);
    }
    c[d.c_k8 + tn] = aP;
    c[d.c_k9 + tn] = aQ;
  }
  const double J8 = m2gs * vm, J9 = p2bs * vm;
  if (PART != 2 && (mk & MPOPF_OUT_JAC)) {
    double *r8 = jv + d.j_k8 + (int64_t)t * d.jk8_per + __ldg(d.jk8_off + n);
    double *r9 = r8 + (d.j_k9 - d.j_k8);
    r8[0] = J8;
    r9[0] = J9;
    int k = 1;
    for (int32_t e = g0; e < g1; ++e, ++k) { r8[k] = 1.0; r9[k] = 1.0; }
    for (int32_t e = s0; e < s1; ++e, ++k) { r8[k] = -1.0; r9[k] = -1.0; }
  }
  if (!(mk & (MPOPF_OUT_HESS | MPOPF_OUT_KKT))) return;
  const double WP = __ldg(lam + d.c_k8 + tn) * m2gs, WQ = __ldg(lam + d.c_k9 + tn) * p2bs;
  if (PART != 2 && (mk & MPOPF_OUT_HESS)) {
    hv[d.h_sh + 2 * (int64_t)tn] = WP;
    hv[d.h_sh + 2 * (int64_t)tn + 1] = WQ;
  }
  if (PART == 1 || !(mk & MPOPF_OUT_KKT)) return;

  const int32_t nd = __ldg(d.bus_nd + n), ndlt = __ldg(d.bus_ndlt + n);
  double *va_row = kv + d.m_va + (int64_t)t * d.mb_va + __ldg(d.mo_va + n);
  double *vm_row = kv + d.m_vm + (int64_t)t * d.mb_vm + __ldg(d.mo_vm + n);
  // One pass over the incidence records in branch order: diagonal sums
  // (diagonal term, reference element, branches, then the bus element) and,
  // at the first branch to each neighbour, that neighbour's entries (summed
  // over parallel branches in branch order).
  double Ddd = __ldg(sx + tn) + dw;
  if (n == d.ref) Ddd = Ddd + __ldg(dv + t);
  double Dvv = __ldg(sx + d.x_vm + tn) + dw;
  double Dvd = 0.0;
  for (int32_t q = s0; q < s1; ++q) {
    const double2 a = ld_rec<COH>(R + (int64_t)q * kRec);      // (S_dd, S_vd)
    const double2 b = ld_rec<COH>(R + (int64_t)q * kRec + 2);  // (S_vv, S_vtvf)
    Ddd = Ddd + a.x;
    Dvv = Dvv + b.x;
    Dvd = (q == s0) ? a.y : Dvd + a.y;
    const int32_t info = __ldg(d.slot_info + q);
    if (info & (1 << 30)) {
      double cdd = negx(a.x), cvd = negx(a.y), cvv = b.y;
      for (int32_t o = __ldg(d.slot_next + q); o >= 0; o = __ldg(d.slot_next + o)) {
        const double2 a2 = ld_rec<COH>(R + (int64_t)o * kRec), b2 = ld_rec<COH>(R + (int64_t)o * kRec + 2);
        cdd = cdd - a2.x;
        cvd = cvd - a2.y;
        cvv = cvv + b2.y;
      }
      const int32_t k = info & 0x0fffffff;
      if (info & (1 << 29)) {  // neighbour index below n
        va_row[k] = cdd;
        vm_row[nd + 1 + k] = cvv;
        vm_row[k] = cvd;
      } else {
        vm_row[k + 1] = cvd;
      }
    }
  }
  const double D8 = __ldg(dv + d.c_k8 + tn), D9 = __ldg(dv + d.c_k9 + tn);
  const double w8 = D8 * J8, w9 = D9 * J9;
  const double Lbus = fma(w9, J9, fma(w8, J8, WP + WQ));
  Dvv = Dvv + Lbus;
  va_row[ndlt] = Ddd;
  if (nd > 0) vm_row[ndlt] = Dvd;
  vm_row[(nd > 0 ? nd + 1 : 0) + ndlt] = Dvv;
}

// Elements [first, end) of the bus x period range (t N + position).
template <unsigned MASK, int PART = 0, bool PTS = false>
__global__ void __launch_bounds__(MPOPF_BUS_BLOCK) k_bus(Dev d, unsigned rt, const double *__restrict__ x,
                                                const double *__restrict__ lam, const double *__restrict__ sx,
                                                const double *__restrict__ dv, double dw, double *__restrict__ grad,
                                                double *__restrict__ c, double *__restrict__ jv,
                                                double *__restrict__ hv, double *__restrict__ kv, int32_t first,
                                                int32_t end) {
  const int32_t idx = first + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (idx >= end) return;
  if (PTS) {
    MPOPF_POINT_OFFSETS(d);
    lam += (int64_t)blockIdx.y * d.m;
  }
  bus_body<MASK, false, true, PART, PTS>(d, idx, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv);
}

// ---------------------------------------------------------------------------
// Generator x period.  Called by whole CTAs (the objective's block tree);
// blk = index of the CTA-sized tile, where the tile's partial sum is stored.
// ---------------------------------------------------------------------------
template <unsigned MASK>
__device__ __forceinline__ void gen_body(const Dev &d, int32_t tg, int32_t end, int32_t blk, unsigned rt,
                                         const double *__restrict__ x, double sigma, const double *__restrict__ sx,
                                         const double *__restrict__ dv, double dw, double *__restrict__ grad,
                                         double *__restrict__ c, double *__restrict__ jv, double *__restrict__ hv,
                                         double *__restrict__ kv) {
  // tg: element t G + g; elements at or past `end` only add 0 to the tile sum
  const unsigned mk = eff<MASK>(rt);
  const int32_t G = d.G;
  const bool live = tg < end;
  const int32_t t = live ? tg / G : 0, g = live ? tg - t * G : 0;
  double pg = 0.0;
  if (live) pg = __ldg(x + d.x_pg + tg);
  if (mk & MPOPF_OUT_OBJ) {
    __shared__ double red[kBlock];
    red[threadIdx.x] = live ? fma(fma(__ldg(d.gen_c2 + g), pg, __ldg(d.gen_c1 + g)), pg, __ldg(d.gen_c0 + g)) : 0.0;
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) d.fpart[blk] = red[0];
  }
  if (!live) return;
  const double c2x2 = __ldg(d.gen_c2x2 + g);
  if (mk & MPOPF_OUT_GRAD) {
    grad[d.x_pg + tg] = fma(c2x2, pg, __ldg(d.gen_c1 + g));
    grad[d.x_qg + tg] = 0.0;
  }
  const double Wobj = sigma * c2x2;
  if (mk & MPOPF_OUT_HESS) hv[tg] = Wobj;
  const int64_t rr = d.c_k10 + (int64_t)(t - 1) * G + g;  // ramp row (t, g)
  const int64_t rq = d.c_k11 + (int64_t)(t - 1) * G + g;  // reactive ramp row (t, g), if present
  if (t >= 1) {
    if (mk & MPOPF_OUT_CONS) {
      c[rr] = pg - __ldg(x + d.x_pg + tg - G);
      if (d.qramp) c[rq] = __ldg(x + d.x_qg + tg) - __ldg(x + d.x_qg + tg - G);
    }
    if (mk & MPOPF_OUT_JAC) {
      jv[d.j_k10 + 2 * ((int64_t)(t - 1) * G + g)] = 1.0;
      jv[d.j_k10 + 2 * ((int64_t)(t - 1) * G + g) + 1] = -1.0;
      if (d.qramp) {
        jv[d.j_k11 + 2 * ((int64_t)(t - 1) * G + g)] = 1.0;
        jv[d.j_k11 + 2 * ((int64_t)(t - 1) * G + g) + 1] = -1.0;
      }
    }
  }
  if (!(mk & MPOPF_OUT_KKT)) return;
  const int32_t nb = __ldg(d.gen_bus + g), rank = __ldg(d.gen_rank + g);
  const int64_t tn = (int64_t)t * d.N + nb;
  const double vm = __ldg(x + d.x_vm + tn);
  const double D8 = __ldg(dv + d.c_k8 + tn), D9 = __ldg(dv + d.c_k9 + tn);
  const double w8 = D8 * (__ldg(d.bus_m2gs + nb) * vm), w9 = D9 * (__ldg(d.bus_p2bs + nb) * vm);
  double *pr = kv + d.m_pg + (t == 0 ? (int64_t)__ldg(d.mo_pg0 + g)
                                     : d.mb_pg0 + (int64_t)(t - 1) * d.mb_pg1 + __ldg(d.mo_pg1 + g));
  pr[0] = w8;
  int k = 1;
  double diag = ((__ldg(sx + d.x_pg + tg) + dw) + Wobj) + D8;
  if (t >= 1) {
    const double D10 = __ldg(dv + rr);
    pr[k++] = negx(D10);
    diag = diag + D10;
  }
  if (t + 1 < d.T) diag = diag + __ldg(dv + rr + G);
  for (int32_t e = 0; e < rank; ++e) pr[k++] = D8;
  pr[k] = diag;
  double *qr = kv + d.m_qg + (t == 0 ? (int64_t)__ldg(d.mo_qg + g)
                                     : d.mb_qg + (int64_t)(t - 1) * d.mb_qg1 + __ldg(d.mo_qg1 + g));
  qr[0] = w9;
  k = 1;
  double qdiag = (__ldg(sx + d.x_qg + tg) + dw) + D9;
  if (d.qramp) {
    if (t >= 1) {
      const double D11 = __ldg(dv + rq);
      qr[k++] = negx(D11);
      qdiag = qdiag + D11;
    }
    if (t + 1 < d.T) qdiag = qdiag + __ldg(dv + rq + G);
  }
  for (int32_t e = 0; e < rank; ++e) qr[k++] = D9;
  qr[k] = qdiag;
}

// Elements [first, end) of the generator x period range (t G + g); tile k's
// partial objective goes to fpart[k] (with PTS, point blockIdx.y's tiles
// follow the earlier points').
template <unsigned MASK, bool PTS = false>
__global__ void __launch_bounds__(kBlock) k_gen(Dev d, unsigned rt, const double *__restrict__ x, double sigma,
                                                const double *__restrict__ sx, const double *__restrict__ dv, double dw,
                                                double *__restrict__ grad, double *__restrict__ c,
                                                double *__restrict__ jv, double *__restrict__ hv,
                                                double *__restrict__ kv, int32_t first, int32_t end) {
  if (PTS) MPOPF_POINT_OFFSETS(d);
  const int32_t blk = PTS ? (int32_t)(blockIdx.y * gridDim.x + blockIdx.x) : (int32_t)blockIdx.x;
  gen_body<MASK>(d, first + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x), end, blk, rt, x, sigma, sx, dv, dw,
                 grad, c, jv, hv, kv);
}

// Objective: fixed-order reduction of the per-tile partial sums by one CTA of
// kBlock threads (strided sequential sums, then a tree).
template <bool COH>
__device__ __forceinline__ void fsum_body(const double *part, int32_t count, double *f) {
  __shared__ double red[kBlock];
  double a = 0.0;
  for (int32_t i = threadIdx.x; i < count; i += kBlock) a = a + ld_part<COH>(part + i);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = kBlock / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *f = red[0];
}

__global__ void __launch_bounds__(kBlock) k_fsum(const double *__restrict__ part, int32_t count,
                                                 double *__restrict__ f) {
  fsum_body<false>(part, count, f);
}

// The objectives of a sweep over several points: CTA j sums point j's
// `count` partials into f[j].
__global__ void __launch_bounds__(kBlock) k_fsum_points(const double *__restrict__ part, int32_t count,
                                                        double *__restrict__ f) {
  fsum_body<false>(part + (int64_t)blockIdx.x * count, count, f + blockIdx.x);
}

unsigned grid_for(int64_t count) { return (unsigned)((count + kBlock - 1) / kBlock); }


// The generator kernel (and the objective sum after it) on stream g, which is
// the caller's stream s or the handle's side stream.
// `after`, when not null, is an event the generator work also waits for (a
// caller's halo exchange of a period shard).
template <unsigned MASK>
void launch_gen_part(const Dev &d, unsigned rt, unsigned mk, const double *x, double sigma, const double *sx,
                     const double *dv, double dw, double *f, double *grad, double *c, double *jv, double *hv,
                     double *kv, cudaStream_t g, Prof *prof, cudaEvent_t after = nullptr) {
  if (after && mk) cudaStreamWaitEvent(g, after, 0);
  // the owned periods' elements; the objective sums exactly the tiles launched
  const int32_t first = d.w0 * d.G, end = d.w1 * d.G;
  const unsigned tiles = grid_for((int64_t)end - first);
  if (mk && d.G > 0) {
    Timed tm(prof, g, KIND_GEN);
    k_gen<MASK><<<tiles, kBlock, 0, g>>>(d, rt, x, sigma, sx, dv, dw, grad, c, jv, hv, kv, first, end);
  }
  if (mk & MPOPF_OUT_OBJ) {
    Timed tm(prof, g, KIND_FSUM);
    k_fsum<<<1, kBlock, 0, g>>>(d.fpart, d.G > 0 ? (int32_t)tiles : 0, f);
  }
}

// With a fork, the generator part runs on the side stream alongside the bus
// kernel, after the branch kernel (measured, CUDA graph of sweeps: 66.8 ->
// 60.1 us per sweep at 2,000 buses x 24, 39.0 -> 33.3 us at 10k buses x 1,
// 1127 -> 1117 us at 10k buses x 168; forked before the branch kernel it
// shared the SMs with the dominant kernel instead).  The side-stream
// launches are not bracketed by profiling events: their durations would
// include the wait for SMs held by the bus kernel.
// Number of period chunks of a chunked evaluation (0: not chunked).  At most
// kMaxChunks; the chunk length grows when the horizon needs more.
int chunk_count(const Dev &d, const Fork *fork, int32_t *per) {
  const int32_t W = d.w1 - d.w0;  // owned periods
  if (!fork || !fork->bus || fork->chunk <= 0 || d.L == 0 || W <= fork->chunk) return 0;
  int32_t P = fork->chunk;
  if ((W + P - 1) / P > kMaxChunks) P = (W + kMaxChunks - 1) / kMaxChunks;
  *per = P;
  return (W + P - 1) / P;
}

// Chunked evaluation: the branch kernel of each chunk of periods on s, the bus
// kernel of that chunk on the fork's bus stream behind an event recorded after
// it, the generator work on the side stream (forked before the first branch
// chunk or after the last); both streams join s at the end.  Every element is
// computed by the same code as in launch_all, so the outputs are the same bit
// for bit.
template <unsigned MASK>
cudaError_t launch_chunked(const Dev &d, unsigned rt, unsigned mk, const double *x, const double *lam, double sigma,
                           const double *sx, const double *dv, double dw, double *f, double *grad, double *c,
                           double *jv, double *hv, double *kv, cudaStream_t s, const Fork *fork, int32_t P,
                           int nch, bool side) {
  cudaError_t e = cudaEventRecord(fork->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->bus, fork->ev_fork, 0);
  const bool gen_first = fork->flags & SCHED_GEN_FIRST;
  if (e == cudaSuccess && side && gen_first) {
    e = cudaStreamWaitEvent(fork->side, fork->ev_fork, 0);
    if (e == cudaSuccess)
      launch_gen_part<MASK>(d, rt, mk, x, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, fork->side, nullptr,
                            fork->gen_after);
  }
  for (int k = 0; k < nch && e == cudaSuccess; ++k) {
    const int32_t t0 = d.w0 + k * P, t1 = std::min(d.w1, t0 + P);
    const int32_t bf = t0 * d.L, be = t1 * d.L;
    launch_branch<MASK>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, bf, be, s);
    e = cudaEventRecord(fork->ev_chunk[k], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->bus, fork->ev_chunk[k], 0);
    if (e != cudaSuccess) break;
    const int32_t nf = t0 * d.N, ne = t1 * d.N;
    k_bus<MASK><<<(unsigned)((ne - nf + MPOPF_BUS_BLOCK - 1) / MPOPF_BUS_BLOCK), MPOPF_BUS_BLOCK, 0, fork->bus>>>(
        d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, nf, ne);
  }
  if (e == cudaSuccess && side && !gen_first) {
    e = cudaStreamWaitEvent(fork->side, fork->ev_chunk[nch - 1], 0);
    if (e == cudaSuccess)
      launch_gen_part<MASK>(d, rt, mk, x, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, fork->side, nullptr,
                            fork->gen_after);
  }
  if (e == cudaSuccess) e = cudaEventRecord(fork->ev_bus, fork->bus);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork->ev_bus, 0);
  if (e == cudaSuccess && side) {
    e = cudaEventRecord(fork->ev_join, fork->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork->ev_join, 0);
  }
  if (e == cudaSuccess && !side)
    launch_gen_part<MASK>(d, rt, mk, x, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, nullptr, fork->gen_after);
  return e;
}

template <unsigned MASK>
cudaError_t launch_all(const Dev &d, unsigned rt, const double *x, const double *lam, double sigma, const double *sx,
                       const double *dv, double dw, double *f, double *grad, double *c, double *jv, double *hv,
                       double *kv, cudaStream_t s, Prof *prof, const Fork *fork) {
  const unsigned mk = MASK ? MASK : rt;
  const unsigned rest = MPOPF_OUT_GRAD | MPOPF_OUT_CONS | MPOPF_OUT_JAC | MPOPF_OUT_HESS | MPOPF_OUT_KKT;
  const bool side = fork && (mk & rest) && (mk && d.G > 0);  // both parts have work
  int32_t P = 0;
  const int nch = prof ? 0 : chunk_count(d, fork, &P);  // per-kernel profiling times whole launches
  if (nch > 0 && (mk & rest))
    return launch_chunked<MASK>(d, rt, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, fork, P, nch, side);
  const int32_t W = d.w1 - d.w0;  // owned periods
  // Programmatic dependent launch: the bus kernel may start while the branch
  // kernel finishes (it waits before reading the records).  The generator
  // work is still forked after the branch kernel (an event recorded between
  // the two launches), so it overlaps the bus kernel; measured at 10k buses x
  // 168 / 2,000 x 24 / 10k x 1: 1.0602 / 0.0527 / 0.0287 ms per sweep against
  // 1.0624 / 0.0555 / 0.0308 ms without (CUDA graphs of sweeps: 1.0558 /
  // 0.0500 / 0.0251 against 1.0577 / 0.0514 / 0.0257 ms).
  const bool pdl = fork && (fork->flags & SCHED_PDL) && !prof && (mk & rest) && d.L > 0;
  auto fork_gen = [&]() -> cudaError_t {
    cudaError_t e = cudaEventRecord(fork->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->side, fork->ev_fork, 0);
    if (e != cudaSuccess) return e;
    launch_gen_part<MASK>(d, rt, mk, x, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, fork->side, nullptr,
                          fork->gen_after);
    return cudaSuccess;
  };
  // SCHED_BUS_TERMS (full sweeps): the bus-end products in a launch of
  // their own before the branch kernel
  const bool bwp = MASK == MPOPF_OUT_ALL && fork && (fork->flags & SCHED_BUS_TERMS) && d.L > 0 && d.N > 0;
  if (bwp) {
    const cudaError_t e = launch_branch_bw<MASK>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, s,
                                                 (fork->flags & SCHED_PDL) && !prof, prof, fork->sms);
    if (e != cudaSuccess) return e;
  } else if ((mk & rest) && d.L > 0) {
    Timed tm(prof, s, KIND_BRANCH);
    (void)W;
    launch_branch<MASK>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, d.w0 * d.L, d.w1 * d.L, s);
  }
  if (side) {
    const cudaError_t e = fork_gen();
    if (e != cudaSuccess) return e;
  }
  // Split bus work (SCHED_SPLIT_BUS): the balance part on the fork's bus
  // stream and the M part on s, side by side after the branch kernel.
  const bool split = fork && (fork->flags & SCHED_SPLIT_BUS) && fork->bus && !prof && (mk & MPOPF_OUT_KKT) &&
                     (mk & (MPOPF_OUT_GRAD | MPOPF_OUT_CONS | MPOPF_OUT_JAC | MPOPF_OUT_HESS));
  if (split) {
    const unsigned grid = (unsigned)(((int64_t)W * d.N + MPOPF_BUS_BLOCK - 1) / MPOPF_BUS_BLOCK);
    const int32_t bf = d.w0 * d.N, be = d.w1 * d.N;
    cudaError_t e = cudaEventRecord(fork->ev_chunk[0], s);  // after the branch kernel
    if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->bus, fork->ev_chunk[0], 0);
    if (e != cudaSuccess) return e;
    k_bus<MASK, 1><<<grid, MPOPF_BUS_BLOCK, 0, fork->bus>>>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, bf, be);
    k_bus<MASK, 2><<<grid, MPOPF_BUS_BLOCK, 0, s>>>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, bf, be);
    e = cudaEventRecord(fork->ev_bus, fork->bus);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork->ev_bus, 0);
    if (e != cudaSuccess) return e;
  } else if (mk & rest) {
    Timed tm(prof, s, KIND_BUS);
    const unsigned grid = (unsigned)(((int64_t)W * d.N + MPOPF_BUS_BLOCK - 1) / MPOPF_BUS_BLOCK);
    const int32_t bf = d.w0 * d.N, be = d.w1 * d.N;
    if (pdl) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(MPOPF_BUS_BLOCK);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, k_bus<MASK>, d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv,
                                               bf, be);
      if (e != cudaSuccess) return e;
    } else {
      k_bus<MASK><<<grid, MPOPF_BUS_BLOCK, 0, s>>>(d, rt, x, lam, sx, dv, dw, grad, c, jv, hv, kv, bf, be);
    }
  }
  if (side) {
    cudaError_t e = cudaEventRecord(fork->ev_join, fork->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork->ev_join, 0);
    return e;
  }
  launch_gen_part<MASK>(d, rt, mk, x, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof,
                        fork ? fork->gen_after : nullptr);
  return cudaSuccess;
}

// Whether a sweep over `points` points forms the bus-end products in a launch
// of their own: the same rule as a single sweep's default schedule, applied
// to all points' branch elements.
bool points_bus_terms(const Dev &d, int32_t points, const Fork *fork) {
  const int64_t wave = (int64_t)fork->sms * MPOPF_BRANCH_BLOCK * MPOPF_BRANCH_MINB;
  return d.N > 0 && (int64_t)points * d.T * d.L >= 2 * wave;
}

// A full sweep at `points` points of one network (the sweep's kernels once
// each, over every point: grid y): the branch kernel on s, the generator work
// and the objectives forked onto the side stream after it, the bus kernel as
// a programmatic dependent launch when the schedule has SCHED_PDL.  S and
// fpart hold the points' incidence records (points x 2 L T kRec doubles) and
// objective partials (points x tiles).  A point's elements run the code of a
// single sweep's, so its outputs are launch_all's at that point bit for bit.
cudaError_t launch_points(const Dev &d0, int32_t points, double *S, double *fpart, double *bw, const double *x,
                          const double *lam, double sigma, const double *sx, const double *dv, double dw, double *f,
                          double *grad, double *c, double *jv, double *hv, double *kv, cudaStream_t s,
                          const Fork *fork) {
  constexpr unsigned A = MPOPF_OUT_ALL;
  Dev d = d0;
  d.S = S;
  d.fpart = fpart;
  d.bw = bw;
  const unsigned P = (unsigned)points;
  if (d.L > 0 && points_bus_terms(d, points, fork)) {
    // the points' bus-end products first (grid y = point), then the branch
    // kernel reading them, its programmatic dependent launch
    const int32_t be = d.T * d.N;
    const unsigned gx = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)be + kBlock - 1) / kBlock, (4 * (int64_t)fork->sms + P - 1) / P));
    k_bw<true><<<dim3(gx, P), kBlock, 0, s>>>(d, x, dv, 0, be);
    const int32_t end = d.T * d.L;
    const dim3 grid((unsigned)(((int64_t)end + MPOPF_BRANCH_BLOCK - 1) / MPOPF_BRANCH_BLOCK), P);
    void (*kern)(Dev, unsigned, const double *, const double *, const double *, const double *, double, double *,
                 double *, double *, double *, double *, int32_t, int32_t) =
        d.all_sym ? k_branch<A, true, true, true> : k_branch<A, false, true, true>;
    if (fork->flags & SCHED_PDL) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = dim3(MPOPF_BRANCH_BLOCK);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, d, A, x, lam, sx, dv, dw, grad, c, jv, hv, kv, 0, end);
      if (e != cudaSuccess) return e;
    } else {
      kern<<<grid, MPOPF_BRANCH_BLOCK, 0, s>>>(d, A, x, lam, sx, dv, dw, grad, c, jv, hv, kv, 0, end);
    }
  } else if (d.L > 0) {
    launch_branch<A, true>(d, A, x, lam, sx, dv, dw, grad, c, jv, hv, kv, 0, d.T * d.L, s, P);
  }
  cudaError_t e = cudaEventRecord(fork->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->side, fork->ev_fork, 0);
  if (e != cudaSuccess) return e;
  const int32_t tg = d.T * d.G;
  const unsigned tiles = grid_for(tg);
  if (d.G > 0)
    k_gen<A, true><<<dim3(tiles, P), kBlock, 0, fork->side>>>(d, A, x, sigma, sx, dv, dw, grad, c, jv, hv, kv, 0, tg);
  k_fsum_points<<<P, kBlock, 0, fork->side>>>(fpart, d.G > 0 ? (int32_t)tiles : 0, f);
  const dim3 grid((unsigned)(((int64_t)d.T * d.N + MPOPF_BUS_BLOCK - 1) / MPOPF_BUS_BLOCK), P);
  const int32_t be = d.T * d.N;
  if ((fork->flags & SCHED_PDL) && d.L > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(MPOPF_BUS_BLOCK);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_bus<A, 0, true>, d, A, x, lam, sx, dv, dw, grad, c, jv, hv, kv, 0, be);
    if (e != cudaSuccess) return e;
  } else {
    k_bus<A, 0, true><<<grid, MPOPF_BUS_BLOCK, 0, s>>>(d, A, x, lam, sx, dv, dw, grad, c, jv, hv, kv, 0, be);
  }
  e = cudaEventRecord(fork->ev_join, fork->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork->ev_join, 0);
  return e;
}

// ---------------------------------------------------------------------------
// Persistent batch kernel: CTAs take items (CTA-sized tiles of one instance's
// branch, generator, bus or objective work) from a global counter in list
// order.  The list holds every branch and generator item before any bus or
// objective item, so an item's prerequisites were all taken earlier by running
// CTAs; a bus item waits until its instance's branch items are done (their
// incidence records written), an objective item until its generator items are.
// The wait is bounded: past the limit the flag ctl[1] is set and the item is
// computed anyway (the host reports an error).
// ---------------------------------------------------------------------------
constexpr long long kWaitLimit = 1LL << 22;  // x ~0.25 us sleep: about a second

__device__ __forceinline__ int32_t ld_acquire(const int32_t *p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The branch items of the batch kernel (phases 0 and 1, CTAs of B threads):
// warps whose 32 elements all lie in the item stage their J and W rows in
// shared memory.
template <int B>
__device__ __forceinline__ void batch_branch_item(const Dev &d, const BatchIO &b, int32_t first, int32_t end) {
  __shared__ __align__(16) double s_stage[B / 32][kStageCap];
  for (int32_t c0 = first; c0 < end; c0 += B) {
    const bool full = c0 + (int32_t)(threadIdx.x & ~31u) + 31 < end;
    if (c0 + (int32_t)threadIdx.x < end)
      branch_body<MPOPF_OUT_ALL, true>(d, c0 + threadIdx.x, MPOPF_OUT_ALL, b.x, b.lam, b.sx, b.dv, b.dw, b.grad,
                                       b.c, b.jv, b.hv, b.kv, full ? s_stage[threadIdx.x >> 5] : nullptr);
  }
}

// PHASE 0: every kind of item in one persistent launch (bus and objective
// items wait for their prerequisites), 256-thread CTAs, 3 per SM.
// PHASE 1: the branch items, in the sweep kernel's shape (64-thread CTAs, 12
// per SM).  PHASE 2, launched after phase 1 (the launch boundary orders the
// bus items after the branch items, so they do not wait): the generator
// items, the bus items and then the objective items, which wait for their
// instance's generator items; 256-thread CTAs (the objective's tile tree),
// 5 per SM at the bus work's 48 registers (the bus kernel alone is 49% slower
// at 3 per SM).  `next` is the launch's work-item counter.
__host__ __device__ constexpr int batch_block(int phase) { return phase == 1 ? MPOPF_BRANCH_BLOCK : kBlock; }
__host__ __device__ constexpr int batch_minb(int phase) {
  return phase == 1 ? MPOPF_BRANCH_MINB : phase == 2 ? 5 : 3;
}
template <int PHASE>
__global__ void __launch_bounds__(batch_block(PHASE), batch_minb(PHASE))
    k_batch(const Dev *__restrict__ devs, const BatchIO *__restrict__ io, const BatchItem *__restrict__ items,
            int32_t n_items, const int32_t *__restrict__ need, int32_t *__restrict__ ctl, int32_t *__restrict__ next) {
  constexpr int B = batch_block(PHASE);
  constexpr bool WAITS = PHASE != 1;  // phases whose items may wait or signal
  __shared__ int32_t s_item;
  __shared__ int32_t s_inst;
  // The instance's descriptors, copied to shared memory when the instance
  // changes (the bodies read their fields many times).
  __shared__ __align__(16) unsigned char s_dev[sizeof(Dev)];
  __shared__ __align__(16) unsigned char s_io[sizeof(BatchIO)];
  if (threadIdx.x == 0) s_inst = -1;
  const Dev &d = *reinterpret_cast<const Dev *>(s_dev);
  const BatchIO &b = *reinterpret_cast<const BatchIO *>(s_io);
  for (;;) {
    __syncthreads();  // the previous item is finished by every thread
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int32_t it = s_item;
    if (it >= n_items) {
      if (PHASE != 2) bulk_done((int)(threadIdx.x & 31));
      return;
    }
    const BatchItem I = items[it];
    if (I.inst != s_inst) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(devs + I.inst);
      for (int w = threadIdx.x; w < (int)(sizeof(Dev) / 4); w += B)
        reinterpret_cast<uint32_t *>(s_dev)[w] = src[w];
      const uint32_t *srci = reinterpret_cast<const uint32_t *>(io + I.inst);
      for (int w = threadIdx.x; w < (int)(sizeof(BatchIO) / 4); w += B)
        reinterpret_cast<uint32_t *>(s_io)[w] = srci[w];
      __syncthreads();
      if (threadIdx.x == 0) s_inst = I.inst;
      // s_inst is read again only after the barrier at the top of the loop
    }
    if (WAITS && I.wait >= 0) {
      if (threadIdx.x == 0) {
        const int32_t *cnt = ctl + 2 + I.wait;
        const int32_t target = need[I.wait];
        long long spins = 0;
        while (ld_acquire(cnt) < target) {
          if (++spins > kWaitLimit) {
            atomicExch(ctl + 1, 1);
            break;
          }
          __nanosleep(256);
        }
      }
      __syncthreads();
    }
    const int32_t end = I.first + I.count;
    if constexpr (PHASE != 2) {
      if (I.kind == ITEM_BRANCH) batch_branch_item<B>(d, b, I.first, end);
    }
    if constexpr (PHASE != 1) {
      static_assert(B == kBlock, "the generator and objective trees need kBlock-thread CTAs");
      if (I.kind == ITEM_GEN) {
        for (int32_t c0 = I.first; c0 < end; c0 += kBlock)  // whole CTA: the objective tile tree
          gen_body<MPOPF_OUT_ALL>(d, c0 + threadIdx.x, end, c0 / kBlock, MPOPF_OUT_ALL, b.x, b.sigma, b.sx, b.dv,
                                  b.dw, b.grad, b.c, b.jv, b.hv, b.kv);
      } else if (I.kind == ITEM_BUS) {
        // records from the same launch (phase 0) are read through L2; from
        // the earlier launch (phase 2), through the read-only path
        for (int32_t c0 = I.first; c0 < end; c0 += kBlock)
          if (c0 + (int32_t)threadIdx.x < end)
            bus_body<MPOPF_OUT_ALL, PHASE == 0>(d, c0 + threadIdx.x, MPOPF_OUT_ALL, b.x, b.lam, b.sx, b.dv, b.dw,
                                                b.grad, b.c, b.jv, b.hv, b.kv);
      } else if (I.kind == ITEM_FSUM) {
        fsum_body<true>(d.fpart, d.G > 0 ? d.fpart_n : 0, b.f);  // partials of the same launch: through L2
      }
    }
    if (WAITS && I.signal >= 0) {  // publish this item's writes, then count it done
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(ctl + 2 + I.signal, 1);
    }
  }
}

}  // namespace

// Periods [t0, t1) of the branch and bus work of a full sweep (every output of
// those periods); the generator work and the objective follow, for the whole
// horizon, in launch_gen_obj.  Together they launch exactly the work of
// launch_all<MPOPF_OUT_ALL>, element for element.
void launch_window(const Dev &d, int32_t t0, int32_t t1, const double *x, const double *lam, const double *sx,
                   const double *dv, double dw, double *grad, double *c, double *jv, double *hv, double *kv,
                   cudaStream_t s) {
  constexpr unsigned A = MPOPF_OUT_ALL;
  if (d.L > 0) {
    const int32_t first = t0 * d.L, end = t1 * d.L;
    launch_branch<A>(d, A, x, lam, sx, dv, dw, grad, c, jv, hv, kv, first, end, s);
  }
  const int32_t first = t0 * d.N, end = t1 * d.N;
  k_bus<A><<<(unsigned)(((int64_t)end - first + MPOPF_BUS_BLOCK - 1) / MPOPF_BUS_BLOCK), MPOPF_BUS_BLOCK, 0, s>>>(d, A, x, lam, sx, dv, dw, grad, c, jv, hv, kv, first,
                                                             end);
}

void launch_gen_obj(const Dev &d, const double *x, double sigma, const double *sx, const double *dv, double dw,
                    double *f, double *grad, double *c, double *jv, double *hv, double *kv, cudaStream_t s) {
  constexpr unsigned A = MPOPF_OUT_ALL;
  if (d.G > 0)
    k_gen<A><<<grid_for((int64_t)d.T * d.G), kBlock, 0, s>>>(d, A, x, sigma, sx, dv, dw, grad, c, jv, hv, kv, 0,
                                                             d.T * d.G);
  k_fsum<<<1, kBlock, 0, s>>>(d.fpart, d.G > 0 ? d.fpart_n : 0, f);
}

namespace {
const void *batch_kernel(int phase) {
  return phase == 2 ? reinterpret_cast<const void *>(k_batch<2>)
                    : phase == 1 ? reinterpret_cast<const void *>(k_batch<1>) : reinterpret_cast<const void *>(k_batch<0>);
}
}  // namespace

int batch_block_threads(int phase) { return batch_block(phase); }

int batch_max_ctas_per_sm(int phase) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel(phase), batch_block(phase), 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

cudaError_t batch_kernel_node(cudaKernelNodeParams *p, void **args, int32_t grid, int phase) {
  p->func = const_cast<void *>(batch_kernel(phase));
  p->gridDim = dim3((unsigned)grid);
  p->blockDim = dim3(batch_block(phase));
  p->sharedMemBytes = 0;
  p->kernelParams = args;
  p->extra = nullptr;
  return cudaSuccess;
}

cudaError_t fork_bus_stream(Fork *fork, bool high_priority) {
  if (fork->bus) cudaStreamDestroy(fork->bus);
  fork->bus = nullptr;
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);  // hi: numerically lowest = highest priority
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&fork->bus, cudaStreamNonBlocking, high_priority ? hi : lo);
  if (e == cudaSuccess && !fork->ev_bus) e = cudaEventCreateWithFlags(&fork->ev_bus, cudaEventDisableTiming);
  for (int k = 0; k < kMaxChunks && e == cudaSuccess; ++k)
    if (!fork->ev_chunk[k]) e = cudaEventCreateWithFlags(&fork->ev_chunk[k], cudaEventDisableTiming);
  return e;
}

int grow_points_scratch(mpopf_handle *h, size_t need, const char *who, cudaStream_t s) {
  if (need <= h->pts_bytes) return MPOPF_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    set_error(std::string(who) + ": the scratch must grow, which a stream capture does not allow; make a first call "
              "of this size (or larger) before capturing");
    return MPOPF_ERR_ARG;
  }
  if (h->pts) {
    // an earlier call's kernels may still use the old scratch
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaFree(h->pts);
    h->pts = nullptr;
    h->pts_bytes = 0;
    if (e != cudaSuccess) {
      set_error(std::string(who) + ": " + cudaGetErrorString(e));
      return MPOPF_ERR_CUDA;
    }
  }
  void *p = nullptr;
  const cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string(who) + ": scratch: " + cudaGetErrorString(e));
    return MPOPF_ERR_ALLOC;
  }
  h->pts = static_cast<double *>(p);
  h->pts_bytes = need;
  return MPOPF_OK;
}

// The default launch schedule of a new handle: the bus kernel as a
// programmatic dependent launch; the bus-end products in a launch of their own
// once the branch launch spans at least two waves of resident CTAs (measured,
// plain launches: 10k buses x 24 / 48 / 168 periods 2.7 / 2.8 / 1.1% faster,
// 2,000 x 96 / 192 2.5 / 2.0%, 118 x 10,080 2.5%; 2,000 x 48 and 10k x 12,
// under two waves, within 1.3%; 2,000 x 24, under one wave, a third slower).
int32_t device_sms(int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 148;  // B300
  }
  return sms;
}

int32_t default_schedule_flags(const Dev &d, int32_t sms) {
  const int64_t wave = (int64_t)sms * MPOPF_BRANCH_BLOCK * MPOPF_BRANCH_MINB;  // resident branch elements
  const int64_t elements = (int64_t)(d.w1 - d.w0) * d.L;
  return SCHED_PDL | (elements >= 2 * wave ? SCHED_BUS_TERMS : 0);
}

int eval_launch_count(const Dev &d, unsigned mk, const Fork *fork) {
  const unsigned rest = MPOPF_OUT_GRAD | MPOPF_OUT_CONS | MPOPF_OUT_JAC | MPOPF_OUT_HESS | MPOPF_OUT_KKT;
  int32_t P = 0;
  const int nch = chunk_count(d, fork, &P);
  int k = 0;
  if ((mk & rest) && nch > 0) k += 2 * nch;  // a branch and a bus launch per chunk
  else {
    if ((mk & rest) && d.L > 0) ++k;
    if (mk & rest) ++k;
    if (mk == MPOPF_OUT_ALL && (fork->flags & SCHED_BUS_TERMS) && d.L > 0 && d.N > 0) ++k;  // k_bw
    if ((fork->flags & SCHED_SPLIT_BUS) && (mk & MPOPF_OUT_KKT) &&
        (mk & (MPOPF_OUT_GRAD | MPOPF_OUT_CONS | MPOPF_OUT_JAC | MPOPF_OUT_HESS)))
      ++k;  // the bus work as two kernels
  }
  if (mk && d.G > 0) ++k;
  if (mk & MPOPF_OUT_OBJ) ++k;
  return k;
}

cudaError_t launch_eval(const Dev &d, unsigned mk, const double *x, const double *lam, double sigma,
                        const double *sx, const double *dv, double dw, double *f, double *grad, double *c,
                        double *jv, double *hv, double *kv, cudaStream_t s, Prof *prof, const Fork *fork) {
  cudaError_t e = cudaSuccess;
  switch (mk) {
    case MPOPF_OUT_OBJ: e = launch_all<MPOPF_OUT_OBJ>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
    case MPOPF_OUT_GRAD: e = launch_all<MPOPF_OUT_GRAD>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
    case MPOPF_OUT_CONS: e = launch_all<MPOPF_OUT_CONS>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
    case MPOPF_OUT_JAC: e = launch_all<MPOPF_OUT_JAC>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
    case MPOPF_OUT_HESS: e = launch_all<MPOPF_OUT_HESS>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
    case MPOPF_OUT_KKT: e = launch_all<MPOPF_OUT_KKT>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
    case MPOPF_OUT_ALL: e = launch_all<MPOPF_OUT_ALL>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
    default: e = launch_all<0>(d, mk, x, lam, sigma, sx, dv, dw, f, grad, c, jv, hv, kv, s, prof, fork); break;
  }
  const cudaError_t l = cudaGetLastError();
  return e != cudaSuccess ? e : l;
}

}  // namespace mpopf

using namespace mpopf;

namespace {
int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

}  // namespace


extern "C" {

int mpopf_launch_count(const mpopf_handle *h, unsigned outputs) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_launch_count: NULL handle");
  return eval_launch_count(h->d, outputs & MPOPF_OUT_ALL, &h->fork);
}

int mpopf_set_sweep_schedule(mpopf_handle *h, int32_t chunk_periods, int32_t flags) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_set_sweep_schedule: NULL handle");
  if (chunk_periods < 0 ||
      (flags & ~(SCHED_BUS_PRIORITY | SCHED_GEN_FIRST | SCHED_PDL | SCHED_SPLIT_BUS | SCHED_BUS_TERMS)))
    return fail(MPOPF_ERR_ARG, "mpopf_set_sweep_schedule: bad argument");
  if ((flags ^ h->fork.flags) & SCHED_BUS_PRIORITY) {
    const cudaError_t e = fork_bus_stream(&h->fork, flags & SCHED_BUS_PRIORITY);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MPOPF_ERR_CUDA, std::string("mpopf_set_sweep_schedule: ") + cudaGetErrorString(e));
    }
  }
  h->fork.chunk = chunk_periods;
  h->fork.flags = flags;
  return MPOPF_OK;
}

int mpopf_set_gen_dependency(mpopf_handle *h, void *event) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_set_gen_dependency: NULL handle");
  h->fork.gen_after = static_cast<cudaEvent_t>(event);
  return MPOPF_OK;
}

int mpopf_get_sweep_schedule(const mpopf_handle *h, int32_t *chunk_periods, int32_t *flags) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_get_sweep_schedule: NULL handle");
  if (chunk_periods) *chunk_periods = h->fork.chunk;
  if (flags) *flags = h->fork.flags;
  return MPOPF_OK;
}

int mpopf_eval(mpopf_handle *h, unsigned outputs, const double *x, const double *lam, double sigma,
               const double *sigma_x, const double *dvec, double delta_w, double *f, double *grad, double *c,
               double *jv, double *hv, double *kv, void *stream) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_eval: NULL handle");
  unsigned mk = outputs & MPOPF_OUT_ALL;
  if (!f) mk &= ~MPOPF_OUT_OBJ;
  if (!grad) mk &= ~MPOPF_OUT_GRAD;
  if (!c) mk &= ~MPOPF_OUT_CONS;
  if (!jv) mk &= ~MPOPF_OUT_JAC;
  if (!hv) mk &= ~MPOPF_OUT_HESS;
  if (!kv) mk &= ~MPOPF_OUT_KKT;
  if (mk == 0) return MPOPF_OK;
  if (!x) return fail(MPOPF_ERR_ARG, "mpopf_eval: NULL x");
  if ((mk & (MPOPF_OUT_HESS | MPOPF_OUT_KKT)) && !lam) return fail(MPOPF_ERR_ARG, "mpopf_eval: NULL lam");
  if ((mk & MPOPF_OUT_KKT) && (!sigma_x || !dvec)) return fail(MPOPF_ERR_ARG, "mpopf_eval: NULL sigma_x or dvec");
  const cudaError_t e = launch_eval(h->d, mk, x, lam, sigma, sigma_x, dvec, delta_w, f, grad, c, jv, hv, kv,
                                    static_cast<cudaStream_t>(stream), h->prof.cap ? &h->prof : nullptr, &h->fork);
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_eval: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

int mpopf_eval_obj(mpopf_handle *h, const double *x, double *f, void *stream) {
  return mpopf_eval(h, MPOPF_OUT_OBJ, x, nullptr, 0.0, nullptr, nullptr, 0.0, f, nullptr, nullptr, nullptr, nullptr,
                    nullptr, stream);
}
int mpopf_eval_grad(mpopf_handle *h, const double *x, double *grad, void *stream) {
  return mpopf_eval(h, MPOPF_OUT_GRAD, x, nullptr, 0.0, nullptr, nullptr, 0.0, nullptr, grad, nullptr, nullptr,
                    nullptr, nullptr, stream);
}
int mpopf_eval_cons(mpopf_handle *h, const double *x, double *c, void *stream) {
  return mpopf_eval(h, MPOPF_OUT_CONS, x, nullptr, 0.0, nullptr, nullptr, 0.0, nullptr, nullptr, c, nullptr, nullptr,
                    nullptr, stream);
}
int mpopf_eval_jac(mpopf_handle *h, const double *x, double *jv, void *stream) {
  return mpopf_eval(h, MPOPF_OUT_JAC, x, nullptr, 0.0, nullptr, nullptr, 0.0, nullptr, nullptr, nullptr, jv, nullptr,
                    nullptr, stream);
}
int mpopf_eval_hess(mpopf_handle *h, const double *x, const double *lam, double sigma, double *hv, void *stream) {
  return mpopf_eval(h, MPOPF_OUT_HESS, x, lam, sigma, nullptr, nullptr, 0.0, nullptr, nullptr, nullptr, nullptr, hv,
                    nullptr, stream);
}
int mpopf_assemble_kkt(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *sigma_x,
                       const double *dvec, double delta_w, double *kv, void *stream) {
  return mpopf_eval(h, MPOPF_OUT_KKT, x, lam, sigma, sigma_x, dvec, delta_w, nullptr, nullptr, nullptr, nullptr,
                    nullptr, kv, stream);
}
int mpopf_sweep(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *sigma_x,
                const double *dvec, double delta_w, double *f, double *grad, double *c, double *jv, double *hv,
                double *kv, void *stream) {
  if (!f || !grad || !c || !jv || !hv || !kv) return fail(MPOPF_ERR_ARG, "mpopf_sweep: NULL output");
  return mpopf_eval(h, MPOPF_OUT_ALL, x, lam, sigma, sigma_x, dvec, delta_w, f, grad, c, jv, hv, kv, stream);
}

int mpopf_sweep_points(mpopf_handle *h, int32_t points, const double *x, const double *lam, double sigma,
                       const double *sigma_x, const double *dvec, double delta_w, double *f, double *grad, double *c,
                       double *jv, double *hv, double *kv, void *stream) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_sweep_points: NULL handle");
  if (is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_sweep_points: not available on a period shard");
  if (points < 1 || points > 65535) return fail(MPOPF_ERR_ARG, "mpopf_sweep_points: points outside [1, 65535]");
  if (!x || !lam || !sigma_x || !dvec || !f || !grad || !c || !jv || !hv || !kv)
    return fail(MPOPF_ERR_ARG, "mpopf_sweep_points: NULL buffer");
  const Dev &d = h->d;
  const size_t rec = (size_t)2 * d.L * d.T * kRec;  // record doubles of one point
  const size_t tiles = grid_for((int64_t)d.T * d.G);
  const size_t bwn = points_bus_terms(d, points, &h->fork) ? (size_t)2 * d.T * d.N : 0;  // bus-end products
  const int rc = grow_points_scratch(h, (size_t)points * (rec + tiles + bwn) * sizeof(double), "mpopf_sweep_points",
                                     static_cast<cudaStream_t>(stream));
  if (rc != MPOPF_OK) return rc;
  cudaError_t e = launch_points(d, points, h->pts, h->pts + (size_t)points * rec,
                                h->pts + (size_t)points * (rec + tiles), x, lam, sigma, sigma_x, dvec, delta_w, f,
                                grad, c, jv, hv, kv, static_cast<cudaStream_t>(stream), &h->fork);
  const cudaError_t l = cudaGetLastError();
  if (e == cudaSuccess) e = l;
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_sweep_points: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

int mpopf_profile_start(mpopf_handle *h, int32_t max_launches) {
  if (!h || max_launches < 1) return fail(MPOPF_ERR_ARG, "mpopf_profile_start: bad argument");
  if (h->prof.cap) return fail(MPOPF_ERR_ARG, "mpopf_profile_start: already profiling");
  Prof &p = h->prof;
  p.ev = new cudaEvent_t[2 * (size_t)max_launches];
  p.kind = new int[max_launches];
  for (int i = 0; i < 2 * max_launches; ++i) {
    const cudaError_t e = cudaEventCreate(&p.ev[i]);
    if (e != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(p.ev[k]);
      delete[] p.ev;
      delete[] p.kind;
      p = Prof();
      return fail(MPOPF_ERR_CUDA, std::string("mpopf_profile_start: ") + cudaGetErrorString(e));
    }
  }
  p.cap = max_launches;
  p.next = 0;
  return MPOPF_OK;
}

int mpopf_profile_stop(mpopf_handle *h, double *ms_sum, int32_t *launches) {
  if (!h || !h->prof.cap) return fail(MPOPF_ERR_ARG, "mpopf_profile_stop: not profiling");
  Prof &p = h->prof;
  int rc = MPOPF_OK;
  for (int k = 0; k < KIND_COUNT; ++k) { if (ms_sum) ms_sum[k] = 0.0; if (launches) launches[k] = 0; }
  for (int i = 0; i < p.next; ++i) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(p.ev[2 * i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]);
    if (e != cudaSuccess) { rc = fail(MPOPF_ERR_CUDA, std::string("mpopf_profile_stop: ") + cudaGetErrorString(e)); break; }
    if (ms_sum) ms_sum[p.kind[i]] += ms;
    if (launches) launches[p.kind[i]] += 1;
  }
  for (int i = 0; i < 2 * p.cap; ++i) cudaEventDestroy(p.ev[i]);
  delete[] p.ev;
  delete[] p.kind;
  p = Prof();
  return rc;
}

}  // extern "C"
