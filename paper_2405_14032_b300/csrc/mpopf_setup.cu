// Setup of libmpopf: validation, layout, per-period templates, device upload and
// expansion of the J, W and M patterns over the horizon.
//
// Sec. III-A of the paper analyses the sparsity of each repeated pattern once
// and expands it over the data array; here the analysis is the per-period
// template (row lengths and offsets of one period, identical for every period
// except the ramp entries of the generator rows at t >= 1) and the expansion is
// a GPU kernel per pattern.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "mpopf_internal.cuh"

namespace mpopf {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

namespace {

// ---------------------------------------------------------------------------
// Pattern expansion kernels (one thread per row or entry).
// ---------------------------------------------------------------------------
__global__ void k_pat_jac(Dev d, int32_t *__restrict__ jrow, int32_t *__restrict__ jcol) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= d.m) return;
  const int64_t T = d.T, L = d.L, N = d.N, G = d.G;
  if (i < T) {
    jrow[i] = (int32_t)i;
    jcol[i] = (int32_t)(i * N + d.ref);
    return;
  }
  const int64_t TL = T * L;
  int64_t r = i - T;
  if (r < 7 * TL) {
    const int k = (int)(r / TL) + 1;
    const int64_t tl = r - (k - 1) * TL, t = tl / L, l = tl - t * L;
    const int64_t f = d.br_f[l], to = d.br_t[l];
    const int64_t vaf = t * N + f, vat = t * N + to, vmf = d.x_vm + t * N + f, vmt = d.x_vm + t * N + to;
    if (k <= 4) {
      const int64_t arc = (k == 1) ? d.x_p + 2 * t * L + l
                        : (k == 2) ? d.x_q + 2 * t * L + l
                        : (k == 3) ? d.x_p + 2 * t * L + L + l
                                   : d.x_q + 2 * t * L + L + l;
      const int64_t o = T + 5 * (k - 1) * TL + tl * 5;
      const int64_t cols[5] = {arc, vaf, vat, vmf, vmt};
      for (int e = 0; e < 5; ++e) { jrow[o + e] = (int32_t)i; jcol[o + e] = (int32_t)cols[e]; }
    } else if (k == 5) {
      const int64_t o = d.j_k5 + tl * 2;
      jrow[o] = (int32_t)i; jcol[o] = (int32_t)vaf;
      jrow[o + 1] = (int32_t)i; jcol[o + 1] = (int32_t)vat;
    } else {
      const int64_t a = (k == 6) ? l : L + l;
      const int64_t o = (k == 6 ? d.j_k6 : d.j_k7) + tl * 2;
      jrow[o] = (int32_t)i; jcol[o] = (int32_t)(d.x_p + 2 * t * L + a);
      jrow[o + 1] = (int32_t)i; jcol[o + 1] = (int32_t)(d.x_q + 2 * t * L + a);
    }
    return;
  }
  r -= 7 * TL;
  if (r < 2 * T * N) {
    const bool P = r < T * N;
    const int64_t tn = P ? r : r - T * N, t = tn / N, nb = tn - t * N;
    int64_t o = (P ? d.j_k8 : d.j_k9) + t * d.jk8_per + d.jk8_off[nb];
    jrow[o] = (int32_t)i; jcol[o] = (int32_t)(d.x_vm + t * N + nb); ++o;
    for (int32_t e = d.bgen_ptr[nb]; e < d.bgen_ptr[nb + 1]; ++e, ++o) {
      jrow[o] = (int32_t)i;
      jcol[o] = (int32_t)((P ? d.x_pg : d.x_qg) + t * G + d.bgen_idx[e]);
    }
    for (int32_t e = d.barc_ptr[nb]; e < d.barc_ptr[nb + 1]; ++e, ++o) {
      jrow[o] = (int32_t)i;
      jcol[o] = (int32_t)((P ? d.x_p : d.x_q) + 2 * t * L + d.barc_idx[e]);
    }
    return;
  }
  r -= 2 * T * N;
  // K10 ramp of pg, then (if present) K11 ramp of qg: [var(t) (+1), var(t - 1) (-1)]
  const bool q = r >= (T - 1) * G;
  if (q) r -= (T - 1) * G;
  const int64_t t = 1 + r / G, g = r - (t - 1) * G;
  const int64_t o = (q ? d.j_k11 : d.j_k10) + r * 2, base = q ? d.x_qg : d.x_pg;
  jrow[o] = (int32_t)i; jcol[o] = (int32_t)(base + t * G + g);
  jrow[o + 1] = (int32_t)i; jcol[o + 1] = (int32_t)(base + (t - 1) * G + g);
}

__global__ void k_pat_hess(Dev d, int32_t *__restrict__ hrow, int32_t *__restrict__ hcol) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= d.nnz_hess) return;
  const int64_t T = d.T, L = d.L, N = d.N, G = d.G;
  int64_t r, c;
  if (e < d.h_br) {
    const int64_t t = e / G, g = e - t * G;
    r = c = d.x_pg + t * G + g;
  } else if (e < d.h_th) {
    const int64_t q = e - d.h_br, tl = q / 10, k = q - tl * 10, t = tl / L, l = tl - t * L;
    const int64_t u[4] = {t * N + d.br_f[l], t * N + d.br_t[l], d.x_vm + t * N + d.br_f[l], d.x_vm + t * N + d.br_t[l]};
    const int pa[10] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
    const int pb[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
    const int64_t A = u[pa[k]], B = u[pb[k]];
    r = A > B ? A : B;
    c = A > B ? B : A;
  } else if (e < d.h_sh) {
    const int64_t q = e - d.h_th, tl = q / 4, k = q - tl * 4, t = tl / L, l = tl - t * L;
    const int64_t a = (k < 2) ? l : L + l;
    r = c = ((k & 1) ? d.x_q : d.x_p) + 2 * t * L + a;
  } else {
    const int64_t q = (e - d.h_sh) / 2;
    r = c = d.x_vm + q;  // q = t N + n
  }
  (void)T;
  hrow[e] = (int32_t)r;
  hcol[e] = (int32_t)c;
}

// M row pointers and columns, one thread per row; columns ascending.
__global__ void k_pat_kkt(Dev d, int64_t *__restrict__ rowptr, int32_t *__restrict__ kcol) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= d.n) return;
  // Row starts come from the templates; columns are written directly.
  const int64_t T = d.T, L = d.L, N = d.N, G = d.G;
  (void)T;
  int64_t start = 0;
  int64_t k = 0;
  auto put = [&](int64_t col) { kcol[start + k] = (int32_t)col; ++k; };
  if (j < d.x_vm) {
    const int64_t t = j / N, nb = j - t * N;
    start = d.m_va + t * d.mb_va + d.mo_va[nb];
    for (int32_t q = d.nbr_ptr[nb]; q < d.nbr_ptr[nb + 1]; ++q)
      if (d.nbr_bus[q] < nb) put(t * N + d.nbr_bus[q]);
    put(j);
  } else if (j < d.x_pg) {
    const int64_t tn = j - d.x_vm, t = tn / N, nb = tn - t * N;
    start = d.m_vm + t * d.mb_vm + d.mo_vm[nb];
    const int32_t q0 = d.nbr_ptr[nb], q1 = d.nbr_ptr[nb + 1];
    if (q1 > q0) {
      bool self_done = false;
      for (int32_t q = q0; q < q1; ++q) {
        const int64_t o = d.nbr_bus[q];
        if (!self_done && o > nb) { put(t * N + nb); self_done = true; }
        put(t * N + o);
      }
      if (!self_done) put(t * N + nb);
    }
    for (int32_t q = q0; q < q1; ++q)
      if (d.nbr_bus[q] < nb) put(d.x_vm + t * N + d.nbr_bus[q]);
    put(j);
  } else if (j < d.x_qg) {
    const int64_t tg = j - d.x_pg, t = tg / G, g = tg - t * G, nb = d.gen_bus[g];
    start = d.m_pg + (t == 0 ? (int64_t)d.mo_pg0[g] : d.mb_pg0 + (t - 1) * d.mb_pg1 + d.mo_pg1[g]);
    put(d.x_vm + t * N + nb);
    if (t >= 1) put(d.x_pg + (t - 1) * G + g);
    for (int32_t q = d.bgen_ptr[nb]; q < d.bgen_ptr[nb] + d.gen_rank[g]; ++q) put(d.x_pg + t * G + d.bgen_idx[q]);
    put(j);
  } else if (j < d.x_p) {
    const int64_t tg = j - d.x_qg, t = tg / G, g = tg - t * G, nb = d.gen_bus[g];
    start = d.m_qg + (t == 0 ? (int64_t)d.mo_qg[g] : d.mb_qg + (t - 1) * d.mb_qg1 + d.mo_qg1[g]);
    put(d.x_vm + t * N + nb);
    if (d.qramp && t >= 1) put(d.x_qg + (t - 1) * G + g);
    for (int32_t q = d.bgen_ptr[nb]; q < d.bgen_ptr[nb] + d.gen_rank[g]; ++q) put(d.x_qg + t * G + d.bgen_idx[q]);
    put(j);
  } else {
    const bool isP = j < d.x_q;
    const int64_t ta = j - (isP ? d.x_p : d.x_q), t = ta / (2 * L), a = ta - t * 2 * L;
    const int64_t l = a < L ? a : a - L;
    const int64_t f = d.br_f[l], to = d.br_t[l], nb = a < L ? f : to;
    const int64_t lo = f < to ? f : to, hi = f < to ? to : f;
    start = isP ? d.m_p + t * d.mb_p + d.mo_p[a] : d.m_q + t * d.mb_q + d.mo_q[a];
    put(t * N + lo);
    put(t * N + hi);
    put(d.x_vm + t * N + lo);
    put(d.x_vm + t * N + hi);
    for (int32_t q = d.bgen_ptr[nb]; q < d.bgen_ptr[nb + 1]; ++q) put((isP ? d.x_pg : d.x_qg) + t * G + d.bgen_idx[q]);
    if (!isP) put(d.x_p + 2 * t * L + a);
    for (int32_t q = d.barc_ptr[nb]; q < d.barc_ptr[nb] + d.arc_rank[a]; ++q)
      put((isP ? d.x_p : d.x_q) + 2 * t * L + d.barc_idx[q]);
    put(j);
  }
  rowptr[j] = start;
  if (j == d.n - 1) rowptr[d.n] = start + k;
}

__global__ void k_bounds(Dev d, double *__restrict__ xl, double *__restrict__ xu, double *__restrict__ gl,
                         double *__restrict__ gu, const double *vmin, const double *vmax, const double *pmin,
                         const double *pmax, const double *qmin, const double *qmax, const double *angmin,
                         const double *angmax, const double *ramp, const double *qramp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = d.N, G = d.G, L = d.L, T = d.T;
  if (i < d.n) {
    double lo = -INFINITY, hi = INFINITY;
    if (i >= d.x_vm && i < d.x_pg) { const int64_t nb = (i - d.x_vm) % N; lo = vmin[nb]; hi = vmax[nb]; }
    else if (i >= d.x_pg && i < d.x_qg) { const int64_t g = (i - d.x_pg) % G; lo = pmin[g]; hi = pmax[g]; }
    else if (i >= d.x_qg && i < d.x_p) { const int64_t g = (i - d.x_qg) % G; lo = qmin[g]; hi = qmax[g]; }
    xl[i] = lo;
    xu[i] = hi;
  }
  if (i < d.m) {
    double lo = 0.0, hi = 0.0;
    const int64_t TL = T * L;
    if (i >= T && i < T + 7 * TL) {
      const int k = (int)((i - T) / TL) + 1;
      const int64_t l = ((i - T) - (k - 1) * TL) % L;
      if (k == 5) { lo = angmin[l]; hi = angmax[l]; }
      if (k == 6 || k == 7) { lo = -INFINITY; hi = 0.0; }
    } else if (d.qramp && i >= d.c_k11) {
      const int64_t g = (i - d.c_k11) % G;
      lo = -qramp[g];
      hi = qramp[g];
    } else if (i >= d.c_k10) {
      const int64_t g = (i - d.c_k10) % G;
      lo = -ramp[g];
      hi = ramp[g];
    }
    gl[i] = lo;
    gu[i] = hi;
  }
}

unsigned grid_for(int64_t count) { return (unsigned)((count + kBlock - 1) / kBlock); }

}  // namespace

cudaError_t launch_patterns(const Dev &d, int32_t *jrow, int32_t *jcol, int32_t *hrow, int32_t *hcol,
                            int64_t *krowptr, int32_t *kcol, double *xl, double *xu, double *gl, double *gu,
                            const double *vmin, const double *vmax, const double *pmin, const double *pmax,
                            const double *qmin, const double *qmax, const double *angmin, const double *angmax,
                            const double *ramp, const double *qramp, cudaStream_t s) {
  if (d.m > 0) k_pat_jac<<<grid_for(d.m), kBlock, 0, s>>>(d, jrow, jcol);
  if (d.nnz_hess > 0) k_pat_hess<<<grid_for(d.nnz_hess), kBlock, 0, s>>>(d, hrow, hcol);
  if (d.n > 0) k_pat_kkt<<<grid_for(d.n), kBlock, 0, s>>>(d, krowptr, kcol);
  const int64_t nm = d.n > d.m ? d.n : d.m;
  k_bounds<<<grid_for(nm), kBlock, 0, s>>>(d, xl, xu, gl, gu, vmin, vmax, pmin, pmax, qmin, qmax, angmin, angmax,
                                          ramp, qramp);
  return cudaGetLastError();
}

}  // namespace mpopf

using namespace mpopf;

namespace {

template <class T>
T *dev_upload(mpopf_handle *h, const std::vector<T> &v, cudaError_t *err) {
  if (*err != cudaSuccess) return nullptr;
  void *p = nullptr;
  const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
  if (h->nblocks >= kMaxBlocks) { *err = cudaErrorMemoryAllocation; return nullptr; }
  *err = cudaMalloc(&p, bytes);
  if (*err != cudaSuccess) return nullptr;
  h->blocks[h->nblocks++] = p;
  if (!v.empty()) *err = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return static_cast<T *>(p);
}

template <class T>
T *dev_alloc(mpopf_handle *h, int64_t count, cudaError_t *err) {
  if (*err != cudaSuccess) return nullptr;
  void *p = nullptr;
  if (h->nblocks >= kMaxBlocks) { *err = cudaErrorMemoryAllocation; return nullptr; }
  *err = cudaMalloc(&p, std::max<int64_t>(count, 1) * sizeof(T));
  if (*err != cudaSuccess) return nullptr;
  h->blocks[h->nblocks++] = p;
  return static_cast<T *>(p);
}

void fork_destroy(mpopf_handle *h) {
  if (h->fork.ev_join) cudaEventDestroy(h->fork.ev_join);
  if (h->fork.ev_fork) cudaEventDestroy(h->fork.ev_fork);
  if (h->fork.side) cudaStreamDestroy(h->fork.side);
  for (cudaEvent_t e : h->fork.ev_chunk)
    if (e) cudaEventDestroy(e);
  if (h->fork.ev_bus) cudaEventDestroy(h->fork.ev_bus);
  if (h->fork.bus) cudaStreamDestroy(h->fork.bus);
  h->fork = Fork();
}

void free_blocks(mpopf_handle *h) {
  for (int i = 0; i < h->nblocks; ++i) cudaFree(h->blocks[i]);
  h->nblocks = 0;
  if (h->stage) cudaFree(h->stage);
  h->stage = nullptr;
  if (h->pts) cudaFree(h->pts);
  h->pts = nullptr;
  h->pts_bytes = 0;
}

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

}  // namespace

namespace {
// Everything setup computes on the host for a network over T periods:
// validated sizes, per-branch constants, adjacency, incidence slots and the
// per-period templates of the J and M patterns (period-invariant).
struct HostModel {
  int64_t N, L, G, D, T, n, m;
  bool qramp;
  std::vector<double> bc, m2gs, p2bs, mgs, bsv;
  std::vector<uint8_t> sym;
  std::vector<int32_t> bgen_ptr, bgen_idx, barc_ptr, barc_idx, bload_ptr, bload_idx, gen_rank, arc_rank;
  std::vector<int32_t> bus_order, inc_ptr, inc_code, nbr_ptr, nbr_bus, nbr_grp, grp_code, bus_nd, bus_ndlt;
  std::vector<int32_t> br_slot, slot_info, slot_next, arc_perm, jk8_off;
  std::vector<int32_t> mo_va, mo_vm, mo_pg0, mo_pg1, mo_qg, mo_qg1, mo_p, mo_q;
  int64_t jk8_per, mb_va, mb_vm, mb_pg0, mb_pg1, mb_qg, mb_qg1, mb_p, mb_q;
};

// Validation and the host model (no device work).  `who` prefixes messages.
int host_model(const mpopf_network *net, int64_t n_periods, const char *who, HostModel *out) {
  HostModel &hm = *out;
  if (!net) return fail(MPOPF_ERR_ARG, std::string(who) + ": NULL network");
  const int64_t N = net->n_bus, L = net->n_branch, G = net->n_gen, D = net->n_load, T = n_periods;
  if (N < 1 || L < 0 || G < 0 || D < 0) return fail(MPOPF_ERR_ARG, std::string(who) + ": need n_bus >= 1 and counts >= 0");
  if (T < 1) return fail(MPOPF_ERR_ARG, std::string(who) + ": need n_periods >= 1");
  if (net->ref_bus < 0 || net->ref_bus >= N) return fail(MPOPF_ERR_ARG, std::string(who) + ": ref_bus out of range");
  // Sizes first (before touching any array), so oversized problems fail cleanly.
  const int64_t n = T * (2 * N + 2 * G + 4 * L);
  const bool qramp = G > 0 && net->gen_qramp != nullptr;
  const int64_t m = T * (1 + 7 * L + 2 * N) + G * (T - 1) * (qramp ? 2 : 1);
  if (n >= ((int64_t)1 << 31) || m >= ((int64_t)1 << 31) || T * L >= ((int64_t)1 << 31))
    return fail(MPOPF_ERR_SIZE, std::string(who) + ": n or m >= 2^31 (32-bit pattern indices)");
  if (N > 0 && (!net->bus_gs || !net->bus_bs || !net->bus_vmin || !net->bus_vmax))
    return fail(MPOPF_ERR_ARG, std::string(who) + ": NULL bus array");
  if (L > 0 && (!net->br_f || !net->br_t || !net->br_r || !net->br_x || !net->br_b || !net->br_tap ||
                !net->br_shift || !net->br_smax || !net->br_angmin || !net->br_angmax))
    return fail(MPOPF_ERR_ARG, std::string(who) + ": NULL branch array");
  if (G > 0 && (!net->gen_bus || !net->gen_c2 || !net->gen_c1 || !net->gen_c0 || !net->gen_pmin ||
                !net->gen_pmax || !net->gen_qmin || !net->gen_qmax || !net->gen_ramp))
    return fail(MPOPF_ERR_ARG, std::string(who) + ": NULL generator array");
  if (D > 0 && !net->load_bus) return fail(MPOPF_ERR_ARG, std::string(who) + ": NULL load array");
  for (int64_t l = 0; l < L; ++l) {
    const int32_t f = net->br_f[l], t = net->br_t[l];
    if (f < 0 || f >= N || t < 0 || t >= N) return fail(MPOPF_ERR_ARG, std::string(who) + ": branch end out of range");
    if (f == t) return fail(MPOPF_ERR_ARG, std::string(who) + ": self-loop branch");
    const double r = net->br_r[l], x = net->br_x[l];
    if (!(r * r + x * x > 0.0)) return fail(MPOPF_ERR_ARG, std::string(who) + ": branch with r = x = 0");
    if (!(net->br_tap[l] != 0.0) || !std::isfinite(net->br_tap[l]))
      return fail(MPOPF_ERR_ARG, std::string(who) + ": branch tap must be finite and nonzero");
  }
  for (int64_t g = 0; g < G; ++g)
    if (net->gen_bus[g] < 0 || net->gen_bus[g] >= N) return fail(MPOPF_ERR_ARG, std::string(who) + ": generator bus out of range");
  if (qramp)
    for (int64_t g = 0; g < G; ++g)
      if (!(net->gen_qramp[g] >= 0.0)) return fail(MPOPF_ERR_ARG, std::string(who) + ": reactive ramp limit must be >= 0");
  for (int64_t k = 0; k < D; ++k)
    if (net->load_bus[k] < 0 || net->load_bus[k] >= N) return fail(MPOPF_ERR_ARG, std::string(who) + ": load bus out of range");

  auto &bc = hm.bc; auto &sym = hm.sym;
  auto &m2gs = hm.m2gs; auto &p2bs = hm.p2bs; auto &mgs = hm.mgs; auto &bsv = hm.bsv;
  auto &bgen_ptr = hm.bgen_ptr; auto &bgen_idx = hm.bgen_idx; auto &barc_ptr = hm.barc_ptr;
  auto &barc_idx = hm.barc_idx; auto &bload_ptr = hm.bload_ptr; auto &bload_idx = hm.bload_idx;
  auto &gen_rank = hm.gen_rank; auto &arc_rank = hm.arc_rank; auto &bus_order = hm.bus_order;
  auto &inc_ptr = hm.inc_ptr; auto &inc_code = hm.inc_code; auto &nbr_ptr = hm.nbr_ptr; auto &nbr_bus = hm.nbr_bus;
  auto &nbr_grp = hm.nbr_grp; auto &grp_code = hm.grp_code; auto &bus_nd = hm.bus_nd; auto &bus_ndlt = hm.bus_ndlt;
  auto &br_slot = hm.br_slot; auto &slot_info = hm.slot_info; auto &slot_next = hm.slot_next;
  auto &arc_perm = hm.arc_perm; auto &jk8_off = hm.jk8_off; auto &jk8_per = hm.jk8_per;
  auto &mo_va = hm.mo_va; auto &mo_vm = hm.mo_vm; auto &mo_pg0 = hm.mo_pg0; auto &mo_pg1 = hm.mo_pg1;
  auto &mo_qg = hm.mo_qg; auto &mo_qg1 = hm.mo_qg1; auto &mo_p = hm.mo_p; auto &mo_q = hm.mo_q;
  auto &mb_va = hm.mb_va; auto &mb_vm = hm.mb_vm; auto &mb_pg0 = hm.mb_pg0; auto &mb_pg1 = hm.mb_pg1;
  auto &mb_qg = hm.mb_qg; auto &mb_qg1 = hm.mb_qg1; auto &mb_p = hm.mb_p; auto &mb_q = hm.mb_q;
  // ---- pi-model terms (textbook: y = 1/(r + jx), Y_ff = (y + jb/2)/tau^2,
  // Y_ft = -y/(tau e^{-j phi}), Y_tf = -y/(tau e^{j phi}), Y_tt = y + jb/2) ----
  bc.assign((size_t)BC_COUNT * L, 0.0);
  sym.assign(L, 0);
  for (int64_t l = 0; l < L; ++l) {
    const double r = net->br_r[l], x = net->br_x[l], chg = net->br_b[l];
    const double den = r * r + x * x;
    const double g = r / den;
    const double b = -x / den;
    const double tau = net->br_tap[l], tau2 = tau * tau;
    const double cph = std::cos(net->br_shift[l]), sph = std::sin(net->br_shift[l]);
    const double gff = g / tau2, bff = (b + 0.5 * chg) / tau2;
    const double gft = -(g * cph - b * sph) / tau, bft = -(g * sph + b * cph) / tau;
    const double gtf = -(g * cph + b * sph) / tau, btf = -(b * cph - g * sph) / tau;
    const double gtt = g, btt = b + 0.5 * chg;
    const double vals[BC_COUNT] = {gff, bff, gft, bft, gtf, btf, gtt, btt, 2.0 * gff, 2.0 * bff, 2.0 * gtt,
                                   2.0 * btt, net->br_smax[l] * net->br_smax[l]};
    for (int k = 0; k < BC_COUNT; ++k) bc[(size_t)k * L + l] = vals[k];
    sym[l] = (std::memcmp(&gtf, &gft, 8) == 0 && std::memcmp(&btf, &bft, 8) == 0) ? 1 : 0;
  }
  m2gs.assign(N, 0.0); p2bs.assign(N, 0.0); mgs.assign(N, 0.0); bsv.assign(N, 0.0);
  for (int64_t i = 0; i < N; ++i) {
    m2gs[i] = -(2.0 * net->bus_gs[i]);
    p2bs[i] = 2.0 * net->bus_bs[i];
    mgs[i] = -net->bus_gs[i];
    bsv[i] = net->bus_bs[i];
  }

  // ---- adjacency ----
  auto csr = [&](int64_t nitems, auto key, std::vector<int32_t> *ptr, std::vector<int32_t> *idx) {
    ptr->assign(N + 1, 0);
    for (int64_t e = 0; e < nitems; ++e) (*ptr)[key(e) + 1]++;
    for (int64_t i = 0; i < N; ++i) (*ptr)[i + 1] += (*ptr)[i];
    idx->assign(nitems, 0);
    std::vector<int32_t> fill(ptr->begin(), ptr->end() - 1);
    for (int64_t e = 0; e < nitems; ++e) (*idx)[fill[key(e)]++] = (int32_t)e;  // ascending e
  };
  csr(G, [&](int64_t g) { return (int64_t)net->gen_bus[g]; }, &bgen_ptr, &bgen_idx);
  csr(2 * L, [&](int64_t a) { return (int64_t)(a < L ? net->br_f[a] : net->br_t[a - L]); }, &barc_ptr, &barc_idx);
  csr(D, [&](int64_t k) { return (int64_t)net->load_bus[k]; }, &bload_ptr, &bload_idx);
  gen_rank.assign(G, 0); arc_rank.assign(2 * L, 0);
  for (int64_t i = 0; i < N; ++i) {
    for (int32_t q = bgen_ptr[i]; q < bgen_ptr[i + 1]; ++q) gen_rank[bgen_idx[q]] = q - bgen_ptr[i];
    for (int32_t q = barc_ptr[i]; q < barc_ptr[i + 1]; ++q) arc_rank[barc_idx[q]] = q - barc_ptr[i];
  }
  // incident branches by branch index (code 2l + end)
  std::vector<std::vector<int32_t>> inc(N);
  for (int64_t l = 0; l < L; ++l) {
    inc[net->br_f[l]].push_back((int32_t)(2 * l));
    inc[net->br_t[l]].push_back((int32_t)(2 * l + 1));
  }
  // Buses in the order the bus kernel processes them.  Natural order: sorting
  // by degree (equal loop trip counts in a warp) was measured slower because
  // the per-bus loads and stores then scatter.
  bus_order.assign(N, 0);
  for (int64_t i = 0; i < N; ++i) bus_order[i] = (int32_t)i;
  // Incidence slots numbered in that order (a warp's records are contiguous);
  // inc_ptr is indexed by position in bus_order, each bus's slots in branch order.
  inc_ptr.assign(N + 1, 0);
  inc_code.reserve(2 * L);
  std::vector<int32_t> slot_start(N);
  for (int64_t pos = 0; pos < N; ++pos) {
    const int32_t i = bus_order[pos];
    slot_start[i] = (int32_t)inc_code.size();
    inc_code.insert(inc_code.end(), inc[i].begin(), inc[i].end());  // ascending in l
    inc_ptr[pos + 1] = (int32_t)inc_code.size();
  }
  nbr_ptr.assign(N + 1, 0); bus_nd.assign(N, 0); bus_ndlt.assign(N, 0);
  for (int64_t i = 0; i < N; ++i) {
    std::vector<int32_t> &v = inc[i];
    std::vector<std::pair<int32_t, int32_t>> nb;  // (neighbour, code)
    for (int32_t code : v) {
      const int64_t l = code >> 1;
      nb.push_back({(code & 1) ? net->br_f[l] : net->br_t[l], code});
    }
    std::stable_sort(nb.begin(), nb.end(), [](auto &a, auto &b) { return a.first < b.first; });
    int32_t nd = 0, ndlt = 0;
    for (size_t k = 0; k < nb.size(); ++k) {
      if (k == 0 || nb[k].first != nb[k - 1].first) {
        nbr_bus.push_back(nb[k].first);
        nbr_grp.push_back((int32_t)grp_code.size());
        ++nd;
        if (nb[k].first < i) ++ndlt;
      }
      grp_code.push_back(nb[k].second);
    }
    nbr_ptr[i + 1] = (int32_t)nbr_bus.size();
    bus_nd[i] = nd;
    bus_ndlt[i] = ndlt;
  }
  nbr_grp.push_back((int32_t)grp_code.size());
  // Per slot: neighbour position and group links; per branch end: its slot;
  // per bus: its slots in ascending arc index (from ends, then to ends).
  br_slot.assign(2 * L, 0); slot_info.assign(2 * L, 0); slot_next.assign(2 * L, -1); arc_perm.assign(2 * L, 0);
  for (int64_t i = 0; i < N; ++i) {
    std::vector<int32_t> nbs;  // distinct neighbours ascending
    for (int32_t q = nbr_ptr[i]; q < nbr_ptr[i + 1]; ++q) nbs.push_back(nbr_bus[q]);
    std::vector<int32_t> last_of(nbs.size(), -1);
    const int32_t s0 = slot_start[i], s1 = s0 + (int32_t)inc[i].size();
    for (int32_t s = s0; s < s1; ++s) {
      const int32_t code = inc_code[s];
      const int64_t l = code >> 1;
      br_slot[(code & 1) * L + l] = s;
      const int32_t nb = (code & 1) ? net->br_f[l] : net->br_t[l];
      const int32_t k = (int32_t)(std::lower_bound(nbs.begin(), nbs.end(), nb) - nbs.begin());
      int32_t info = k;
      if (last_of[k] < 0) info |= 1 << 30;  // leader: first branch to nb in branch order
      else slot_next[last_of[k]] = s;
      if (nb < i) info |= 1 << 29;
      last_of[k] = s;
      slot_info[s] = info;
    }
    int32_t k = s0;
    for (int pass = 0; pass < 2; ++pass)
      for (int32_t q = s0; q < s1; ++q)
        if ((inc_code[q] & 1) == pass) arc_perm[k++] = q;
  }

  // ---- templates ----
  jk8_off.assign(N, 0);
  int64_t acc = 0;
  for (int64_t i = 0; i < N; ++i) {
    jk8_off[i] = (int32_t)acc;
    acc += 1 + (bgen_ptr[i + 1] - bgen_ptr[i]) + (barc_ptr[i + 1] - barc_ptr[i]);
  }
  jk8_per = acc;  // = N + G + 2L
  auto prefix = [](const std::vector<int64_t> &len, std::vector<int32_t> *off) {
    off->assign(len.size(), 0);
    int64_t s = 0;
    for (size_t k = 0; k < len.size(); ++k) { (*off)[k] = (int32_t)s; s += len[k]; }
    return s;
  };
  std::vector<int64_t> len_va(N), len_vm(N), len_pg0(G), len_pg1(G), len_qg(G), len_qg1(G), len_p(2 * L),
      len_q(2 * L);
  for (int64_t i = 0; i < N; ++i) {
    len_va[i] = bus_ndlt[i] + 1;
    len_vm[i] = (bus_nd[i] > 0 ? bus_nd[i] + 1 : 0) + bus_ndlt[i] + 1;
  }
  for (int64_t g = 0; g < G; ++g) {
    len_pg0[g] = 1 + gen_rank[g] + 1;
    len_pg1[g] = 2 + gen_rank[g] + 1;
    len_qg[g] = 1 + gen_rank[g] + 1;
    len_qg1[g] = (qramp ? 2 : 1) + gen_rank[g] + 1;
  }
  for (int64_t a = 0; a < 2 * L; ++a) {
    const int64_t bus = a < L ? net->br_f[a] : net->br_t[a - L];
    const int64_t kb = bgen_ptr[bus + 1] - bgen_ptr[bus];
    len_p[a] = 4 + kb + arc_rank[a] + 1;
    len_q[a] = 4 + kb + 1 + arc_rank[a] + 1;
  }
  mb_va = prefix(len_va, &mo_va); mb_vm = prefix(len_vm, &mo_vm);
  mb_pg0 = prefix(len_pg0, &mo_pg0); mb_pg1 = prefix(len_pg1, &mo_pg1);
  mb_qg = prefix(len_qg, &mo_qg); mb_qg1 = prefix(len_qg1, &mo_qg1);
  mb_p = prefix(len_p, &mo_p); mb_q = prefix(len_q, &mo_q);
  const int64_t big = (int64_t)1 << 31;
  if (mb_vm >= big || mb_p >= big || mb_q >= big || jk8_per * 1 >= big)
    return fail(MPOPF_ERR_SIZE, std::string(who) + ": one period of M exceeds 32-bit offsets");

  hm.N = N; hm.L = L; hm.G = G; hm.D = D; hm.T = T; hm.n = n; hm.m = m; hm.qramp = qramp;
  return MPOPF_OK;
}

// Offsets of every variable, row, J, W and M block of a T-period layout, from
// d.N, d.L, d.G, d.qramp, d.jk8_per and the per-period M block sizes d.mb_*.
void set_offsets(Dev &d, int64_t T) {
  const int64_t N = d.N, L = d.L, G = d.G;
  d.T = (int32_t)T;
  d.n = T * (2 * N + 2 * G + 4 * L);
  d.m = T * (1 + 7 * L + 2 * N) + G * (T - 1) * (d.qramp ? 2 : 1);
  d.x_vm = T * N; d.x_pg = 2 * T * N; d.x_qg = 2 * T * N + T * G; d.x_p = 2 * T * N + 2 * T * G;
  d.x_q = d.x_p + 2 * T * L;
  d.c_k8 = T + 7 * T * L; d.c_k9 = d.c_k8 + T * N; d.c_k10 = d.c_k9 + T * N; d.c_k11 = d.c_k10 + (T - 1) * G;
  d.j_k5 = T + 20 * T * L; d.j_k6 = d.j_k5 + 2 * T * L; d.j_k7 = d.j_k6 + 2 * T * L; d.j_k8 = d.j_k7 + 2 * T * L;
  d.j_k9 = d.j_k8 + T * d.jk8_per; d.j_k10 = d.j_k9 + T * d.jk8_per;
  d.j_k11 = d.j_k10 + 2 * (T - 1) * G;
  d.nnz_jac = d.j_k11 + (d.qramp ? 2 * (T - 1) * G : 0);
  d.h_br = T * G; d.h_th = d.h_br + 10 * T * L; d.h_sh = d.h_th + 4 * T * L; d.nnz_hess = d.h_sh + 2 * T * N;
  d.m_va = 0;
  d.m_vm = d.m_va + T * d.mb_va;
  d.m_pg = d.m_vm + T * d.mb_vm;
  d.m_qg = d.m_pg + d.mb_pg0 + (T - 1) * d.mb_pg1;
  d.m_p = d.m_qg + d.mb_qg + (T - 1) * d.mb_qg1;
  d.m_q = d.m_p + T * d.mb_p;
  d.nnz_kkt = d.m_q + T * d.mb_q;
  d.w0 = 0;
  d.w1 = (int32_t)T;
}

// Template sizes of a host model into a device descriptor.
void set_templates(Dev &d, const HostModel &hm) {
  d.N = (int32_t)hm.N; d.L = (int32_t)hm.L; d.G = (int32_t)hm.G; d.D = (int32_t)hm.D;
  d.qramp = hm.qramp ? 1 : 0;
  d.jk8_per = hm.jk8_per;
  d.mb_va = hm.mb_va; d.mb_vm = hm.mb_vm; d.mb_pg0 = hm.mb_pg0; d.mb_pg1 = hm.mb_pg1; d.mb_qg = hm.mb_qg;
  d.mb_qg1 = hm.mb_qg1; d.mb_p = hm.mb_p; d.mb_q = hm.mb_q;
}

}  // namespace

namespace {
// The handle of a T-period model (mpopf_setup; a period shard's local model).
int setup_model(const mpopf_network *net, int32_t n_periods, const double *pd, const double *qd, const char *who,
                mpopf_handle **out, mpopf_pattern *pat) {
  if (!out) return fail(MPOPF_ERR_ARG, std::string(who) + ": NULL output handle");
  *out = nullptr;
  HostModel hm;
  const int rc = host_model(net, n_periods, who, &hm);
  if (rc != MPOPF_OK) return rc;
  const int64_t N = hm.N, L = hm.L, G = hm.G, D = hm.D, T = hm.T, n = hm.n, m = hm.m;
  const bool qramp = hm.qramp;
  if (D > 0 && (!pd || !qd)) return fail(MPOPF_ERR_ARG, std::string(who) + ": NULL load array");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string(who) + ": no CUDA device");
  }

  const auto &bc = hm.bc; const auto &sym = hm.sym;
  const auto &m2gs = hm.m2gs; const auto &p2bs = hm.p2bs; const auto &mgs = hm.mgs; const auto &bsv = hm.bsv;
  const auto &bgen_ptr = hm.bgen_ptr; const auto &bgen_idx = hm.bgen_idx; const auto &barc_ptr = hm.barc_ptr;
  const auto &barc_idx = hm.barc_idx; const auto &bload_ptr = hm.bload_ptr; const auto &bload_idx = hm.bload_idx;
  const auto &gen_rank = hm.gen_rank; const auto &arc_rank = hm.arc_rank; const auto &bus_order = hm.bus_order;
  const auto &inc_ptr = hm.inc_ptr; const auto &inc_code = hm.inc_code; const auto &nbr_ptr = hm.nbr_ptr;
  const auto &nbr_bus = hm.nbr_bus; const auto &nbr_grp = hm.nbr_grp; const auto &grp_code = hm.grp_code;
  const auto &bus_nd = hm.bus_nd; const auto &bus_ndlt = hm.bus_ndlt; const auto &br_slot = hm.br_slot;
  const auto &slot_info = hm.slot_info; const auto &slot_next = hm.slot_next; const auto &arc_perm = hm.arc_perm;
  const auto &jk8_off = hm.jk8_off;
  const auto &mo_va = hm.mo_va; const auto &mo_vm = hm.mo_vm; const auto &mo_pg0 = hm.mo_pg0;
  const auto &mo_pg1 = hm.mo_pg1; const auto &mo_qg = hm.mo_qg; const auto &mo_qg1 = hm.mo_qg1;
  const auto &mo_p = hm.mo_p; const auto &mo_q = hm.mo_q;
  mpopf_handle *h = new mpopf_handle();
  std::memset(h, 0, sizeof(*h));
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string(who) + ": no current CUDA device");
  }
  Dev &d = h->d;
  set_templates(d, hm);
  set_offsets(d, T);
  d.ref = net->ref_bus;

  cudaError_t err = cudaSuccess;
  std::vector<int32_t> brf(net->br_f, net->br_f + L), brt(net->br_t, net->br_t + L);
  d.br_f = dev_upload(h, brf, &err);
  d.br_t = dev_upload(h, brt, &err);
  d.bc = dev_upload(h, bc, &err);
  d.br_sym = dev_upload(h, sym, &err);
  d.all_sym = std::all_of(sym.begin(), sym.end(), [](uint8_t v) { return v != 0; }) ? 1 : 0;
  d.bus_m2gs = dev_upload(h, m2gs, &err);
  d.bus_p2bs = dev_upload(h, p2bs, &err);
  d.bus_mgs = dev_upload(h, mgs, &err);
  d.bus_bs = dev_upload(h, bsv, &err);
  d.bgen_ptr = dev_upload(h, bgen_ptr, &err); d.bgen_idx = dev_upload(h, bgen_idx, &err);
  d.barc_ptr = dev_upload(h, barc_ptr, &err); d.barc_idx = dev_upload(h, barc_idx, &err);
  d.bload_ptr = dev_upload(h, bload_ptr, &err); d.bload_idx = dev_upload(h, bload_idx, &err);
  d.inc_ptr = dev_upload(h, inc_ptr, &err); d.inc_code = dev_upload(h, inc_code, &err);
  d.nbr_ptr = dev_upload(h, nbr_ptr, &err); d.nbr_bus = dev_upload(h, nbr_bus, &err);
  d.nbr_grp = dev_upload(h, nbr_grp, &err); d.grp_code = dev_upload(h, grp_code, &err);
  d.bus_nd = dev_upload(h, bus_nd, &err); d.bus_ndlt = dev_upload(h, bus_ndlt, &err);
  std::vector<int32_t> gbus(net->gen_bus, net->gen_bus + G);
  d.gen_bus = dev_upload(h, gbus, &err);
  d.gen_rank = dev_upload(h, gen_rank, &err);
  std::vector<double> c2(net->gen_c2, net->gen_c2 + G), c1(net->gen_c1, net->gen_c1 + G),
      c0(net->gen_c0, net->gen_c0 + G), c2x2(G);
  for (int64_t g = 0; g < G; ++g) c2x2[g] = 2.0 * c2[g];
  d.gen_c2 = dev_upload(h, c2, &err); d.gen_c1 = dev_upload(h, c1, &err);
  d.gen_c0 = dev_upload(h, c0, &err); d.gen_c2x2 = dev_upload(h, c2x2, &err);
  d.arc_rank = dev_upload(h, arc_rank, &err);
  d.jk8_off = dev_upload(h, jk8_off, &err);
  d.mo_va = dev_upload(h, mo_va, &err); d.mo_vm = dev_upload(h, mo_vm, &err);
  d.mo_pg0 = dev_upload(h, mo_pg0, &err); d.mo_pg1 = dev_upload(h, mo_pg1, &err);
  d.mo_qg = dev_upload(h, mo_qg, &err); d.mo_qg1 = dev_upload(h, mo_qg1, &err); d.mo_p = dev_upload(h, mo_p, &err); d.mo_q = dev_upload(h, mo_q, &err);
  std::vector<double> vpd(pd ? pd : (const double *)nullptr, pd ? pd + T * D : (const double *)nullptr);
  std::vector<double> vqd(qd ? qd : (const double *)nullptr, qd ? qd + T * D : (const double *)nullptr);
  d.pd = dev_upload(h, vpd, &err);
  d.qd = dev_upload(h, vqd, &err);
  d.br_slot = dev_upload(h, br_slot, &err);
  d.bus_order = dev_upload(h, bus_order, &err);
  d.arc_perm = dev_upload(h, arc_perm, &err);
  d.slot_info = dev_upload(h, slot_info, &err);
  d.slot_next = dev_upload(h, slot_next, &err);
  {
    // the branch kernel's integers packed for 16-byte loads
    std::vector<int32_t> brp((size_t)4 * BRP_COUNT * L);
    for (int64_t l = 0; l < L; ++l) {
      const int32_t f = net->br_f[l], to = net->br_t[l];
      const int32_t q[BRP_COUNT][4] = {
          {f, to, br_slot[l], br_slot[L + l]},
          {mo_p[l], mo_p[L + l], mo_q[l], mo_q[L + l]},
          {arc_rank[l], arc_rank[L + l], bgen_ptr[f + 1] - bgen_ptr[f], bgen_ptr[to + 1] - bgen_ptr[to]}};
      for (int k = 0; k < BRP_COUNT; ++k)
        for (int e = 0; e < 4; ++e) brp[4 * ((size_t)k * L + l) + e] = q[k][e];
    }
    d.brp = reinterpret_cast<const int4 *>(dev_upload(h, brp, &err));
  }
  d.S = dev_alloc<double>(h, T * 2 * L * kRec, &err);
  d.bw = dev_alloc<double>(h, 2 * T * N, &err);
  d.fpart_n = (int32_t)std::max<int64_t>(1, (T * G + kBlock - 1) / kBlock);
  d.fpart = dev_alloc<double>(h, d.fpart_n, &err);
  // patterns and bounds
  mpopf_pattern &P = h->pat;
  int32_t *jrow = dev_alloc<int32_t>(h, d.nnz_jac, &err), *jcol = dev_alloc<int32_t>(h, d.nnz_jac, &err);
  int32_t *hrow = dev_alloc<int32_t>(h, d.nnz_hess, &err), *hcol = dev_alloc<int32_t>(h, d.nnz_hess, &err);
  int64_t *krp = dev_alloc<int64_t>(h, n + 1, &err);
  int32_t *kcol = dev_alloc<int32_t>(h, d.nnz_kkt, &err);
  double *xl = dev_alloc<double>(h, n, &err), *xu = dev_alloc<double>(h, n, &err);
  double *gl = dev_alloc<double>(h, m, &err), *gu = dev_alloc<double>(h, m, &err);
  h->work = dev_alloc<double>(h, m, &err);
  // temporary bound sources
  std::vector<double> tmp_src;
  auto cat = [&](const double *p, int64_t k) { if (k > 0) tmp_src.insert(tmp_src.end(), p, p + k); };
  cat(net->bus_vmin, N); cat(net->bus_vmax, N);
  if (G > 0) { cat(net->gen_pmin, G); cat(net->gen_pmax, G); cat(net->gen_qmin, G); cat(net->gen_qmax, G); cat(net->gen_ramp, G); }
  if (qramp) cat(net->gen_qramp, G);
  if (L > 0) { cat(net->br_angmin, L); cat(net->br_angmax, L); }
  double *src = dev_upload(h, tmp_src, &err);
  if (err != cudaSuccess) {
    const bool oom = err == cudaErrorMemoryAllocation;
    std::string msg = std::string(who) + ": " + cudaGetErrorString(err);
    free_blocks(h);
    delete h;
    cudaGetLastError();
    return fail(oom ? MPOPF_ERR_ALLOC : MPOPF_ERR_CUDA, msg);
  }
  const double *vmin = src, *vmax = src + N;
  const double *pmin = src + 2 * N, *pmax = pmin + G, *qmin = pmax + G, *qmax = qmin + G, *ramp = qmax + G;
  const double *qramp_src = qramp ? ramp + G : nullptr;
  const double *angmin = src + 2 * N + 5 * G + (qramp ? G : 0), *angmax = angmin + L;
  err = launch_patterns(d, jrow, jcol, hrow, hcol, krp, kcol, xl, xu, gl, gu, vmin, vmax, pmin, pmax, qmin, qmax,
                        angmin, angmax, ramp, qramp_src, 0);
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    std::string msg = std::string(who) + ": pattern expansion: " + cudaGetErrorString(err);
    free_blocks(h);
    delete h;
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, msg);
  }
  err = cudaStreamCreateWithFlags(&h->fork.side, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&h->fork.ev_fork, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&h->fork.ev_join, cudaEventDisableTiming);
  if (err == cudaSuccess) err = fork_bus_stream(&h->fork, false);
  h->fork.sms = device_sms(h->device);
  h->fork.flags = default_schedule_flags(d, h->fork.sms);  // the default launch schedule
  if (err != cudaSuccess) {
    std::string msg = std::string(who) + ": side stream: " + cudaGetErrorString(err);
    fork_destroy(h);
    free_blocks(h);
    delete h;
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, msg);
  }
  P.n = n; P.m = m; P.nnz_jac = d.nnz_jac; P.nnz_hess = d.nnz_hess; P.nnz_kkt = d.nnz_kkt;
  P.n_bus = d.N; P.n_branch = d.L; P.n_gen = d.G; P.n_load = d.D; P.n_periods = d.T;
  P.jac_row = jrow; P.jac_col = jcol; P.hess_row = hrow; P.hess_col = hcol;
  P.kkt_rowptr = krp; P.kkt_col = kcol; P.xl = xl; P.xu = xu; P.gl = gl; P.gu = gu;
  if (pat) *pat = P;
  *out = h;
  return MPOPF_OK;
}
}  // namespace

extern "C" {

const char *mpopf_last_error(void) { return g_err.c_str(); }

int mpopf_setup(const mpopf_network *net, int32_t n_periods, const double *pd, const double *qd, mpopf_handle **out,
                mpopf_pattern *pat) {
  return setup_model(net, n_periods, pd, qd, "mpopf_setup", out, pat);
}

// ---------------------------------------------------------------------------
// Period shards.  Only the ramp rows (Eq. 1k) couple periods, so the horizon
// splits into contiguous blocks of periods.  A shard owning [t0, t1) is the
// model of periods [t0 - h0, t1 + h1) (h0 = 1 if t0 > 0, h1 = 1 if t1 < T),
// evaluated on its owned periods only: every owned entry is then computed by
// exactly the arithmetic of the whole-horizon model.  The halo periods carry
// the two values an owned entry reads from a neighbour: pg (and qg with the
// reactive ramp) of period t0 - 1, read by the ramp rows at t0, and D of the
// ramp rows at t1, added last to the pg (qg) diagonals of M at t1 - 1.
// ---------------------------------------------------------------------------
int mpopf_shard_plan(const mpopf_network *net, int32_t n_periods, int32_t t0, int32_t t1, mpopf_shard_layout *plan) {
  if (!plan) return fail(MPOPF_ERR_ARG, "mpopf_shard_plan: NULL layout");
  if (!(n_periods >= 1 && t0 >= 0 && t1 > t0 && t1 <= n_periods))
    return fail(MPOPF_ERR_ARG, "mpopf_shard_plan: need 0 <= t0 < t1 <= n_periods");
  HostModel hm;
  const int rc = host_model(net, n_periods, "mpopf_shard_plan", &hm);
  if (rc != MPOPF_OK) return rc;
  const int64_t T = n_periods, N = hm.N, L = hm.L, G = hm.G;
  const int32_t h0 = t0 > 0 ? 1 : 0, h1 = t1 < T ? 1 : 0;
  const int64_t W = t1 - t0, Tl = W + h0 + h1;
  Dev g, l;
  std::memset(&g, 0, sizeof g);
  set_templates(g, hm);
  l = g;
  set_offsets(g, T);
  set_offsets(l, Tl);
  mpopf_shard_layout &P = *plan;
  std::memset(&P, 0, sizeof P);
  P.n_periods = (int32_t)T; P.t0 = t0; P.t1 = t1; P.local_periods = (int32_t)Tl;
  P.own0 = h0; P.own1 = (int32_t)(h0 + W);
  P.halo_len = (int32_t)G; P.halo_blocks = hm.qramp ? 2 : 1;
  P.n = l.n; P.m = l.m; P.nnz_jac = l.nnz_jac; P.nnz_hess = l.nnz_hess; P.nnz_kkt = l.nnz_kkt;
  const int64_t o0 = P.own0, o1 = P.own1;
  for (int b = 0; b < 2; ++b) {
    const bool on = b == 0 || hm.qramp;
    const int64_t xb = b == 0 ? l.x_pg : l.x_qg, rb = b == 0 ? l.c_k10 : l.c_k11;
    P.x_recv[b] = on && h0 ? xb + (o0 - 1) * G : -1;
    P.x_send[b] = on && h1 ? xb + (o1 - 1) * G : -1;
    P.d_recv[b] = on && h1 ? rb + (o1 - 1) * G : -1;  // ramp rows of local period o1
    P.d_send[b] = on && h0 ? rb + (o0 - 1) * G : -1;  // ramp rows of local period o0
  }
  auto add = [&](int32_t what, int64_t loc, int64_t glob, int64_t cnt) {
    if (cnt <= 0 || P.n_ranges >= MPOPF_SHARD_MAX_RANGES) return;
    P.ranges[P.n_ranges++] = mpopf_range{what, 0, loc, glob, cnt};
  };
  // variables: owned periods, and every local period (halos included)
  const int64_t cnt[6] = {N, N, G, G, 2 * L, 2 * L};
  const int64_t lx[6] = {0, l.x_vm, l.x_pg, l.x_qg, l.x_p, l.x_q}, gx[6] = {0, g.x_vm, g.x_pg, g.x_qg, g.x_p, g.x_q};
  for (int k = 0; k < 6; ++k) add(MPOPF_RANGE_X, lx[k] + o0 * cnt[k], gx[k] + t0 * cnt[k], W * cnt[k]);
  for (int k = 0; k < 6; ++k) add(MPOPF_RANGE_XALL, lx[k], gx[k] + (t0 - h0) * cnt[k], Tl * cnt[k]);
  // rows of the owned periods (a ramp row (t, g) belongs to period t >= 1)
  const int64_t ta = t0 > 1 ? t0 : 1, lta = ta - t0 + h0, nr = (t1 - ta) * G;
  add(MPOPF_RANGE_ROWS, o0, t0, W);
  for (int k = 1; k <= 7; ++k) add(MPOPF_RANGE_ROWS, Tl + (k - 1) * Tl * L + o0 * L, T + (k - 1) * T * L + t0 * L, W * L);
  add(MPOPF_RANGE_ROWS, l.c_k8 + o0 * N, g.c_k8 + t0 * N, W * N);
  add(MPOPF_RANGE_ROWS, l.c_k9 + o0 * N, g.c_k9 + t0 * N, W * N);
  add(MPOPF_RANGE_ROWS, l.c_k10 + (lta - 1) * G, g.c_k10 + (ta - 1) * G, nr);
  if (hm.qramp) add(MPOPF_RANGE_ROWS, l.c_k11 + (lta - 1) * G, g.c_k11 + (ta - 1) * G, nr);
  // J entries of those rows
  add(MPOPF_RANGE_JAC, o0, t0, W);
  for (int k = 1; k <= 4; ++k)
    add(MPOPF_RANGE_JAC, Tl + 5 * (k - 1) * Tl * L + o0 * 5 * L, T + 5 * (k - 1) * T * L + t0 * 5 * L, 5 * W * L);
  add(MPOPF_RANGE_JAC, l.j_k5 + o0 * 2 * L, g.j_k5 + t0 * 2 * L, 2 * W * L);
  add(MPOPF_RANGE_JAC, l.j_k6 + o0 * 2 * L, g.j_k6 + t0 * 2 * L, 2 * W * L);
  add(MPOPF_RANGE_JAC, l.j_k7 + o0 * 2 * L, g.j_k7 + t0 * 2 * L, 2 * W * L);
  add(MPOPF_RANGE_JAC, l.j_k8 + o0 * l.jk8_per, g.j_k8 + t0 * g.jk8_per, W * g.jk8_per);
  add(MPOPF_RANGE_JAC, l.j_k9 + o0 * l.jk8_per, g.j_k9 + t0 * g.jk8_per, W * g.jk8_per);
  add(MPOPF_RANGE_JAC, l.j_k10 + 2 * (lta - 1) * G, g.j_k10 + 2 * (ta - 1) * G, 2 * nr);
  if (hm.qramp) add(MPOPF_RANGE_JAC, l.j_k11 + 2 * (lta - 1) * G, g.j_k11 + 2 * (ta - 1) * G, 2 * nr);
  // W entries of the owned periods' elements
  add(MPOPF_RANGE_HESS, o0 * G, t0 * G, W * G);
  add(MPOPF_RANGE_HESS, l.h_br + o0 * 10 * L, g.h_br + t0 * 10 * L, 10 * W * L);
  add(MPOPF_RANGE_HESS, l.h_th + o0 * 4 * L, g.h_th + t0 * 4 * L, 4 * W * L);
  add(MPOPF_RANGE_HESS, l.h_sh + o0 * 2 * N, g.h_sh + t0 * 2 * N, 2 * W * N);
  // M values of the owned variables' rows (each kind's rows are contiguous)
  auto off1 = [](int64_t t, int64_t b0, int64_t b1) { return t == 0 ? 0 : b0 + (t - 1) * b1; };
  add(MPOPF_RANGE_KKT, l.m_va + o0 * l.mb_va, g.m_va + t0 * g.mb_va, W * g.mb_va);
  add(MPOPF_RANGE_KKT, l.m_vm + o0 * l.mb_vm, g.m_vm + t0 * g.mb_vm, W * g.mb_vm);
  const int64_t pg_l = off1(o1, l.mb_pg0, l.mb_pg1) - off1(o0, l.mb_pg0, l.mb_pg1);
  const int64_t pg_g = off1(t1, g.mb_pg0, g.mb_pg1) - off1(t0, g.mb_pg0, g.mb_pg1);
  const int64_t qg_l = off1(o1, l.mb_qg, l.mb_qg1) - off1(o0, l.mb_qg, l.mb_qg1);
  const int64_t qg_g = off1(t1, g.mb_qg, g.mb_qg1) - off1(t0, g.mb_qg, g.mb_qg1);
  if (pg_l != pg_g || qg_l != qg_g) return fail(MPOPF_ERR_ARG, "mpopf_shard_plan: inconsistent generator rows");
  add(MPOPF_RANGE_KKT, l.m_pg + off1(o0, l.mb_pg0, l.mb_pg1), g.m_pg + off1(t0, g.mb_pg0, g.mb_pg1), pg_g);
  add(MPOPF_RANGE_KKT, l.m_qg + off1(o0, l.mb_qg, l.mb_qg1), g.m_qg + off1(t0, g.mb_qg, g.mb_qg1), qg_g);
  add(MPOPF_RANGE_KKT, l.m_p + o0 * l.mb_p, g.m_p + t0 * g.mb_p, W * g.mb_p);
  add(MPOPF_RANGE_KKT, l.m_q + o0 * l.mb_q, g.m_q + t0 * g.mb_q, W * g.mb_q);
  return MPOPF_OK;
}

int mpopf_shard_setup(const mpopf_network *net, int32_t n_periods, int32_t t0, int32_t t1, const double *pd,
                      const double *qd, mpopf_handle **out, mpopf_pattern *pat) {
  if (!out) return fail(MPOPF_ERR_ARG, "mpopf_shard_setup: NULL output handle");
  *out = nullptr;
  mpopf_shard_layout plan;
  int rc = mpopf_shard_plan(net, n_periods, t0, t1, &plan);  // validates the whole-horizon model too
  if (rc != MPOPF_OK) return rc;
  const int64_t D = net->n_load, first = t0 - plan.own0;  // loads of periods [t0 - h0, t1 + h1)
  rc = setup_model(net, plan.local_periods, pd ? pd + first * D : nullptr, qd ? qd + first * D : nullptr,
                   "mpopf_shard_setup", out, pat);
  if (rc != MPOPF_OK) return rc;
  (*out)->d.w0 = plan.own0;
  (*out)->d.w1 = plan.own1;
  (*out)->fork.flags = default_schedule_flags((*out)->d, (*out)->fork.sms);  // sized by the owned periods
  return MPOPF_OK;
}


int mpopf_get_pattern(const mpopf_handle *h, mpopf_pattern *pat) {
  if (!h || !pat) return fail(MPOPF_ERR_ARG, "mpopf_get_pattern: NULL argument");
  *pat = h->pat;
  return MPOPF_OK;
}

int mpopf_set_loads(mpopf_handle *h, const double *d_pd, const double *d_qd, void *stream) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_set_loads: NULL handle");
  const size_t bytes = (size_t)h->d.T * h->d.D * sizeof(double);
  if (bytes == 0) return MPOPF_OK;
  if (!d_pd || !d_qd) return fail(MPOPF_ERR_ARG, "mpopf_set_loads: NULL load array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(const_cast<double *>(h->d.pd), d_pd, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(const_cast<double *>(h->d.qd), d_qd, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_set_loads: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

void mpopf_destroy(mpopf_handle *h) {
  if (!h) return;
  fork_destroy(h);
  hostpipe_destroy(h);
  kkt_solver_destroy(h);
  free_blocks(h);
  delete h;
}

}  // extern "C"
