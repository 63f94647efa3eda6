// Pipelined full sweep from host buffers (mpopf_sweep_host): the horizon in
// period windows, each window's inputs copied in on one stream, its branch and
// bus kernels on the caller's stream, its outputs copied out on a third stream,
// so the copies in both directions overlap each other and the kernels.  The
// kernels launched are exactly those of mpopf_sweep (launch_window per
// window, then launch_gen_obj), so the outputs equal the device sweep's.
#include <algorithm>
#include <cstring>
#include <string>

#include "mpopf_internal.cuh"

using namespace mpopf;

namespace {
int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

// Strided row-block copies between same-layout host and device arrays: height
// blocks of width doubles, pitch doubles apart, starting at offset.
struct Copier {
  cudaError_t err = cudaSuccess;
  bool ok() const { return err == cudaSuccess; }
  void check(cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  }
  void rows(double *dst, const double *src, int64_t off, int64_t pitch, int64_t width, int64_t height,
            cudaMemcpyKind kind, cudaStream_t st) {
    if (!ok() || width <= 0 || height <= 0) return;
    const size_t wb = (size_t)width * sizeof(double), pb = (size_t)pitch * sizeof(double);
    if (height == 1) {
      check(cudaMemcpyAsync(dst + off, src + off, wb, kind, st));
    } else if (pb <= (size_t)INT32_MAX) {
      check(cudaMemcpy2DAsync(dst + off, pb, src + off, pb, wb, (size_t)height, kind, st));
    } else {
      for (int64_t r = 0; r < height && ok(); ++r)
        check(cudaMemcpyAsync(dst + off + r * pitch, src + off + r * pitch, wb, kind, st));
    }
  }
};

int hostpipe_create(mpopf_handle *h) {
  HostPipe *p = new HostPipe();
  std::memset(p, 0, sizeof(*p));
  cudaError_t e = cudaStreamCreateWithFlags(&p->in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->gen, cudaEventDisableTiming);
  for (int k = 0; k < kHostWindows && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_c[k], cudaEventDisableTiming);
  }
  h->pipe = p;
  if (e != cudaSuccess) {
    hostpipe_destroy(h);
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_sweep_host: streams: ") + cudaGetErrorString(e));
  }
  return MPOPF_OK;
}
}  // namespace

void mpopf::hostpipe_destroy(mpopf_handle *h) {
  HostPipe *p = h->pipe;
  if (!p) return;
  if (p->in) cudaStreamDestroy(p->in);
  if (p->out) cudaStreamDestroy(p->out);
  if (p->start) cudaEventDestroy(p->start);
  if (p->gen) cudaEventDestroy(p->gen);
  for (int k = 0; k < kHostWindows; ++k) {
    if (p->ev_in[k]) cudaEventDestroy(p->ev_in[k]);
    if (p->ev_c[k]) cudaEventDestroy(p->ev_c[k]);
  }
  delete p;
  h->pipe = nullptr;
}

extern "C" {

int mpopf_sweep_host(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *sigma_x,
                     const double *dvec, double delta_w, double *f, double *grad, double *c, double *jv, double *hv,
                     double *kv, void *stream) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_sweep_host: NULL handle");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_sweep_host: not available on a period shard");
  if (!x || !lam || !sigma_x || !dvec || !f || !grad || !c || !jv || !hv || !kv)
    return fail(MPOPF_ERR_ARG, "mpopf_sweep_host: NULL buffer");
  const Dev &d = h->d;
  const size_t n = d.n, m = d.m;
  const size_t words = 2 * n + 2 * m + 1 + n + m + d.nnz_jac + d.nnz_hess + d.nnz_kkt;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!h->stage) {
    void *p = nullptr;
    const cudaError_t e = cudaMalloc(&p, words * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MPOPF_ERR_ALLOC, std::string("mpopf_sweep_host: staging: ") + cudaGetErrorString(e));
    }
    h->stage = static_cast<double *>(p);
    h->stage_bytes = words * sizeof(double);
  }
  if (!h->pipe) {
    const int rc = hostpipe_create(h);
    if (rc != MPOPF_OK) return rc;
  }
  HostPipe &P = *h->pipe;
  double *dx = h->stage, *dl = dx + n, *dsx = dl + m, *ddv = dsx + n;
  double *df = ddv + m, *dg = df + 1, *dc = dg + n, *dj = dc + m, *dh = dj + d.nnz_jac, *dk = dh + d.nnz_hess;
  const int64_t T = d.T, N = d.N, L = d.L, G = d.G, TL = T * L, TN = T * N, TG = T * G;
  const int64_t ramps = (d.qramp ? 2 : 1);
  const cudaMemcpyKind H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
  // Periods in windows: inputs of window k go in on P.in, its branch and bus
  // work runs on the caller's stream, its outputs come out on P.out, so the
  // copies in both directions and the kernels overlap.  The generator work and
  // the objective (whole horizon) and their outputs come last.  A period's
  // outputs are about 3.5 times its inputs, so the windows grow by 3 from a
  // short first one (about T / 84 periods: outputs start moving early, and each
  // window's inputs are in before the previous window's outputs are out) until
  // an even split of the rest is smaller; the last window takes what is left.
  int64_t wstart[kHostWindows + 1] = {0};
  int32_t nw = 0;
  for (int64_t size = std::max<int64_t>(1, T / 84); wstart[nw] < T; ++nw) {
    const int64_t left = T - wstart[nw], wl = kHostWindows - nw;  // windows left, this one included
    const int64_t take = wl == 1 ? left : std::min(size, (left + wl - 1) / wl);
    wstart[nw + 1] = wstart[nw] + take;
    size = 3 * take;
  }
  Copier cp;
  cp.check(cudaEventRecord(P.start, s));
  cp.check(cudaStreamWaitEvent(P.in, P.start, 0));
  cp.check(cudaStreamWaitEvent(P.out, P.start, 0));
  for (int32_t k = 0; k < nw && cp.ok(); ++k) {
    const int64_t t0 = wstart[k], t1 = wstart[k + 1], tw = t1 - t0;
    const int64_t r0 = std::max<int64_t>(t0, 1) - 1, r1 = t1 - 1;  // ramp rows (t - 1) G + g of these periods
    // inputs: x and Sigma_x by variable kind; lambda and D by row kind
    for (int v = 0; v < 2; ++v) {
      double *dst = v == 0 ? dx : dsx;
      const double *src = v == 0 ? x : sigma_x;
      cp.rows(dst, src, t0 * N, TN, tw * N, 2, H2D, P.in);                     // va, vm
      cp.rows(dst, src, d.x_pg + t0 * G, TG, tw * G, 2, H2D, P.in);           // pg, qg
      cp.rows(dst, src, d.x_p + 2 * t0 * L, 2 * TL, 2 * tw * L, 2, H2D, P.in);  // p, q
    }
    for (int v = 0; v < 2; ++v) {
      double *dst = v == 0 ? dl : ddv;
      const double *src = v == 0 ? lam : dvec;
      if (k == 0) cp.rows(dst, src, 0, 0, T, 1, H2D, P.in);                 // K0, all periods
      cp.rows(dst, src, T + t0 * L, TL, tw * L, 7, H2D, P.in);                // K1..K7
      cp.rows(dst, src, d.c_k8 + t0 * N, TN, tw * N, 2, H2D, P.in);          // K8, K9
      cp.rows(dst, src, d.c_k10 + r0 * G, (T - 1) * G, (r1 - r0) * G, ramps, H2D, P.in);  // K10 (K11)
    }
    cp.check(cudaEventRecord(P.ev_in[k], P.in));
    cp.check(cudaStreamWaitEvent(s, P.ev_in[k], 0));
    if (!cp.ok()) break;
    launch_window(d, (int32_t)t0, (int32_t)t1, dx, dl, dsx, ddv, delta_w, dg, dc, dj, dh, dk, s);
    cp.check(cudaGetLastError());
    cp.check(cudaEventRecord(P.ev_c[k], s));
    cp.check(cudaStreamWaitEvent(P.out, P.ev_c[k], 0));
    // outputs of these periods
    cp.rows(grad, dg, t0 * N, TN, tw * N, 2, D2H, P.out);                      // va, vm
    cp.rows(grad, dg, d.x_p + 2 * t0 * L, 2 * TL, 2 * tw * L, 2, D2H, P.out);  // p, q
    cp.rows(c, dc, T + t0 * L, TL, tw * L, 7, D2H, P.out);                     // K1..K7
    cp.rows(c, dc, d.c_k8 + t0 * N, TN, tw * N, 2, D2H, P.out);               // K8, K9
    cp.rows(jv, dj, T + 5 * t0 * L, 5 * TL, 5 * tw * L, 4, D2H, P.out);        // K1..K4
    cp.rows(jv, dj, d.j_k5 + 2 * t0 * L, 2 * TL, 2 * tw * L, 3, D2H, P.out);   // K5..K7
    cp.rows(jv, dj, d.j_k8 + t0 * d.jk8_per, T * d.jk8_per, tw * d.jk8_per, 2, D2H, P.out);  // K8, K9
    cp.rows(hv, dh, d.h_br + 10 * t0 * L, 0, 10 * tw * L, 1, D2H, P.out);      // branch blocks
    cp.rows(hv, dh, d.h_th + 4 * t0 * L, 0, 4 * tw * L, 1, D2H, P.out);        // thermal
    cp.rows(hv, dh, d.h_sh + 2 * t0 * N, 0, 2 * tw * N, 1, D2H, P.out);        // shunt
    cp.rows(kv, dk, d.m_va + t0 * d.mb_va, 0, tw * d.mb_va, 1, D2H, P.out);    // va rows
    cp.rows(kv, dk, d.m_vm + t0 * d.mb_vm, 0, tw * d.mb_vm, 1, D2H, P.out);    // vm rows
    cp.rows(kv, dk, d.m_p + t0 * d.mb_p, 0, tw * d.mb_p, 1, D2H, P.out);       // p rows
    cp.rows(kv, dk, d.m_q + t0 * d.mb_q, 0, tw * d.mb_q, 1, D2H, P.out);       // q rows
  }
  if (cp.ok()) {
    launch_gen_obj(d, dx, sigma, dsx, ddv, delta_w, df, dg, dc, dj, dh, dk, s);
    cp.check(cudaGetLastError());
    cp.check(cudaEventRecord(P.gen, s));
    cp.check(cudaStreamWaitEvent(P.out, P.gen, 0));
    cp.rows(f, df, 0, 0, 1, 1, D2H, P.out);
    cp.rows(c, dc, 0, 0, T, 1, D2H, P.out);                                    // K0 (T doubles: once)
    cp.rows(jv, dj, 0, 0, T, 1, D2H, P.out);                                   // K0
    cp.rows(grad, dg, d.x_pg, 0, 2 * TG, 1, D2H, P.out);                       // pg, qg
    cp.rows(c, dc, d.c_k10, 0, ramps * (T - 1) * G, 1, D2H, P.out);             // K10 (K11)
    cp.rows(jv, dj, d.j_k10, 0, d.nnz_jac - d.j_k10, 1, D2H, P.out);            // K10 (K11)
    cp.rows(hv, dh, 0, 0, TG, 1, D2H, P.out);                                  // objective
    cp.rows(kv, dk, d.m_pg, 0, d.m_p - d.m_pg, 1, D2H, P.out);                 // pg, qg rows
  }
  // wait for everything enqueued, also after an error
  const cudaError_t e1 = cudaStreamSynchronize(P.out);
  const cudaError_t e2 = cudaStreamSynchronize(P.in);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  cp.check(e1);
  cp.check(e2);
  cp.check(e3);
  if (!cp.ok()) return fail(MPOPF_ERR_CUDA, std::string("mpopf_sweep_host: ") + cudaGetErrorString(cp.err));
  return MPOPF_OK;
}

}  // extern "C"
