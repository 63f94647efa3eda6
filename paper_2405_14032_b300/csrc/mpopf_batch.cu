// Batched evaluation of many independent multi-period AC OPF instances of
// uneven size in one persistent launch, replayed as a CUDA graph, with a
// schedule chosen by measurement (autotuner).
//
// The work list holds CTA-sized tiles ("items") of every instance: all branch
// tiles, then generator tiles, then bus tiles, then one objective item per
// instance.  The schedule decides the instance order in the list (as given, or
// largest first), the tile size (1, 2 or 4 CTA-sized chunks per item) and the
// persistent grid (CTAs per SM).  Results do not depend on the schedule: each
// value is computed by the same sequence of operations whichever CTA runs it.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "mpopf_internal.cuh"

using namespace mpopf;

struct mpopf_batch {
  int32_t K = 0;
  int device = 0;
  std::vector<mpopf_handle *> hs;
  Dev *d_devs = nullptr;
  BatchIO *d_io = nullptr;
  BatchItem *d_items = nullptr;
  int32_t *d_need = nullptr;  // [2K]: branch items, generator items per instance
  int32_t *d_ctl = nullptr;   // [2 + 2K]
  int32_t n_items = 0;
  int32_t sched[3] = {0, 1, 0};  // order (0 given, 1 largest first), tile chunks, CTAs per SM (0 = max)
  int32_t grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void *args[7];
  int32_t K_arg = 0;
  bool io_set = false;
};

namespace {

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

int64_t work_of(const Dev &d) { return (int64_t)d.T * (d.L + d.N + d.G); }

// Build the item list for a schedule and upload it (synchronous, setup time).
cudaError_t build_items(mpopf_batch *b) {
  const int32_t K = b->K;
  std::vector<int32_t> order(K);
  std::iota(order.begin(), order.end(), 0);
  if (b->sched[0] == 1)
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t c) { return work_of(b->hs[a]->d) > work_of(b->hs[c]->d); });
  const int32_t chunk = kBlock * std::max(1, b->sched[1]);
  std::vector<BatchItem> items;
  std::vector<int32_t> need(2 * K, 0);
  auto add = [&](int32_t kind, int32_t k, int64_t units) {
    for (int64_t f = 0; f < units; f += chunk) {
      items.push_back(BatchItem{k, kind, (int32_t)f, (int32_t)std::min<int64_t>(chunk, units - f)});
      if (kind == ITEM_BRANCH) ++need[k];
      if (kind == ITEM_GEN) ++need[K + k];
    }
  };
  for (int32_t k : order) add(ITEM_BRANCH, k, (int64_t)b->hs[k]->d.T * b->hs[k]->d.L);
  for (int32_t k : order) add(ITEM_GEN, k, (int64_t)b->hs[k]->d.T * b->hs[k]->d.G);
  for (int32_t k : order) add(ITEM_BUS, k, (int64_t)b->hs[k]->d.T * b->hs[k]->d.N);
  for (int32_t k : order) items.push_back(BatchItem{k, ITEM_FSUM, 0, 1});
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  cudaError_t e = cudaMalloc(&b->d_items, items.size() * sizeof(BatchItem));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_need, need.data(), need.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  b->n_items = (int32_t)items.size();
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int per_sm = b->sched[2] > 0 ? std::min(b->sched[2], batch_max_ctas_per_sm()) : batch_max_ctas_per_sm();
  b->grid = std::max(1, std::min(sms * per_sm, b->n_items));
  return e;
}

// (Re)build the graph: reset the counters, then the persistent kernel.
cudaError_t build_graph(mpopf_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  if (e != cudaSuccess) return e;
  cudaMemsetParams mp = {};
  mp.dst = b->d_ctl;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = (size_t)(2 + 2 * b->K);
  mp.height = 1;
  mp.pitch = 0;
  cudaGraphNode_t nmem = nullptr, nker = nullptr;
  e = cudaGraphAddMemsetNode(&nmem, b->graph, nullptr, 0, &mp);
  if (e != cudaSuccess) return e;
  b->K_arg = b->K;
  b->args[0] = &b->d_devs;
  b->args[1] = &b->d_io;
  b->args[2] = &b->d_items;
  b->args[3] = &b->n_items;
  b->args[4] = &b->d_need;
  b->args[5] = &b->d_ctl;
  b->args[6] = &b->K_arg;
  cudaKernelNodeParams kp = {};
  e = batch_kernel_node(&kp, b->args, b->d_devs, b->d_io, b->d_items, b->n_items, b->d_need, b->d_ctl, b->K, b->grid);
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&nker, b->graph, &nmem, 1, &kp);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  return e;
}

void release(mpopf_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_devs);
  cudaFree(b->d_io);
  cudaFree(b->d_items);
  cudaFree(b->d_need);
  cudaFree(b->d_ctl);
}

}  // namespace

extern "C" {

int mpopf_batch_create(mpopf_handle *const *hs, int32_t k, mpopf_batch **out) {
  if (!hs || !out || k < 1) return fail(MPOPF_ERR_ARG, "mpopf_batch_create: need k >= 1 handles");
  *out = nullptr;
  for (int32_t i = 0; i < k; ++i)
    if (!hs[i]) return fail(MPOPF_ERR_ARG, "mpopf_batch_create: NULL handle");
  mpopf_batch *b = new mpopf_batch();
  b->K = k;
  b->hs.assign(hs, hs + k);
  cudaGetDevice(&b->device);
  std::vector<Dev> devs(k);
  for (int32_t i = 0; i < k; ++i) devs[i] = hs[i]->d;
  cudaError_t e = cudaMalloc(&b->d_devs, k * sizeof(Dev));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_devs, devs.data(), k * sizeof(Dev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_io, k * sizeof(BatchIO));
  if (e == cudaSuccess) e = cudaMemset(b->d_io, 0, k * sizeof(BatchIO));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_need, 2 * k * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, (2 + 2 * k) * sizeof(int32_t));
  if (e == cudaSuccess) e = build_items(b);
  if (e == cudaSuccess) e = build_graph(b);
  if (e != cudaSuccess) {
    release(b);
    delete b;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MPOPF_ERR_ALLOC : MPOPF_ERR_CUDA,
                std::string("mpopf_batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return MPOPF_OK;
}

int mpopf_batch_set_io(mpopf_batch *b, const mpopf_batch_io *io, void *stream) {
  if (!b || !io) return fail(MPOPF_ERR_ARG, "mpopf_batch_set_io: NULL argument");
  std::vector<BatchIO> v(b->K);
  for (int32_t i = 0; i < b->K; ++i) {
    const mpopf_batch_io &s = io[i];
    if (!s.x || !s.lam || !s.sigma_x || !s.dvec || !s.f || !s.grad || !s.c || !s.jv || !s.hv || !s.kv)
      return fail(MPOPF_ERR_ARG, "mpopf_batch_set_io: NULL array in instance " + std::to_string(i));
    v[i] = BatchIO{s.x, s.lam, s.sigma_x, s.dvec, s.f, s.grad, s.c, s.jv, s.hv, s.kv, s.sigma, s.delta_w};
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(b->d_io, v.data(), b->K * sizeof(BatchIO), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // v is a host temporary
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_batch_set_io: ") + cudaGetErrorString(e));
  b->io_set = true;
  return MPOPF_OK;
}

int mpopf_batch_sweep(mpopf_batch *b, void *stream) {
  if (!b) return fail(MPOPF_ERR_ARG, "mpopf_batch_sweep: NULL batch");
  if (!b->io_set) return fail(MPOPF_ERR_ARG, "mpopf_batch_sweep: call mpopf_batch_set_io first");
  const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_batch_sweep: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

int mpopf_batch_status(mpopf_batch *b) {
  if (!b) return fail(MPOPF_ERR_ARG, "mpopf_batch_status: NULL batch");
  int32_t flag = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&flag, b->d_ctl + 1, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_batch_status: ") + cudaGetErrorString(e));
  if (flag) return fail(MPOPF_ERR_CUDA, "mpopf_batch_status: a dependency wait exceeded its limit");
  return MPOPF_OK;
}

int mpopf_batch_set_schedule(mpopf_batch *b, int32_t order, int32_t tile_chunks, int32_t ctas_per_sm) {
  if (!b || order < 0 || order > 1 || tile_chunks < 1 || tile_chunks > 64 || ctas_per_sm < 0)
    return fail(MPOPF_ERR_ARG, "mpopf_batch_set_schedule: bad argument");
  b->sched[0] = order;
  b->sched[1] = tile_chunks;
  b->sched[2] = ctas_per_sm;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = build_items(b);
  if (e == cudaSuccess) e = build_graph(b);
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_batch_set_schedule: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

int mpopf_batch_get_schedule(const mpopf_batch *b, int32_t *sched, int32_t *grid, int32_t *n_items) {
  if (!b || !sched) return fail(MPOPF_ERR_ARG, "mpopf_batch_get_schedule: NULL argument");
  std::memcpy(sched, b->sched, sizeof b->sched);
  if (grid) *grid = b->grid;
  if (n_items) *n_items = b->n_items;
  return MPOPF_OK;
}

int mpopf_batch_tune(mpopf_batch *b, void *stream, int32_t reps, double *best_ms) {
  if (!b || reps < 1) return fail(MPOPF_ERR_ARG, "mpopf_batch_tune: bad argument");
  if (!b->io_set) return fail(MPOPF_ERR_ARG, "mpopf_batch_tune: call mpopf_batch_set_io first");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(MPOPF_ERR_CUDA, "mpopf_batch_tune: event creation failed");
  const int maxc = batch_max_ctas_per_sm();
  double best = 1e300;
  int32_t best_s[3] = {b->sched[0], b->sched[1], b->sched[2]};
  int rc = MPOPF_OK;
  for (int32_t order = 0; order <= 1 && rc == MPOPF_OK; ++order)
    for (int32_t tile : {1, 2, 4})
      for (int32_t cps = 1; cps <= maxc; ++cps) {
        rc = mpopf_batch_set_schedule(b, order, tile, cps);
        if (rc != MPOPF_OK) break;
        for (int w = 0; w < 2; ++w) cudaGraphLaunch(b->exec, st);
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) cudaGraphLaunch(b->exec, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(MPOPF_ERR_CUDA, "mpopf_batch_tune: launch failed"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < best) {
          best = ms / reps;
          best_s[0] = order; best_s[1] = tile; best_s[2] = cps;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MPOPF_OK) return rc;
  if (best_ms) *best_ms = best;
  return mpopf_batch_set_schedule(b, best_s[0], best_s[1], best_s[2]);
}

void mpopf_batch_destroy(mpopf_batch *b) {
  if (!b) return;
  release(b);
  delete b;
}

}  // extern "C"
