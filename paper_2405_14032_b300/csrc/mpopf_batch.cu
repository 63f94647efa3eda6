// Batched evaluation of many independent multi-period AC OPF instances of
// uneven size in one persistent launch, replayed as a CUDA graph, with a
// schedule chosen by measurement (autotuner).
//
// The work list holds tiles ("items") of every instance: generator tiles,
// branch tiles and bus tiles, then one objective item per instance.  The
// horizon of each instance is cut into chunks of P periods; the bus tiles of a
// chunk wait only for that chunk's branch tiles (whose incidence records they
// sum) and come in the list one chunk behind them, so bus work overlaps branch
// work.  The schedule decides the instance order (as given, or largest first),
// the tile size (CTA-sized chunks per item), the persistent grid (CTAs per SM)
// and P (0: the whole horizon), and one launch or two: with two, the first
// launch takes the branch tiles (in the sweep kernel's 64-thread CTAs) and the
// second the generator tiles, the bus tiles and the objective items, so the
// launch boundary replaces the bus tiles' waits and the bus work runs at its
// own occupancy.  Or no persistent launch at all: each instance's plain sweep
// (mpopf_sweep's launches) on one of S parallel branches of the graph
// (instances dealt round-robin in the schedule's order), so that the plain
// kernels of several instances share the GPU.  Results do not depend on the
// schedule: each value is computed by the same sequence of operations
// whichever CTA runs it.
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
  int32_t *d_need = nullptr;  // [n_counters]
  int32_t *d_ctl = nullptr;   // [3 + n_counters]
  int32_t n_items = 0, n_counters = 0, cap_ctl = 0;
  // order (0 given, 1 largest first), tile chunks, CTAs per SM (0 = max),
  // periods per chunk (0 = all), launches (1 or 2; 0: plain sweeps on
  // parallel branches, CTAs per SM then the number of branches, 0 = 16)
  int32_t sched[5] = {0, 1, 0, 0, 1};
  int32_t grid = 0;
  // two-launch schedule: items [0, n_items1) go to the first launch, the rest
  // to the second (grid2 CTAs)
  int32_t n_items1 = 0, n_items2 = 0, grid2 = 0;
  BatchItem *d_items2 = nullptr;
  int32_t *d_next2 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void *args[7], *args2[7];
  bool io_set = false;
  std::vector<BatchIO> io_host;          // the instances' pointers (plain-sweep schedule)
  std::vector<cudaStream_t> br_streams;  // capture streams of the plain-sweep schedule
  std::vector<cudaEvent_t> br_join;
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_start = nullptr;
  std::vector<int32_t> need_host;  // dependency targets as built (the stall hook restores them)
  int32_t stall_counter = -1;      // counter whose target the stall hook raised, or -1
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
  const bool two = b->sched[4] == 2;
  // tiles are whole CTAs of the launch that runs them
  const int32_t chunks = std::max(1, b->sched[1]);
  const int32_t tile = kBlock * chunks, tile_branch = (two ? batch_block_threads(1) : kBlock) * chunks;
  std::vector<BatchItem> items;
  std::vector<int32_t> need;
  auto add = [&](int32_t kind, int32_t k, int64_t u0, int64_t u1, int32_t wait, int32_t signal) {
    const int32_t t = kind == ITEM_BRANCH ? tile_branch : tile;
    for (int64_t f = u0; f < u1; f += t) {
      items.push_back(BatchItem{k, kind, (int32_t)f, (int32_t)std::min<int64_t>(t, u1 - f), wait, signal});
      if (signal >= 0) ++need[signal];
    }
  };
  std::vector<int32_t> gen_counter(K, -1);
  int32_t n1 = 0;
  if (two) {
    // first launch: every branch tile; second: the generator tiles, the bus
    // tiles, then the objectives (each waits for its generator tiles)
    for (int32_t k : order) {
      const Dev &d = b->hs[k]->d;
      add(ITEM_BRANCH, k, 0, (int64_t)d.T * d.L, -1, -1);
    }
    n1 = (int32_t)items.size();
    for (int32_t k : order) {
      const Dev &d = b->hs[k]->d;
      gen_counter[k] = (int32_t)need.size();
      need.push_back(0);
      add(ITEM_GEN, k, 0, (int64_t)d.T * d.G, -1, gen_counter[k]);
    }
    for (int32_t k : order) {
      const Dev &d = b->hs[k]->d;
      add(ITEM_BUS, k, 0, (int64_t)d.T * d.N, -1, -1);
    }
    for (int32_t k : order) items.push_back(BatchItem{k, ITEM_FSUM, 0, 1, gen_counter[k], -1});
  } else {
    for (int32_t k : order) {  // generator tiles first (no prerequisites)
      const Dev &d = b->hs[k]->d;
      gen_counter[k] = (int32_t)need.size();
      need.push_back(0);
      add(ITEM_GEN, k, 0, (int64_t)d.T * d.G, -1, gen_counter[k]);
    }
    // Branch and bus tiles by period chunks, the bus tiles one chunk behind.
    struct Chunk { int32_t k, t0, t1, counter; };
    std::vector<std::vector<Chunk>> per(K);
    int32_t rounds = 0;
    for (int32_t k : order) {
      const Dev &d = b->hs[k]->d;
      const int32_t P = b->sched[3] > 0 ? b->sched[3] : d.T;
      for (int32_t t0 = 0; t0 < d.T; t0 += P) {
        per[k].push_back(Chunk{k, t0, std::min(d.T, t0 + P), (int32_t)need.size()});
        need.push_back(0);
      }
      rounds = std::max(rounds, (int32_t)per[k].size());
    }
    for (int32_t r = 0; r <= rounds; ++r)
      for (int32_t k : order) {
        const Dev &d = b->hs[k]->d;
        if (r < (int32_t)per[k].size()) {
          const Chunk &c = per[k][r];
          add(ITEM_BRANCH, k, (int64_t)c.t0 * d.L, (int64_t)c.t1 * d.L, -1, c.counter);
        }
        if (r >= 1 && r - 1 < (int32_t)per[k].size()) {
          const Chunk &c = per[k][r - 1];
          add(ITEM_BUS, k, (int64_t)c.t0 * d.N, (int64_t)c.t1 * d.N, d.L > 0 ? c.counter : -1, -1);
        }
      }
    for (int32_t k : order) items.push_back(BatchItem{k, ITEM_FSUM, 0, 1, gen_counter[k], -1});
    n1 = (int32_t)items.size();
  }
  cudaError_t e = cudaSuccess;
  const int32_t n_ctl = 3 + (int32_t)need.size();
  if (n_ctl > b->cap_ctl) {
    cudaFree(b->d_need);
    cudaFree(b->d_ctl);
    b->d_need = nullptr;
    b->d_ctl = nullptr;
    e = cudaMalloc(&b->d_need, std::max<size_t>(need.size(), 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, n_ctl * sizeof(int32_t));
    b->cap_ctl = n_ctl;
  }
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, items.size() * sizeof(BatchItem));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !need.empty())
    e = cudaMemcpy(b->d_need, need.data(), need.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  b->n_items = (int32_t)items.size();
  b->n_items1 = n1;
  b->n_items2 = b->n_items - n1;
  b->n_counters = (int32_t)need.size();
  b->d_items2 = b->d_items + n1;
  b->d_next2 = b->d_ctl + 2 + b->n_counters;
  b->need_host = need;
  b->stall_counter = -1;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int phase1 = two ? 1 : 0;
  const int max1 = batch_max_ctas_per_sm(phase1);
  // CTAs per SM apply to the one-launch form; the two launches run at their
  // occupancy maximum
  const int per_sm = (!two && b->sched[2] > 0) ? std::min(b->sched[2], max1) : max1;
  b->grid = std::max(1, std::min(sms * per_sm, std::max(1, b->n_items1)));
  b->grid2 = two ? std::max(1, std::min(sms * batch_max_ctas_per_sm(2), std::max(1, b->n_items2))) : 0;
  return e;
}

std::vector<int32_t> instance_order(const mpopf_batch *b) {
  std::vector<int32_t> order(b->K);
  std::iota(order.begin(), order.end(), 0);
  if (b->sched[0] == 1)
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t c) { return work_of(b->hs[a]->d) > work_of(b->hs[c]->d); });
  return order;
}

// The plain-sweep schedule's graph, captured from S streams: a start event
// forks every stream off the capture stream, instance k of the order runs
// its sweep (launch_eval, the handle's own side stream and schedule) on
// stream k mod S, and every stream joins the capture stream at the end.
cudaError_t capture_plain_sweeps(mpopf_batch *b) {
  const int32_t S = std::min<int32_t>(b->sched[2] ? b->sched[2] : 16, b->K);
  cudaError_t e = cudaSuccess;
  if (!b->cap) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess && !b->ev_start) e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming);
  while (e == cudaSuccess && (int32_t)b->br_streams.size() < S) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (st) b->br_streams.push_back(st);
    if (ev) b->br_join.push_back(ev);
  }
  if (e != cudaSuccess) return e;
  const std::vector<int32_t> order = instance_order(b);
  e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t c = cudaEventRecord(b->ev_start, b->cap);
  for (int32_t s = 0; s < S && c == cudaSuccess; ++s) c = cudaStreamWaitEvent(b->br_streams[s], b->ev_start, 0);
  for (int32_t k = 0; k < b->K && c == cudaSuccess; ++k) {
    const int32_t i = order[k];
    const BatchIO &io = b->io_host[i];
    c = launch_eval(b->hs[i]->d, MPOPF_OUT_ALL, io.x, io.lam, io.sigma, io.sx, io.dv, io.dw, io.f, io.grad, io.c,
                    io.jv, io.hv, io.kv, b->br_streams[k % S], nullptr, &b->hs[i]->fork);
  }
  for (int32_t s = 0; s < S && c == cudaSuccess; ++s) {
    c = cudaEventRecord(b->br_join[s], b->br_streams[s]);
    if (c == cudaSuccess) c = cudaStreamWaitEvent(b->cap, b->br_join[s], 0);
  }
  e = cudaStreamEndCapture(b->cap, &b->graph);  // ends the capture whatever happened inside it
  if (c != cudaSuccess) e = c;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  return e;
}

// (Re)build the graph: reset the counters, then the persistent kernel (or the
// plain sweeps, once the instances' pointers are known).
cudaError_t build_graph(mpopf_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (b->sched[4] == 0) return b->io_set ? capture_plain_sweeps(b) : cudaSuccess;
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  if (e != cudaSuccess) return e;
  cudaMemsetParams mp = {};
  mp.dst = b->d_ctl;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = (size_t)(3 + b->n_counters);
  mp.height = 1;
  mp.pitch = 0;
  cudaGraphNode_t nmem = nullptr, nker = nullptr, nker2 = nullptr;
  e = cudaGraphAddMemsetNode(&nmem, b->graph, nullptr, 0, &mp);
  if (e != cudaSuccess) return e;
  const bool two = b->sched[4] == 2;
  b->args[0] = &b->d_devs;
  b->args[1] = &b->d_io;
  b->args[2] = &b->d_items;
  b->args[3] = &b->n_items1;
  b->args[4] = &b->d_need;
  b->args[5] = &b->d_ctl;
  b->args[6] = &b->d_ctl;  // the first launch counts items in ctl[0]
  cudaKernelNodeParams kp = {};
  e = batch_kernel_node(&kp, b->args, b->grid, two ? 1 : 0);
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&nker, b->graph, &nmem, 1, &kp);
  if (e == cudaSuccess && two) {
    b->args2[0] = &b->d_devs;
    b->args2[1] = &b->d_io;
    b->args2[2] = &b->d_items2;
    b->args2[3] = &b->n_items2;
    b->args2[4] = &b->d_need;
    b->args2[5] = &b->d_ctl;
    b->args2[6] = &b->d_next2;
    cudaKernelNodeParams kp2 = {};
    e = batch_kernel_node(&kp2, b->args2, b->grid2, 2);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&nker2, b->graph, &nker, 1, &kp2);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  return e;
}

void release(mpopf_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t st : b->br_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->br_join) cudaEventDestroy(ev);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
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
  for (int32_t i = 0; i < k; ++i)
    if (mpopf::is_shard(hs[i]->d)) return fail(MPOPF_ERR_ARG, "mpopf_batch_create: not available on a period shard");
  {
    // an instance's scratch (incidence records, objective partials) belongs to
    // its handle, so a handle may appear only once
    std::vector<mpopf_handle *> sorted(hs, hs + k);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(MPOPF_ERR_ARG, "mpopf_batch_create: a handle appears twice");
  }
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
  b->io_host = v;
  b->io_set = true;
  if (b->sched[4] == 0) {  // the plain sweeps' graph holds the pointers: capture it again
    e = build_graph(b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MPOPF_ERR_CUDA, std::string("mpopf_batch_set_io: ") + cudaGetErrorString(e));
    }
  }
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

int mpopf_batch_test_stall(mpopf_batch *b, int32_t on) {
  if (!b) return fail(MPOPF_ERR_ARG, "mpopf_batch_test_stall: NULL batch");
  cudaError_t e = cudaSuccess;
  if (b->stall_counter >= 0) {  // restore
    const int32_t c = b->stall_counter;
    e = cudaMemcpy(b->d_need + c, &b->need_host[c], sizeof(int32_t), cudaMemcpyHostToDevice);
    b->stall_counter = -1;
  }
  if (e == cudaSuccess && on && b->sched[4] == 0)
    return fail(MPOPF_ERR_ARG, "mpopf_batch_test_stall: no bus tile waits (plain sweeps)");
  if (e == cudaSuccess && on) {
    // the first counter a bus tile waits on (a chunk of some instance's branch tiles)
    int32_t c = -1;
    std::vector<BatchItem> items(b->n_items);
    e = cudaMemcpy(items.data(), b->d_items, items.size() * sizeof(BatchItem), cudaMemcpyDeviceToHost);
    for (const BatchItem &it : items)
      if (it.kind == ITEM_BUS && it.wait >= 0) { c = it.wait; break; }
    if (e == cudaSuccess && c < 0) return fail(MPOPF_ERR_ARG, "mpopf_batch_test_stall: no bus tile waits");
    if (e == cudaSuccess) {
      const int32_t raised = b->need_host[c] + 1;
      e = cudaMemcpy(b->d_need + c, &raised, sizeof(int32_t), cudaMemcpyHostToDevice);
      b->stall_counter = c;
    }
  }
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_batch_test_stall: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

int mpopf_batch_set_schedule(mpopf_batch *b, int32_t order, int32_t tile_chunks, int32_t ctas_per_sm,
                             int32_t chunk_periods, int32_t launches) {
  if (!b || order < 0 || order > 1 || tile_chunks < 1 || tile_chunks > 64 || ctas_per_sm < 0 || chunk_periods < 0 ||
      launches < 0 || launches > 2 || (launches == 0 && ctas_per_sm > 64))
    return fail(MPOPF_ERR_ARG, "mpopf_batch_set_schedule: bad argument");
  b->sched[0] = order;
  b->sched[1] = tile_chunks;
  b->sched[2] = ctas_per_sm;
  b->sched[3] = chunk_periods;
  b->sched[4] = launches;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = build_items(b);
  if (e == cudaSuccess) e = build_graph(b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_batch_set_schedule: ") + cudaGetErrorString(e));
  }
  return MPOPF_OK;
}

int mpopf_batch_get_schedule(const mpopf_batch *b, int32_t *sched, int32_t *grid, int32_t *n_items) {
  if (!b || !sched) return fail(MPOPF_ERR_ARG, "mpopf_batch_get_schedule: NULL argument");
  std::memcpy(sched, b->sched, sizeof b->sched);  // [5]
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
  const int maxc = batch_max_ctas_per_sm(0);
  double best = 1e300;
  int32_t best_s[5] = {b->sched[0], b->sched[1], b->sched[2], b->sched[3], b->sched[4]};
  int32_t maxT = 1;
  for (auto *h : b->hs) maxT = std::max(maxT, h->d.T);
  std::vector<int32_t> chunks = {0};
  for (int32_t P : {1, 2, 4, 8, 16}) if (P < maxT) chunks.push_back(P);
  int rc = MPOPF_OK;
  auto trial = [&](int32_t order, int32_t tile, int32_t cps, int32_t P, int32_t launches) {
    if (rc != MPOPF_OK) return;
    rc = mpopf_batch_set_schedule(b, order, tile, cps, P, launches);
    if (rc != MPOPF_OK) return;
    for (int w = 0; w < 2; ++w) cudaGraphLaunch(b->exec, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) cudaGraphLaunch(b->exec, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = fail(MPOPF_ERR_CUDA, "mpopf_batch_tune: launch failed");
      return;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / reps < best) {
      best = ms / reps;
      best_s[0] = order; best_s[1] = tile; best_s[2] = cps; best_s[3] = P; best_s[4] = launches;
    }
  };
  // coordinate search: grid and tile with whole-horizon chunks (one launch),
  // tile (two launches), then the chunk length (one launch), then the instance
  // order
  for (int32_t cps = 1; cps <= maxc; ++cps)
    for (int32_t tile : {1, 2, 4}) trial(0, tile, cps, 0, 1);
  for (int32_t tile : {1, 2, 4, 8}) trial(0, tile, 0, 0, 2);
  if (best_s[4] == 1)
    for (int32_t P : chunks) trial(0, best_s[1], best_s[2], P, 1);
  // plain sweeps on 4 .. 64 parallel branches (largest instances first)
  for (int32_t S : {4, 8, 16, 32, 64})
    if (S <= 2 * b->K) trial(1, 1, S, 0, 0);
  trial(1, best_s[1], best_s[2], best_s[3], best_s[4]);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MPOPF_OK) return rc;
  if (best_ms) *best_ms = best;
  return mpopf_batch_set_schedule(b, best_s[0], best_s[1], best_s[2], best_s[3], best_s[4]);
}

void mpopf_batch_destroy(mpopf_batch *b) {
  if (!b) return;
  release(b);
  delete b;
}

}  // extern "C"
