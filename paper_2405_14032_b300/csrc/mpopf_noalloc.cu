// Condensed-matrix assembly that allocates nothing, for callers that cannot
// call cudaMalloc.
//
// Who needs it: code that must not allocate device memory once it is running
// -- processes that reserve all device memory up front and forbid allocation
// afterwards (real-time or embedded controllers, serving processes whose
// memory is managed by a pool), and plugins that run inside a host application
// that owns the device's memory.  The regular mpopf_assemble_kkt uses the
// per-branch scratch buffer that mpopf_setup allocates inside the handle; this
// variant uses instead a fixed array in the library's own device image, so the
// call itself never allocates.
//
// The scratch is a file-scope __device__ array of kScratchDoubles doubles
// (32 MiB).  Every GPU that loads the library holds it until the process
// exits.  Its device address is looked up with cudaGetSymbolAddress (no
// allocation): the first call on a device does that set-up and must come
// before any stream capture; later calls look the address up again (so a
// re-created device context is picked up), except on a stream that is
// capturing, where the address found by an earlier call on that device is
// used.  All calls on a device share the array and it keeps the last call's
// contents; the kernels overwrite every scratch record they later read, so
// nothing needs clearing, but two calls that overlap on the GPU (different
// streams, no ordering) race on it.
#include <mutex>
#include <string>

#include "mpopf_internal.cuh"

namespace {

constexpr long long kScratchDoubles = 4LL * 1024 * 1024;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_kkt_scratch[kScratchDoubles];

std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_kkt_scratch on device `dev`, which is current.  With
// `refresh` the address is looked up again and the cached value replaced;
// without it (a capturing stream) the value an earlier call cached is used.
cudaError_t scratch_address(int dev, bool refresh, double **out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> guard(g_lock);
  if (refresh) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_kkt_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  if (!g_scratch_addr[dev]) return cudaErrorNotReady;
  *out = static_cast<double *>(g_scratch_addr[dev]);
  return cudaSuccess;
}

int fail(int code, const std::string &msg) {
  mpopf::set_error(msg);
  return code;
}

}  // namespace

extern "C" int mpopf_assemble_kkt_noalloc(mpopf_handle *h, const double *x, const double *lam, double sigma,
                                          const double *sigma_x, const double *dvec, double delta_w, double *kv,
                                          void *stream) {
  if (!h) return fail(MPOPF_ERR_ARG, "mpopf_assemble_kkt_noalloc: NULL handle");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_assemble_kkt_noalloc: not available on a period shard");
  if (!x || !lam || !sigma_x || !dvec || !kv) return fail(MPOPF_ERR_ARG, "mpopf_assemble_kkt_noalloc: NULL array");
  const long long need = 2LL * mpopf::kRec * h->d.T * h->d.L;
  if (need > kScratchDoubles)
    return fail(MPOPF_ERR_SIZE, "mpopf_assemble_kkt_noalloc: needs " + std::to_string(need) +
                                    " scratch doubles (12 per branch x period), over the static maximum of " +
                                    std::to_string(kScratchDoubles) + " (T x L <= 349525)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_assemble_kkt_noalloc: ") + cudaGetErrorString(e));
  }
  if (dev != h->device)
    return fail(MPOPF_ERR_ARG, "mpopf_assemble_kkt_noalloc: the current device (" + std::to_string(dev) +
                                   ") is not the handle's (" + std::to_string(h->device) + ")");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_assemble_kkt_noalloc: stream state: ") + cudaGetErrorString(e));
  }
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  double *scratch = nullptr;
  e = scratch_address(dev, !capturing, &scratch);
  if (e == cudaErrorNotReady)
    return fail(MPOPF_ERR_ARG, "mpopf_assemble_kkt_noalloc: the first call on a device must come before any "
                               "stream capture (it looks up the scratch address)");
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_assemble_kkt_noalloc: scratch lookup: ") + cudaGetErrorString(e));
  }
  mpopf::Dev d = h->d;
  d.S = scratch;
  e = mpopf::launch_eval(d, MPOPF_OUT_KKT, x, lam, sigma, sigma_x, dvec, delta_w, nullptr, nullptr, nullptr,
                         nullptr, nullptr, kv, s, nullptr);
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_assemble_kkt_noalloc: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}
