// FP64 issue-rate probe: the denominator of the roofline of the FP64-bound
// kernels, measured with a kernel of this library rather than derived.
//
// Every thread runs eight independent chains of fused multiply-adds
// (acc = fma(acc, a, b), a and b chosen so that the values stay normal and
// bounded); eight CTAs of 256 threads per SM keep far more chains in flight
// than the FP64 pipe's latency needs, so the pipe's issue rate is the limit.
// The rate is FP64 thread-instructions (one fma = one instruction, as the
// kernels' operation counts are stated) per second over the best of three
// timed launches after one warm-up launch.
#include <algorithm>
#include <string>

#include "mpopf_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma_chain(double *__restrict__ out, int32_t iters, double a, double b) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = 1.0 + 1e-3 * (double)(k + (tid & 7));
  for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s = s + acc[k];
  out[tid] = s;  // keeps the chains live
}

int fail(int code, const std::string &msg) {
  mpopf::set_error(msg);
  return code;
}

}  // namespace

extern "C" int mpopf_fp64_issue_rate(int32_t iters, double *inst_per_s, double *seconds) {
  if (iters < 1 || !inst_per_s) return fail(MPOPF_ERR_ARG, "mpopf_fp64_issue_rate: bad argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_fp64_issue_rate: ") + cudaGetErrorString(e));
  }
  const int grid = sms * 8;
  double *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, sizeof(double) * (size_t)grid * kThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = -1.f;
  // a < 1 and b > 0 pull every chain toward the fixed point b / (1 - a) = 2
  const double a = 0.9990234375, b = 0.001953125;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    k_dfma_chain<<<grid, kThreads, 0, s>>>(out, iters, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0) best = best < 0.f ? ms : std::min(best, ms);
  }
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_fp64_issue_rate: ") + cudaGetErrorString(e));
  }
  const double fmas = (double)grid * kThreads * (double)iters * kChains;
  *inst_per_s = fmas / (best * 1e-3);
  if (seconds) *seconds = best * 1e-3;
  return MPOPF_OK;
}
