// COO -> CSC compression of the Jacobian and of the lower-triangle Lagrangian
// Hessian (Sec. III-A: the COO matrices are optionally compressed to CSC).
//
// The CSC pattern is built once per handle and matrix, on the device: entries
// ordered by (column, row), equal (row, column) pairs in COO order -- the
// order of two stable counting sorts, by row and then by column.  Each
// compression is one kernel: a gather for J (no duplicate
// entries), a fixed-order sum of each run of duplicates for W (the first
// entry, then the others added in COO order), so the values are deterministic
// and equal the CPU reference bit for bit.
#include <algorithm>
#include <string>
#include <vector>

#include "mpopf_internal.cuh"

namespace mpopf {
namespace {

// Each thread takes kStreams outputs a stride apart (u, u + stride, ...), so a
// warp's index loads and stores stay coalesced and a thread has kStreams
// independent gathers of COO values in flight.
constexpr int kStreams = 4;
template <bool SEG>
__global__ void __launch_bounds__(kBlock) k_csc_values(int64_t nnz, int64_t stride, const int64_t *__restrict__ seg,
                                                       const int32_t *__restrict__ src,
                                                       const double *__restrict__ coo, double *__restrict__ out) {
  const int64_t u0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u0 >= stride) return;
  if constexpr (!SEG) {
    int32_t s[kStreams];
    double v[kStreams];
#pragma unroll
    for (int k = 0; k < kStreams; ++k) s[k] = u0 + k * stride < nnz ? __ldg(src + u0 + k * stride) : 0;
#pragma unroll
    for (int k = 0; k < kStreams; ++k) v[k] = u0 + k * stride < nnz ? __ldg(coo + s[k]) : 0.0;
#pragma unroll
    for (int k = 0; k < kStreams; ++k)
      if (u0 + k * stride < nnz) out[u0 + k * stride] = v[k];
  } else {
#pragma unroll
    for (int k = 0; k < kStreams; ++k) {
      const int64_t u = u0 + k * stride;
      if (u >= nnz) break;
      const int64_t p0 = seg[u], p1 = seg[u + 1];
      double acc = coo[src[p0]];
      for (int64_t p = p0 + 1; p < p1; ++p) acc = acc + coo[src[p]];
      out[u] = acc;
    }
  }
}

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

// Exclusive scan of n int32 counts into n + 1 int64 offsets (setup time): per
// 1024-element block a local scan and the block total, the block totals
// scanned on the host, then the block offsets added.
constexpr int kScanBlock = 1024;  // elements per CTA (256 threads x 4)

__global__ void __launch_bounds__(kBlock) k_scan_local(const int32_t *__restrict__ in, int64_t n,
                                                       int64_t *__restrict__ out, int64_t *__restrict__ totals) {
  __shared__ int64_t part[kBlock];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + 4 * (int64_t)threadIdx.x;
  int64_t v[4], sum = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    sum += v[j];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < kBlock; off <<= 1) {  // inclusive scan of the thread sums
    const int64_t add = (int)threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - sum;  // exclusive prefix of this thread
  for (int j = 0; j < 4; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == kBlock - 1) totals[blockIdx.x] = part[threadIdx.x];
}

__global__ void __launch_bounds__(kBlock) k_scan_add(int64_t n, const int64_t *__restrict__ offsets,
                                                     int64_t *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += offsets[i / kScanBlock];
}

// out[0..n] = exclusive prefix sums of in[0..n); returns the total in *total.
cudaError_t exclusive_scan(const int32_t *in, int64_t n, int64_t *out, int64_t *total) {
  const int64_t nb = std::max<int64_t>(1, (n + kScanBlock - 1) / kScanBlock);
  int64_t *totals = nullptr;
  cudaError_t e = cudaMalloc(&totals, nb * sizeof(int64_t));
  if (e != cudaSuccess) return e;
  if (n > 0) k_scan_local<<<(unsigned)nb, kBlock>>>(in, n, out, totals);
  std::vector<int64_t> h(nb, 0);
  e = cudaGetLastError();
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(h.data(), totals, nb * sizeof(int64_t), cudaMemcpyDeviceToHost);
  int64_t acc = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t t = h[b];
    h[b] = acc;
    acc += t;
  }
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(totals, h.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) k_scan_add<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock>>>(n, totals, out);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(out + n, &acc, sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(totals);
  *total = acc;
  return e;
}

// Entries per column.
__global__ void __launch_bounds__(kBlock) k_col_count(int64_t nnz, const int32_t *__restrict__ col,
                                                      int32_t *__restrict__ cnt) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < nnz) atomicAdd(cnt + col[k], 1);
}

// Each entry into its column's segment, in arbitrary order within the column.
__global__ void __launch_bounds__(kBlock) k_col_scatter(int64_t nnz, const int32_t *__restrict__ col,
                                                        const int64_t *__restrict__ start,
                                                        int32_t *__restrict__ fill, int32_t *__restrict__ order) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int32_t c = col[k];
  order[start[c] + atomicAdd(fill + c, 1)] = (int32_t)k;
}

// One thread per column: its segment sorted by (row, COO entry) -- the order
// two stable counting sorts (by row, then by column) give -- and its number of
// distinct rows.
__global__ void __launch_bounds__(kBlock) k_col_sort(int64_t ncols, const int64_t *__restrict__ start,
                                                     const int32_t *__restrict__ row, int32_t *__restrict__ order,
                                                     int32_t *__restrict__ distinct) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const int64_t s = start[c], e = start[c + 1];
  for (int64_t i = s + 1; i < e; ++i) {  // insertion sort (columns hold tens of entries)
    const int32_t k = order[i], r = row[k];
    int64_t j = i - 1;
    while (j >= s && (row[order[j]] > r || (row[order[j]] == r && order[j] > k))) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = k;
  }
  int32_t u = 0;
  for (int64_t i = s; i < e; ++i) u += (i == s || row[order[i]] != row[order[i - 1]]) ? 1 : 0;
  distinct[c] = u;
}

// One thread per column: a CSC entry per run of equal rows (its row and, with
// duplicates, the run's first sorted position).
__global__ void __launch_bounds__(kBlock) k_col_emit(int64_t ncols, const int64_t *__restrict__ start,
                                                     const int64_t *__restrict__ colptr,
                                                     const int32_t *__restrict__ row,
                                                     const int32_t *__restrict__ order, int32_t *__restrict__ rowidx,
                                                     int64_t *__restrict__ seg) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  int64_t j = colptr[c];
  for (int64_t i = start[c]; i < start[c + 1]; ++i)
    if (i == start[c] || row[order[i]] != row[order[i - 1]]) {
      rowidx[j] = row[order[i]];
      if (seg) seg[j] = i;
      ++j;
    }
}

// A device allocation owned by the handle.
template <class T>
cudaError_t alloc_owned(mpopf_handle *h, int64_t count, T **dst) {
  *dst = nullptr;
  if (h->nblocks >= kMaxBlocks) return cudaErrorMemoryAllocation;
  void *p = nullptr;
  const cudaError_t e = cudaMalloc(&p, std::max<int64_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->blocks[h->nblocks++] = p;
  *dst = static_cast<T *>(p);
  return cudaSuccess;
}

unsigned grid_of(int64_t count) { return (unsigned)std::max<int64_t>(1, (count + kBlock - 1) / kBlock); }

// The CSC pattern on the device: entries counted and scattered into their
// columns, each column's segment sorted by (row, COO entry), runs of equal
// rows numbered.  The result equals two stable counting sorts of the entry
// list by row and then by column.
int build_csc(mpopf_handle *h, int which) {
  const mpopf_pattern &P = h->pat;
  const int64_t nnz = which == MPOPF_CSC_JAC ? P.nnz_jac : P.nnz_hess;
  const int64_t ncols = P.n;
  if (nnz >= ((int64_t)1 << 31))
    return fail(MPOPF_ERR_SIZE, "mpopf_csc_pattern: 2^31 or more entries (32-bit entry numbers)");
  const int32_t *row = which == MPOPF_CSC_JAC ? P.jac_row : P.hess_row;
  const int32_t *col = which == MPOPF_CSC_JAC ? P.jac_col : P.hess_col;
  CscState &c = h->csc[which];
  int32_t *cnt = nullptr, *fill = nullptr;
  int64_t *start = nullptr;
  int32_t *order = nullptr, *rowidx = nullptr;
  int64_t *colptr = nullptr, *seg = nullptr;
  int64_t total = 0, nnz_csc = 0;
  cudaError_t e = cudaMalloc(&cnt, std::max<int64_t>(ncols, 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&fill, std::max<int64_t>(ncols, 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&start, (ncols + 1) * sizeof(int64_t));
  if (e == cudaSuccess) e = alloc_owned(h, nnz, &order);
  if (e == cudaSuccess) e = alloc_owned(h, ncols + 1, &colptr);
  if (e == cudaSuccess) e = cudaMemset(cnt, 0, std::max<int64_t>(ncols, 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(fill, 0, std::max<int64_t>(ncols, 1) * sizeof(int32_t));
  if (e == cudaSuccess && nnz > 0) {
    k_col_count<<<grid_of(nnz), kBlock>>>(nnz, col, cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = exclusive_scan(cnt, ncols, start, &total);
  if (e == cudaSuccess && nnz > 0) {
    k_col_scatter<<<grid_of(nnz), kBlock>>>(nnz, col, start, fill, order);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && ncols > 0) {
    k_col_sort<<<grid_of(ncols), kBlock>>>(ncols, start, row, order, cnt);  // cnt <- distinct rows per column
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = exclusive_scan(cnt, ncols, colptr, &nnz_csc);
  const bool dups = nnz_csc != nnz;
  if (e == cudaSuccess) e = alloc_owned(h, nnz_csc, &rowidx);
  if (e == cudaSuccess && dups) e = alloc_owned(h, nnz_csc + 1, &seg);
  if (e == cudaSuccess && ncols > 0) {
    k_col_emit<<<grid_of(ncols), kBlock>>>(ncols, start, colptr, row, order, rowidx, dups ? seg : nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && dups) e = cudaMemcpy(seg + nnz_csc, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(cnt);
  cudaFree(fill);
  cudaFree(start);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MPOPF_ERR_ALLOC : MPOPF_ERR_CUDA,
                std::string("mpopf_csc_pattern: ") + cudaGetErrorString(e));
  }
  c.colptr = colptr;
  c.rowidx = rowidx;
  c.src = order;
  c.seg = dups ? seg : nullptr;
  c.nnz = nnz_csc;
  c.built = true;
  return MPOPF_OK;
}

}  // namespace
}  // namespace mpopf

using namespace mpopf;

extern "C" {

int mpopf_csc_pattern(mpopf_handle *h, int32_t which, mpopf_csc *out) {
  if (!h || !out) return fail(MPOPF_ERR_ARG, "mpopf_csc_pattern: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_csc_pattern: not available on a period shard");
  if (which != MPOPF_CSC_JAC && which != MPOPF_CSC_HESS)
    return fail(MPOPF_ERR_ARG, "mpopf_csc_pattern: which must be MPOPF_CSC_JAC or MPOPF_CSC_HESS");
  if (!h->csc[which].built) {
    const int rc = build_csc(h, which);
    if (rc != MPOPF_OK) return rc;
  }
  const CscState &c = h->csc[which];
  out->nnz = c.nnz;
  out->colptr = c.colptr;
  out->rowidx = c.rowidx;
  return MPOPF_OK;
}

int mpopf_coo_to_csc(mpopf_handle *h, int32_t which, const double *coo_vals, double *csc_vals, void *stream) {
  if (!h || !coo_vals || !csc_vals) return fail(MPOPF_ERR_ARG, "mpopf_coo_to_csc: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_coo_to_csc: not available on a period shard");
  if (which != MPOPF_CSC_JAC && which != MPOPF_CSC_HESS)
    return fail(MPOPF_ERR_ARG, "mpopf_coo_to_csc: which must be MPOPF_CSC_JAC or MPOPF_CSC_HESS");
  const CscState &c = h->csc[which];
  if (!c.built) return fail(MPOPF_ERR_ARG, "mpopf_coo_to_csc: call mpopf_csc_pattern for this matrix first");
  if (c.nnz == 0) return MPOPF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t stride = (c.nnz + kStreams - 1) / kStreams;
  const unsigned grid = (unsigned)((stride + kBlock - 1) / kBlock);
  if (c.seg)
    k_csc_values<true><<<grid, kBlock, 0, st>>>(c.nnz, stride, c.seg, c.src, coo_vals, csc_vals);
  else
    k_csc_values<false><<<grid, kBlock, 0, st>>>(c.nnz, stride, nullptr, c.src, coo_vals, csc_vals);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_coo_to_csc: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

}  // extern "C"
