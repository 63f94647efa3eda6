// COO -> CSC compression of the Jacobian and of the lower-triangle Lagrangian
// Hessian (Sec. III-A: the COO matrices are optionally compressed to CSC).
//
// The CSC pattern is built once per handle and matrix by two stable counting
// sorts on the host (by row, then by column: entries end up ordered by
// (column, row), equal (row, column) pairs in COO order), then copied to the
// device.  Each compression is one kernel: a gather for J (no duplicate
// entries), a fixed-order sum of each run of duplicates for W (the first
// entry, then the others added in COO order), so the values are deterministic
// and equal the CPU reference bit for bit.
#include <string>
#include <vector>

#include "mpopf_internal.cuh"

namespace mpopf {
namespace {

template <bool SEG>
__global__ void __launch_bounds__(kBlock) k_csc_values(int64_t nnz, const int64_t *__restrict__ seg,
                                                       const int32_t *__restrict__ src,
                                                       const double *__restrict__ coo, double *__restrict__ out) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= nnz) return;
  if (!SEG) {
    out[u] = coo[src[u]];
    return;
  }
  const int64_t p0 = seg[u], p1 = seg[u + 1];
  double acc = coo[src[p0]];
  for (int64_t p = p0 + 1; p < p1; ++p) acc = acc + coo[src[p]];
  out[u] = acc;
}

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

// Stable counting sort of the entry list `order` by key[order[k]] in [0, nkeys).
void counting_sort(const std::vector<int32_t> &key, int64_t nkeys, std::vector<int32_t> &order) {
  std::vector<int64_t> start(nkeys + 1, 0);
  for (int32_t e : order) start[key[e] + 1] += 1;
  for (int64_t k = 0; k < nkeys; ++k) start[k + 1] += start[k];
  std::vector<int32_t> out(order.size());
  for (int32_t e : order) out[start[key[e]]++] = e;
  order.swap(out);
}

template <class T>
cudaError_t upload(mpopf_handle *h, const std::vector<T> &v, T **dst) {
  *dst = nullptr;
  if (h->nblocks >= kMaxBlocks) return cudaErrorMemoryAllocation;
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(v.size(), 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->blocks[h->nblocks++] = p;
  if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  *dst = static_cast<T *>(p);
  return e;
}

int build_csc(mpopf_handle *h, int which) {
  const mpopf_pattern &P = h->pat;
  const int64_t nnz = which == MPOPF_CSC_JAC ? P.nnz_jac : P.nnz_hess;
  const int64_t nrows = which == MPOPF_CSC_JAC ? P.m : P.n, ncols = P.n;
  if (nnz >= ((int64_t)1 << 31))
    return fail(MPOPF_ERR_SIZE, "mpopf_csc_pattern: 2^31 or more entries (32-bit entry numbers)");
  std::vector<int32_t> row(nnz), col(nnz);
  cudaError_t e = cudaSuccess;
  if (nnz > 0) {
    e = cudaMemcpy(row.data(), which == MPOPF_CSC_JAC ? P.jac_row : P.hess_row, nnz * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(col.data(), which == MPOPF_CSC_JAC ? P.jac_col : P.hess_col, nnz * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_csc_pattern: ") + cudaGetErrorString(e));
  }
  std::vector<int32_t> order(nnz);
  for (int64_t k = 0; k < nnz; ++k) order[k] = (int32_t)k;
  counting_sort(row, nrows, order);
  counting_sort(col, ncols, order);
  // runs of equal (row, column): one CSC entry each
  std::vector<int64_t> colptr(ncols + 1, 0), seg;
  std::vector<int32_t> rowidx;
  rowidx.reserve(nnz);
  seg.reserve(nnz + 1);
  for (int64_t k = 0; k < nnz; ++k) {
    const int32_t ek = order[k];
    if (k == 0 || row[ek] != row[order[k - 1]] || col[ek] != col[order[k - 1]]) {
      rowidx.push_back(row[ek]);
      seg.push_back(k);
      colptr[col[ek] + 1] += 1;
    }
  }
  seg.push_back(nnz);
  for (int64_t j = 0; j < ncols; ++j) colptr[j + 1] += colptr[j];
  CscState &c = h->csc[which];
  const bool dups = (int64_t)rowidx.size() != nnz;
  e = upload(h, colptr, &c.colptr);
  if (e == cudaSuccess) e = upload(h, rowidx, &c.rowidx);
  if (e == cudaSuccess) e = upload(h, order, &c.src);
  if (e == cudaSuccess && dups) e = upload(h, seg, &c.seg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MPOPF_ERR_ALLOC : MPOPF_ERR_CUDA,
                std::string("mpopf_csc_pattern: ") + cudaGetErrorString(e));
  }
  if (!dups) c.seg = nullptr;
  c.nnz = (int64_t)rowidx.size();
  c.built = true;
  return MPOPF_OK;
}

}  // namespace
}  // namespace mpopf

using namespace mpopf;

extern "C" {

int mpopf_csc_pattern(mpopf_handle *h, int32_t which, mpopf_csc *out) {
  if (!h || !out) return fail(MPOPF_ERR_ARG, "mpopf_csc_pattern: NULL argument");
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
  if (which != MPOPF_CSC_JAC && which != MPOPF_CSC_HESS)
    return fail(MPOPF_ERR_ARG, "mpopf_coo_to_csc: which must be MPOPF_CSC_JAC or MPOPF_CSC_HESS");
  const CscState &c = h->csc[which];
  if (!c.built) return fail(MPOPF_ERR_ARG, "mpopf_coo_to_csc: call mpopf_csc_pattern for this matrix first");
  if (c.nnz == 0) return MPOPF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)((c.nnz + kBlock - 1) / kBlock);
  if (c.seg)
    k_csc_values<true><<<grid, kBlock, 0, st>>>(c.nnz, c.seg, c.src, coo_vals, csc_vals);
  else
    k_csc_values<false><<<grid, kBlock, 0, st>>>(c.nnz, nullptr, c.src, coo_vals, csc_vals);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_coo_to_csc: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

}  // extern "C"
