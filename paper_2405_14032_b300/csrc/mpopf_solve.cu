// Factorisation and solve of the condensed matrix M by a library sparse
// Cholesky (Sec. III-B: the paper factorises M with a sparse direct solver,
// cuDSS).  cuDSS is not available here; cuSOLVER's sparse Cholesky
// (csrchol: analysis once, numeric factorisation and triangular solves on the
// device) stands in.  This file only prepares the library's input: the first
// call orders the symmetrised pattern of M (METIS nested dissection, host),
// builds the permuted full CSR pattern B = P M P^T with a gather map from the
// lower CSR values of M, and runs the library's symbolic analysis; every
// factorisation gathers the values of B (one kernel) and calls the library.
#include <algorithm>
#include <string>
#include <vector>

#pragma GCC diagnostic push
#pragma GCC diagnostic ignored "-Wdeprecated-declarations"
#include <cusolverSp.h>
#include <cusolverSp_LOWLEVEL_PREVIEW.h>
#include <cusparse.h>

#include "mpopf_internal.cuh"

namespace mpopf {

struct KktSolver {
  cusolverSpHandle_t sp = nullptr;
  cusparseMatDescr_t descr = nullptr;
  csrcholInfo_t info = nullptr;
  int32_t n = 0, nnz = 0;
  int32_t *rowptr = nullptr, *colind = nullptr;  // B = P M P^T, full symmetric, rows sorted
  int32_t *src = nullptr;                        // lower-CSR index of M for each entry of B
  int32_t *perm = nullptr;                       // B row i = M row perm[i]
  double *vals = nullptr, *bperm = nullptr, *xperm = nullptr;
  void *buffer = nullptr;
  bool factored = false;
};

namespace {

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

__global__ void __launch_bounds__(kBlock) k_gather(int32_t nnz, const int32_t *__restrict__ src,
                                                   const double *__restrict__ kv, double *__restrict__ out) {
  const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) out[k] = kv[src[k]];
}

// out[i] = in[perm[i]] (forward) or out[perm[i]] = in[i] (back)
template <bool BACK>
__global__ void __launch_bounds__(kBlock) k_permute(int32_t n, const int32_t *__restrict__ perm,
                                                    const double *__restrict__ in, double *__restrict__ out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (BACK) out[perm[i]] = in[i];
  else out[i] = in[perm[i]];
}

unsigned grid_for(int64_t count) { return (unsigned)((count + kBlock - 1) / kBlock); }

const char *sp_status(cusolverStatus_t s) {
  switch (s) {
    case CUSOLVER_STATUS_SUCCESS: return "success";
    case CUSOLVER_STATUS_NOT_INITIALIZED: return "not initialized";
    case CUSOLVER_STATUS_ALLOC_FAILED: return "allocation failed";
    case CUSOLVER_STATUS_INVALID_VALUE: return "invalid value";
    case CUSOLVER_STATUS_ARCH_MISMATCH: return "architecture mismatch";
    case CUSOLVER_STATUS_INTERNAL_ERROR: return "internal error";
    case CUSOLVER_STATUS_MATRIX_TYPE_NOT_SUPPORTED: return "matrix type not supported";
    default: return "cusolver error";
  }
}

template <class T>
cudaError_t upload(const std::vector<T> &v, T **dst) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(v.size(), 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  *dst = static_cast<T *>(p);
  if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Ordering, permuted pattern and symbolic analysis (first call).
int build(mpopf_handle *h, KktSolver *S) {
  const mpopf_pattern &P = h->pat;
  const int64_t n = P.n, nnzl = P.nnz_kkt;
  if (2 * nnzl - n >= ((int64_t)1 << 31)) return fail(MPOPF_ERR_SIZE, "mpopf_kkt_factor: M too large for int32");
  std::vector<int64_t> lrp(n + 1);
  std::vector<int32_t> lci(nnzl);
  cudaError_t e = cudaMemcpy(lrp.data(), P.kkt_rowptr, (n + 1) * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && nnzl) e = cudaMemcpy(lci.data(), P.kkt_col, nnzl * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_kkt_factor: ") + cudaGetErrorString(e));
  // full symmetric pattern of M (row-sorted), each entry with its lower index
  std::vector<int32_t> cnt(n + 1, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = lrp[i]; k < lrp[i + 1]; ++k) {
      ++cnt[i + 1];
      if (lci[k] != i) ++cnt[lci[k] + 1];
    }
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  const int64_t nnz = cnt[n];
  std::vector<int32_t> fci(nnz), fsrc(nnz), fill(cnt.begin(), cnt.end() - 1);
  // rows ascending; within a row, columns from lower entries of that row come in
  // ascending order, then transposed entries (i < col) also ascending
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = lrp[i]; k < lrp[i + 1]; ++k) {
      const int32_t j = lci[k];
      fci[fill[i]] = j;
      fsrc[fill[i]++] = (int32_t)k;
      if (j != i) {
        fci[fill[j]] = (int32_t)i;
        fsrc[fill[j]++] = (int32_t)k;
      }
    }
  // each row is the merge of two ascending runs: sort rows by column
  for (int64_t i = 0; i < n; ++i) {
    std::vector<std::pair<int32_t, int32_t>> row;
    row.reserve(cnt[i + 1] - cnt[i]);
    for (int64_t k = cnt[i]; k < cnt[i + 1]; ++k) row.push_back({fci[k], fsrc[k]});
    std::sort(row.begin(), row.end());
    for (int64_t k = cnt[i]; k < cnt[i + 1]; ++k) { fci[k] = row[k - cnt[i]].first; fsrc[k] = row[k - cnt[i]].second; }
  }
  cusolverStatus_t st = cusolverSpCreate(&S->sp);
  if (st == CUSOLVER_STATUS_SUCCESS && cusparseCreateMatDescr(&S->descr) != CUSPARSE_STATUS_SUCCESS)
    st = CUSOLVER_STATUS_INTERNAL_ERROR;
  if (st == CUSOLVER_STATUS_SUCCESS) {
    cusparseSetMatType(S->descr, CUSPARSE_MATRIX_TYPE_GENERAL);
    cusparseSetMatIndexBase(S->descr, CUSPARSE_INDEX_BASE_ZERO);
  }
  // fill-reducing ordering (METIS nested dissection on the host)
  std::vector<int32_t> p(n);
  if (st == CUSOLVER_STATUS_SUCCESS)
    st = cusolverSpXcsrmetisndHost(S->sp, (int)n, (int)nnz, S->descr, cnt.data(), fci.data(), nullptr, p.data());
  if (st != CUSOLVER_STATUS_SUCCESS) return fail(MPOPF_ERR_CUDA, std::string("mpopf_kkt_factor: ordering: ") + sp_status(st));
  // B = P M P^T: row i of B is row p[i] of M, column j of B is column p[j]
  std::vector<int32_t> inv(n);
  for (int64_t i = 0; i < n; ++i) inv[p[i]] = (int32_t)i;
  std::vector<int32_t> brp(n + 1, 0), bci(nnz), bsrc(nnz);
  for (int64_t i = 0; i < n; ++i) brp[i + 1] = brp[i] + (cnt[p[i] + 1] - cnt[p[i]]);
  for (int64_t i = 0; i < n; ++i) {
    std::vector<std::pair<int32_t, int32_t>> row;
    const int64_t r = p[i];
    for (int64_t k = cnt[r]; k < cnt[r + 1]; ++k) row.push_back({inv[fci[k]], fsrc[k]});
    std::sort(row.begin(), row.end());
    for (size_t k = 0; k < row.size(); ++k) { bci[brp[i] + k] = row[k].first; bsrc[brp[i] + k] = row[k].second; }
  }
  S->n = (int32_t)n;
  S->nnz = (int32_t)nnz;
  e = upload(brp, &S->rowptr);
  if (e == cudaSuccess) e = upload(bci, &S->colind);
  if (e == cudaSuccess) e = upload(bsrc, &S->src);
  if (e == cudaSuccess) e = upload(p, &S->perm);
  if (e == cudaSuccess) e = cudaMalloc(&S->vals, std::max<int64_t>(nnz, 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&S->bperm, std::max<int64_t>(n, 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&S->xperm, std::max<int64_t>(n, 1) * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_ALLOC, std::string("mpopf_kkt_factor: ") + cudaGetErrorString(e));
  }
  st = cusolverSpCreateCsrcholInfo(&S->info);
  if (st == CUSOLVER_STATUS_SUCCESS)
    st = cusolverSpXcsrcholAnalysis(S->sp, S->n, S->nnz, S->descr, S->rowptr, S->colind, S->info);
  size_t internal = 0, work = 0;
  if (st == CUSOLVER_STATUS_SUCCESS)
    st = cusolverSpDcsrcholBufferInfo(S->sp, S->n, S->nnz, S->descr, S->vals, S->rowptr, S->colind, S->info,
                                      &internal, &work);
  if (st != CUSOLVER_STATUS_SUCCESS)
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_kkt_factor: analysis: ") + sp_status(st));
  e = cudaMalloc(&S->buffer, std::max<size_t>(work, 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MPOPF_ERR_ALLOC, std::string("mpopf_kkt_factor: workspace: ") + cudaGetErrorString(e));
  }
  return MPOPF_OK;
}

}  // namespace

void kkt_solver_destroy(mpopf_handle *h) {
  KktSolver *S = h->solver;
  if (!S) return;
  if (S->info) cusolverSpDestroyCsrcholInfo(S->info);
  if (S->descr) cusparseDestroyMatDescr(S->descr);
  if (S->sp) cusolverSpDestroy(S->sp);
  for (void *p : {(void *)S->rowptr, (void *)S->colind, (void *)S->src, (void *)S->perm, (void *)S->vals,
                  (void *)S->bperm, (void *)S->xperm, S->buffer})
    if (p) cudaFree(p);
  delete S;
  h->solver = nullptr;
}

}  // namespace mpopf

using namespace mpopf;

extern "C" {

int mpopf_kkt_factor(mpopf_handle *h, const double *kv, int64_t *zero_pivot, void *stream) {
  if (!h || !kv) return fail(MPOPF_ERR_ARG, "mpopf_kkt_factor: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_kkt_factor: not available on a period shard");
  if (zero_pivot) *zero_pivot = -1;
  if (!h->solver) {
    h->solver = new KktSolver();
    const int rc = build(h, h->solver);
    if (rc != MPOPF_OK) {
      kkt_solver_destroy(h);
      return rc;
    }
  }
  KktSolver &S = *h->solver;
  S.factored = false;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cusolverStatus_t cs = cusolverSpSetStream(S.sp, st);
  if (S.nnz > 0) k_gather<<<grid_for(S.nnz), kBlock, 0, st>>>(S.nnz, S.src, kv, S.vals);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_kkt_factor: ") + cudaGetErrorString(e));
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverSpDcsrcholFactor(S.sp, S.n, S.nnz, S.descr, S.vals, S.rowptr, S.colind, S.info, S.buffer);
  int pos = -1;
  if (cs == CUSOLVER_STATUS_SUCCESS) cs = cusolverSpDcsrcholZeroPivot(S.sp, S.info, 0.0, &pos);
  if (cs != CUSOLVER_STATUS_SUCCESS)
    return fail(MPOPF_ERR_CUDA, std::string("mpopf_kkt_factor: ") + sp_status(cs));
  if (pos >= 0) {
    if (zero_pivot) {
      int32_t row = 0;
      cudaMemcpy(&row, S.perm + pos, 4, cudaMemcpyDeviceToHost);
      *zero_pivot = row;
    }
    return fail(MPOPF_ERR_NUMERIC, "mpopf_kkt_factor: M is not positive definite (zero or negative pivot)");
  }
  S.factored = true;
  return MPOPF_OK;
}

int mpopf_kkt_solve(mpopf_handle *h, const double *rhs, double *dx, void *stream) {
  if (!h || !rhs || !dx) return fail(MPOPF_ERR_ARG, "mpopf_kkt_solve: NULL argument");
  if (mpopf::is_shard(h->d)) return fail(MPOPF_ERR_ARG, "mpopf_kkt_solve: not available on a period shard");
  if (!h->solver || !h->solver->factored)
    return fail(MPOPF_ERR_ARG, "mpopf_kkt_solve: call mpopf_kkt_factor successfully first");
  KktSolver &S = *h->solver;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cusolverStatus_t cs = cusolverSpSetStream(S.sp, st);
  if (S.n > 0) k_permute<false><<<grid_for(S.n), kBlock, 0, st>>>(S.n, S.perm, rhs, S.bperm);
  if (cs == CUSOLVER_STATUS_SUCCESS) cs = cusolverSpDcsrcholSolve(S.sp, S.n, S.bperm, S.xperm, S.info, S.buffer);
  if (S.n > 0) k_permute<true><<<grid_for(S.n), kBlock, 0, st>>>(S.n, S.perm, S.xperm, dx);
  const cudaError_t e = cudaGetLastError();
  if (cs != CUSOLVER_STATUS_SUCCESS) return fail(MPOPF_ERR_CUDA, std::string("mpopf_kkt_solve: ") + sp_status(cs));
  if (e != cudaSuccess) return fail(MPOPF_ERR_CUDA, std::string("mpopf_kkt_solve: ") + cudaGetErrorString(e));
  return MPOPF_OK;
}

}  // extern "C"

#pragma GCC diagnostic pop
