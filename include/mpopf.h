/*
 * mpopf.h -- C ABI of libmpopf: the data-parallel hot path inside each
 * interior-point iteration of the multi-period AC OPF method of
 * arXiv 2405.14032 (Shin, Rao, Schanen, Maldonado, Anitescu), on one NVIDIA
 * B300 (sm_103a).
 *
 * The library evaluates the NLP callbacks of the multi-period AC OPF model
 * (Eq. 1, in the standard form of Eq. 3) and assembles the condensed KKT matrix
 * M = W + delta_w I + Sigma_x + J^T D J of the lifted-KKT interior-point method
 * (Sec. III-B).  All values are IEEE binary64.
 *
 * Conventions (every entry point):
 *   - Device pointers are CUDA device memory owned by the caller unless stated
 *     otherwise; outputs are written, never read.  Pointers must be 8-byte
 *     aligned.  Host pointers are plain host memory (pinned memory makes the
 *     copies of mpopf_sweep_host asynchronous).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Work is enqueued asynchronously on it; nothing synchronises
 *     unless stated.  Calls on one handle must not overlap in time (they share
 *     the handle's scratch buffer).  The evaluation calls run their generator
 *     kernels on a side stream of the handle, forked from `stream` and joined
 *     back into it with events, so work enqueued on `stream` afterwards sees
 *     every output (under stream capture the fork is a parallel graph branch).
 *   - Return value: MPOPF_OK (0) or a negative code; mpopf_last_error() gives a
 *     message (thread-local).  No call allocates device memory except
 *     mpopf_setup (and, once, mpopf_sweep_host for its staging buffers,
 *     mpopf_csc_pattern for a CSC pattern, each on first use).
 *   - Outputs are deterministic: identical inputs give bitwise-identical
 *     outputs (no atomics on values).  There is no CPU fallback: without a
 *     CUDA device every call returns MPOPF_ERR_CUDA.
 *
 * Model layout (0-based; N buses, L branches, G generators, D loads, T periods;
 * arc a = l is the from end of branch l, arc a = L + l its to end):
 *   variables x [n], n = T (2N + 2G + 4L), kind-major then period then component:
 *     va[t][i] at t N + i;  vm at T N + t N + i;  pg at 2TN + t G + g;
 *     qg at 2TN + TG + t G + g;  p[t][a] at 2TN + 2TG + 2tL + a;
 *     q[t][a] at 2TN + 2TG + 2TL + 2tL + a.
 *   constraint rows [m], m = T (1 + 7L + 2N) + G (T - 1) (+ G (T - 1) with K11):
 *     K0  reference angle       t                      va[t][ref]              = 0
 *     K1  from-end P flow      T + 0TL + tL + l        p[t][l]   - P_fr        = 0
 *     K2  from-end Q flow      T + 1TL + tL + l        q[t][l]   - Q_fr        = 0
 *     K3  to-end P flow        T + 2TL + tL + l        p[t][L+l] - P_to        = 0
 *     K4  to-end Q flow        T + 3TL + tL + l        q[t][L+l] - Q_to        = 0
 *     K5  angle difference     T + 4TL + tL + l        va_f - va_t  in [angmin, angmax]
 *     K6  thermal, from end    T + 5TL + tL + l        p^2 + q^2 - smax^2 <= 0
 *     K7  thermal, to end      T + 6TL + tL + l        (arc L + l)
 *     K8  P balance            T + 7TL + tN + n        sum pg - sum p_a - gs vm^2 - sum Pd = 0
 *     K9  Q balance            T + 7TL + TN + tN + n   sum qg - sum q_a + bs vm^2 - sum Qd = 0
 *     K10 P ramp (t >= 1)      T + 7TL + 2TN + (t-1)G + g   pg[t] - pg[t-1] in [-ramp, ramp]
 *     K11 Q ramp (t >= 1)      T + 7TL + 2TN + (T-1)G + (t-1)G + g   qg[t] - qg[t-1] in
 *                              [-qramp, qramp]; only when gen_qramp is given (the
 *                              reactive ramp that Eq. 1 of the paper leaves commented out)
 *   Flows are the pi-model of a branch with series admittance 1/(r + jx),
 *   charging b, tap tau and shift phi (Eq. 1d, 1e print the mutual term only).
 *   Objective (Eq. 1a): f = sum_{t,g} c2 pg^2 + c1 pg + c0.
 *
 * Patterns (fixed at setup, Sec. III-A "pre-analyzed sparsity patterns"):
 *   J (COO): rows ascending; within a row the J order
 *     K0 [va_ref]; K1..K4 [arc, va_f, va_t, vm_f, vm_t]; K5 [va_f, va_t];
 *     K6/K7 [p_a, q_a]; K8 [vm_n, pg of the bus ascending, p_a of the bus
 *     ascending]; K9 the same with qg, q_a; K10 [pg_t, pg_{t-1}];
 *     K11 [qg_t, qg_{t-1}].
 *   W = sigma grad^2 f + sum_i lambda_i grad^2 c_i (Eq. 4), lower COO
 *     (row >= col), duplicates allowed (a consumer sums them), groups in order:
 *     objective (t, g) [pg,pg]; branch (t, l) 10 entries over (va_f, va_t,
 *     vm_f, vm_t) pairs (0,0),(1,0),(1,1),(2,0),(2,1),(2,2),(3,0),(3,1),(3,2),
 *     (3,3); thermal (t, l) [p_from, q_from, p_to, q_to] diagonals; shunt
 *     (t, n) [vm,vm] P part then Q part.
 *   M (CSR, lower incl. the full diagonal): pattern = diag U pattern(W) U
 *     {pairs of columns sharing a J row}; columns ascending in each row.
 *   Sign convention: the caller passes lambda as it appears in W; the paper's
 *     p_x = grad f - J^T y implies lambda = -y.
 */
#ifndef MPOPF_H
#define MPOPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MPOPF_OK = 0,
  MPOPF_ERR_ARG = -1,   /* bad argument (NULL pointer, index out of range, ...) */
  MPOPF_ERR_SIZE = -2,  /* sizes overflow the index types (n, m must be < 2^31) */
  MPOPF_ERR_CUDA = -3,  /* CUDA error (no device, launch failure, ...) */
  MPOPF_ERR_ALLOC = -4,  /* device allocation failed */
  MPOPF_ERR_NUMERIC = -5 /* numerical failure (mpopf_kkt_factor: M not positive definite) */
};

/* Output selection bits for mpopf_eval. */
enum {
  MPOPF_OUT_OBJ = 1,
  MPOPF_OUT_GRAD = 2,
  MPOPF_OUT_CONS = 4,
  MPOPF_OUT_JAC = 8,
  MPOPF_OUT_HESS = 16,
  MPOPF_OUT_KKT = 32,
  MPOPF_OUT_ALL = 63
};

/* Network data (Eq. 1 and its nomenclature), host arrays owned by the caller;
 * mpopf_setup copies them.  Per-unit values.  Requirements: n_bus >= 1,
 * 0 <= ref_bus < n_bus, branch ends in range and distinct (self-loops are
 * rejected), tap != 0, r^2 + x^2 > 0, generator and load buses in range. */
typedef struct {
  int32_t n_bus, n_branch, n_gen, n_load, ref_bus;
  const double *bus_gs, *bus_bs, *bus_vmin, *bus_vmax;          /* [N] */
  const int32_t *br_f, *br_t;                                   /* [L] */
  const double *br_r, *br_x, *br_b, *br_tap, *br_shift;        /* [L] */
  const double *br_smax, *br_angmin, *br_angmax;                /* [L] */
  const int32_t *gen_bus;                                       /* [G] */
  const double *gen_c2, *gen_c1, *gen_c0;                       /* [G] */
  const double *gen_pmin, *gen_pmax, *gen_qmin, *gen_qmax, *gen_ramp; /* [G] */
  const int32_t *load_bus;                                      /* [D] */
  const double *gen_qramp; /* [G] reactive ramp limits (>= 0), or NULL: no K11 rows */
} mpopf_network;

/* Sizes and patterns.  Every pointer is DEVICE memory owned by the handle and
 * valid until mpopf_destroy. */
typedef struct {
  int64_t n, m, nnz_jac, nnz_hess, nnz_kkt;
  int32_t n_bus, n_branch, n_gen, n_load, n_periods;
  const int32_t *jac_row, *jac_col;    /* [nnz_jac] */
  const int32_t *hess_row, *hess_col;  /* [nnz_hess], row >= col */
  const int64_t *kkt_rowptr;           /* [n + 1] */
  const int32_t *kkt_col;              /* [nnz_kkt], ascending, col <= row */
  const double *xl, *xu;               /* [n] variable bounds (Eq. 1g-1i), +-INFINITY if none */
  const double *gl, *gu;               /* [m] row bounds (Eq. 1f, 1j, 1k; equalities 0) */
} mpopf_pattern;

typedef struct mpopf_handle mpopf_handle;

/* Setup (once): validates the network, builds the layout and every pattern
 * (Sec. III-A: sparsity analysed once per pattern, then expanded over the
 * data), uploads network data and the loads pd/qd (host [T][D], row-major; may
 * be NULL when D = 0), and allocates the handle's scratch.  Synchronous.
 * On success *out is a new handle and *pat (may be NULL) its patterns. */
int mpopf_setup(const mpopf_network *net, int32_t n_periods, const double *pd, const double *qd,
                mpopf_handle **out, mpopf_pattern *pat);

/* Period shards: the horizon split into contiguous blocks of periods, one per
 * GPU (Sec. II: only the ramp rows, Eq. 1k, couple periods).
 *
 * A shard owning periods [t0, t1) of a T-period model is the local model of
 * periods [t0 - h0, t1 + h1), h0 = (t0 > 0), h1 = (t1 < T): one halo period
 * before and / or after the owned ones.  Its handle (mpopf_shard_setup)
 * evaluates the owned periods only, with the same kernels and arithmetic as a
 * whole-horizon handle, so every owned output entry equals the whole-horizon
 * model's entry bit for bit, except f, which is the sum over the owned
 * periods only (the whole f is the sum over the shards, a scalar
 * all-reduce).  Inputs and outputs of a shard handle use the local model's
 * layout (T_loc = t1 - t0 + h0 + h1 periods; sizes in the layout below);
 * entries of the halo periods are inputs only (two of them are read, see
 * below) and are never written.  The handle's pattern (mpopf_pattern) is the
 * local model's.  Only mpopf_eval, the callbacks built on it, mpopf_sweep,
 * the schedule, launch-count and profiling calls, mpopf_set_loads and
 * mpopf_get_pattern accept a shard handle; every other entry point returns
 * MPOPF_ERR_ARG for it.
 *
 * The halo exchange of one evaluation (before it; G doubles per block, block
 * 0 = P, block 1 = Q with the reactive ramp K11):
 *   x[x_recv[b] ..] <- the previous shard's x[x_send[b] ..]:  pg (qg) of
 *     period t0 - 1, read by the ramp rows at t0;
 *   dvec[d_recv[b] ..] <- the next shard's dvec[d_send[b] ..]:  D of the ramp
 *     rows at t1, the last term of the pg (qg) diagonals of M at t1 - 1 (the
 *     (pg[t1-1], pg[t1-1]) contribution D * 1 * 1 of those rows);
 * an offset is -1 where the neighbour does not exist.  Nothing else crosses a
 * shard boundary.
 *
 * Ranges map local entries to the whole-horizon model's (count entries from
 * `local` in the shard's array correspond to count entries from `global` in
 * the whole model's array): MPOPF_RANGE_X the owned variables (x, grad,
 * sigma_x), MPOPF_RANGE_XALL every local variable, halo periods included (for
 * mapping pattern columns), MPOPF_RANGE_ROWS the owned rows (c, lam, dvec),
 * MPOPF_RANGE_JAC / _HESS / _KKT the owned values of J, W and M. */
enum {
  MPOPF_RANGE_X = 0,
  MPOPF_RANGE_XALL = 1,
  MPOPF_RANGE_ROWS = 2,
  MPOPF_RANGE_JAC = 3,
  MPOPF_RANGE_HESS = 4,
  MPOPF_RANGE_KKT = 5
};
#define MPOPF_SHARD_MAX_RANGES 64
typedef struct {
  int32_t what;     /* MPOPF_RANGE_* */
  int32_t reserved; /* 0 */
  int64_t local, global, count;
} mpopf_range;
typedef struct {
  int32_t n_periods, t0, t1;       /* whole horizon T; owned periods [t0, t1) */
  int32_t local_periods;           /* T_loc */
  int32_t own0, own1;              /* owned periods in local numbering: [h0, h0 + t1 - t0) */
  int32_t halo_len, halo_blocks;   /* G; 1, or 2 with the reactive ramp */
  int64_t n, m, nnz_jac, nnz_hess, nnz_kkt;  /* sizes of the local model's arrays */
  int64_t x_recv[2], x_send[2];    /* halo offsets into the local x (-1: none) */
  int64_t d_recv[2], d_send[2];    /* halo offsets into the local dvec (-1: none) */
  int32_t n_ranges;
  int32_t reserved;
  mpopf_range ranges[MPOPF_SHARD_MAX_RANGES];
} mpopf_shard_layout;

/* Layout of the shard [t0, t1) of a T-period model: host computation only (no
 * device needed), validates the network like mpopf_setup.  MPOPF_ERR_ARG
 * unless 0 <= t0 < t1 <= n_periods. */
int mpopf_shard_plan(const mpopf_network *net, int32_t n_periods, int32_t t0, int32_t t1, mpopf_shard_layout *plan);
/* Handle of the shard [t0, t1): like mpopf_setup for the local model; pd, qd
 * are the loads of the WHOLE horizon (host [n_periods][D]), of which the
 * local periods' rows are copied. */
int mpopf_shard_setup(const mpopf_network *net, int32_t n_periods, int32_t t0, int32_t t1, const double *pd,
                      const double *qd, mpopf_handle **out, mpopf_pattern *pat);

/* Pattern of an existing handle. */
int mpopf_get_pattern(const mpopf_handle *h, mpopf_pattern *pat);

/* Replace the per-period loads (Eq. 1b, 1c right-hand sides) from DEVICE
 * arrays d_pd, d_qd [T][D]; stream-ordered copy into the handle. */
int mpopf_set_loads(mpopf_handle *h, const double *d_pd, const double *d_qd, void *stream);

/* Evaluation at x [n] (device).  Each output pointer may be NULL (skipped);
 * `outputs` selects with MPOPF_OUT_* bits which non-NULL outputs to compute.
 *   f       [1]          objective (Eq. 1a); deterministic tree reduction
 *   grad    [n]          gradient of f
 *   c       [m]          constraint values
 *   jv      [nnz_jac]    J values in the COO order of the pattern
 *   hv      [nnz_hess]   W values (needs lam [m], sigma)
 *   kv      [nnz_kkt]    M = W + diag(sigma_x + delta_w) + J^T diag(dvec) J
 *                        (Sec. III-B condensed matrix; needs lam, sigma,
 *                        sigma_x [n], dvec [m], delta_w)
 * Reads x, lam, sigma_x, dvec once; computes each product once.  */
int mpopf_eval(mpopf_handle *h, unsigned outputs, const double *x, const double *lam, double sigma,
               const double *sigma_x, const double *dvec, double delta_w, double *f, double *grad, double *c,
               double *jv, double *hv, double *kv, void *stream);

/* The individual callbacks (each = mpopf_eval with one output bit). */
int mpopf_eval_obj(mpopf_handle *h, const double *x, double *f, void *stream);
int mpopf_eval_grad(mpopf_handle *h, const double *x, double *grad, void *stream);
int mpopf_eval_cons(mpopf_handle *h, const double *x, double *c, void *stream);
int mpopf_eval_jac(mpopf_handle *h, const double *x, double *jv, void *stream);
int mpopf_eval_hess(mpopf_handle *h, const double *x, const double *lam, double sigma, double *hv, void *stream);
int mpopf_assemble_kkt(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *sigma_x,
                       const double *dvec, double delta_w, double *kv, void *stream);

/* Full sweep: all six outputs in one pass (= mpopf_eval with MPOPF_OUT_ALL). */
int mpopf_sweep(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *sigma_x,
                const double *dvec, double delta_w, double *f, double *grad, double *c, double *jv, double *hv,
                double *kv, void *stream);

/* Full sweeps of one network at k points (iterates: a line search's trial
 * points, perturbed iterates, scenarios of the same network) in one launch of
 * each sweep kernel over all k points (Eq. 3, 4, 6 at every point).  Point j's
 * inputs and outputs are the j-th of k consecutive arrays of mpopf_sweep's
 * sizes, all on the device: x [k][n], lam [k][m], sigma_x [k][n], dvec [k][m];
 * f [k], grad [k][n], c [k][m], jv [k][nnz_jac], hv [k][nnz_hess],
 * kv [k][nnz_kkt]; sigma and delta_w are shared by the k points.  Each point's
 * outputs equal mpopf_sweep's at that point bit for bit.  1 <= k <= 65535.
 * When the k points' branch elements span at least two waves of the device
 * (k T L >= 2 x SMs x 768), the bus-end products D8 (m2gs vm), D9 (p2bs vm)
 * are formed in a launch of their own first, as MPOPF_SCHED_BUS_TERMS does
 * for a single sweep.  Scratch for the points' incidence records, objective
 * partials and those products (k x (2 L T x 48 + 8 ceil(T G / 256)
 * [+ 16 T N]) bytes) is allocated by the first
 * call that needs more than the handle holds (after a device-wide
 * synchronisation when it replaces a smaller one) and kept by the handle;
 * calls on one handle must not overlap.  MPOPF_ERR_ARG for a NULL buffer, k
 * outside the range, a shard handle, or a call under stream capture that
 * would have to grow the scratch (make one call of that size first);
 * MPOPF_ERR_ALLOC when the scratch cannot be allocated. */
int mpopf_sweep_points(mpopf_handle *h, int32_t k, const double *x, const double *lam, double sigma,
                       const double *sigma_x, const double *dvec, double delta_w, double *f, double *grad, double *c,
                       double *jv, double *hv, double *kv, void *stream);

/* Full sweep from HOST buffers: copies x, lam, sigma_x, dvec to the device,
 * runs the sweep and copies all six outputs back to the host buffers; returns
 * when the outputs are in the host buffers.  The horizon is processed in up to
 * eight windows of periods: the inputs of a window are copied in on one
 * internal stream, its branch and bus work runs on `stream`, and its outputs
 * are copied out on a second internal stream, so copies in both directions
 * overlap each other and the kernels (with pinned host buffers); the generator
 * work and the objective run last, over the whole horizon.  The outputs equal
 * those of mpopf_sweep bit for bit.  Staging buffers, the two streams and
 * their events are created on the first call and kept by the handle. */
int mpopf_sweep_host(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *sigma_x,
                     const double *dvec, double delta_w, double *f, double *grad, double *c, double *jv,
                     double *hv, double *kv, void *stream);

/* Matrix-free derivative products (no J or W is materialised).  Each value
 * follows the same element-by-element order as the condensed matrix: an
 * element's local sum over its rows (J order), then the elements in order.
 *
 * mpopf_vjp: gx [n] = J^T y for y [m] (device); optionally the load adjoint
 *   gpd, gqd [T][D] = (dc/dPd)^T y, (dc/dQd)^T y = -y at the P / Q balance row
 *   of the load's bus (Eq. 1b, 1c); pass both or neither (NULL).
 * mpopf_jvp: out [m] = J v for v [n]; with load tangents dpd, dqd [T][D] (both
 *   or neither) the balance rows also get -sum_d dpd[t][d] (Q likewise), i.e.
 *   the tangent of c(x, Pd, Qd).
 * mpopf_hvp: hv [n] = W v, W = sigma grad^2 f + sum_i lambda_i grad^2 c_i
 *   (Eq. 4) for lam [m], v [n].
 * All use the handle's scratch (calls on one handle must not overlap). */
int mpopf_vjp(mpopf_handle *h, const double *x, const double *y, double *gx, double *gpd, double *gqd, void *stream);
/* The same products with J's values as mpopf_eval_jac / mpopf_sweep wrote them
 * at the same x (jv [nnz_jac], device; NULL: recompute, as above): the branch
 * rows are read instead of recomputed (no sin/cos, about a quarter of the FP64
 * work), with bit-for-bit the same results. */
int mpopf_vjp_jv(mpopf_handle *h, const double *x, const double *jv, const double *y, double *gx, double *gpd,
                 double *gqd, void *stream);
int mpopf_jvp_jv(mpopf_handle *h, const double *x, const double *jv, const double *v, const double *dpd,
                 const double *dqd, double *jv_out, void *stream);
int mpopf_jvp(mpopf_handle *h, const double *x, const double *v, const double *dpd, const double *dqd, double *jv_out,
              void *stream);
int mpopf_hvp(mpopf_handle *h, const double *x, const double *lam, double sigma, const double *v, double *hv,
              void *stream);
/* The same products for k vectors at one point, each kernel launched once
 * over all k (1 <= k <= 65535).  Vector j's input and output are the j-th of
 * k consecutive arrays of the single product's sizes, all on the device:
 *   mpopf_vjp_many: y [k][m] -> gx [k][n], gpd, gqd [k][T][D] (both or NULL);
 *   mpopf_jvp_many: v [k][n], dpd, dqd [k][T][D] (both or NULL) -> out [k][m];
 *   mpopf_hvp_many: v [k][n] -> hv [k][n].
 * jv [nnz_jac] / hw [nnz_hess] (NULL: recompute): J's / W's values at the
 * same x (and lam, sigma) as mpopf_eval_jac / _hess or mpopf_sweep wrote
 * them, read by the branch elements instead of recomputed.  Each vector's
 * result equals the single product's (mpopf_vjp_jv, mpopf_jvp_jv, mpopf_hvp)
 * bit for bit.  mpopf_vjp_many and mpopf_hvp_many keep their incidence
 * records (k x 2 L T x 16 bytes) in the handle's scratch, grown like
 * mpopf_sweep_points's (shared with it); calls on one handle must not
 * overlap.  MPOPF_ERR_ARG for a NULL argument, k outside the range, a shard
 * handle or a scratch that would have to grow under stream capture;
 * MPOPF_ERR_ALLOC when the scratch cannot be allocated. */
int mpopf_vjp_many(mpopf_handle *h, int32_t k, const double *x, const double *jv, const double *y, double *gx,
                   double *gpd, double *gqd, void *stream);
int mpopf_jvp_many(mpopf_handle *h, int32_t k, const double *x, const double *jv, const double *v,
                   const double *dpd, const double *dqd, double *out, void *stream);
int mpopf_hvp_many(mpopf_handle *h, int32_t k, const double *x, const double *lam, double sigma, const double *hw,
                   const double *v, double *hv, void *stream);

/* Interior-point algebra around the condensed matrix (Sec. III-B, Eq. 5).
 * x [n] is the point, s [m] the slacks of the rows g(x) - s = 0, y [m] the
 * multipliers, zl_x/zu_x [n] and zl_s/zu_s [m] the bound duals, all device
 * arrays owned by the caller.  Bounds come from the pattern: x in [xl, xu];
 * s in [gl, gu] for inequality rows and in [gl - eps_tol, gu + eps_tol] for
 * equality rows (gl == gu), the paper's relaxation of g(x) = 0 to a band of
 * half-width eps.  A +-INFINITY bound contributes nothing and its dual is
 * ignored.  Precondition: every finite bound is strictly inactive (v strictly
 * inside, at a finite distance).
 * With rl = 1/(v - lo), ru = 1/(hi - v) (0 for an infinite bound), v in {x, s}:
 *   Sigma = zl rl + zu ru,  C = 1/(1 + delta_c (Sigma_s + delta_w)),
 *   D = (Sigma_s + delta_w) C.
 * mpopf_ipm_prepare: sigma_x [n], dvec = D [m], cvec = C [m] (sigma_x and dvec
 *   are the Sigma_x and D that mpopf_assemble_kkt / mpopf_sweep take) and the
 *   workspace recip [2n + 2m] = rl_x [n], ru_x [n], rl_s [m], ru_s [m], which
 *   the two calls below read.  All divisions of the algebra happen here.
 * mpopf_ipm_rhs: rhs [n] = q_x + A^T (C q_s + D q_y) with A = J(x); after
 *   eliminating the bound-dual rows of Eq. 5 the dual terms cancel and
 *   q_x = grad f - A^T y + mu (ru_x - rl_x),  q_s = y + mu (ru_s - rl_s),
 *   q_y = c - s; grad [n] = grad f(x) and c [m] = c(x) as the eval callbacks
 *   return them; recip, dvec, cvec from mpopf_ipm_prepare at the same point.
 *   The two transposed products are merged into one J^T w,
 *   w = C q_s + D q_y - y, kept in the handle's scratch.  With the Lagrangian
 *   f - y^T c the Hessian block of M is W at lambda = -y, sigma = 1, and dx
 *   solves M dx = rhs, the condensed form of Eq. 5 with its right-hand side as
 *   printed.
 * mpopf_ipm_recover: from dx [n] the remaining blocks of Eq. 5:
 *   ds = C (A dx + delta_c q_s - q_y),  dy = (Sigma_s + delta_w) ds - q_s,
 *   dzl = zl - rl (mu + zl dv),  dzu = zu - ru (mu - zu dv)   (v = x, s; dv = dx, ds)
 *   into ds, dy, dzl_s, dzu_s [m] and dzl_x, dzu_x [n] (0 where the bound is
 *   infinite); recip and cvec from mpopf_ipm_prepare at the same point.  The
 *   recovered ds is the one that solves Eq. 5; the sign of A dx printed with
 *   the recovery formula does not.
 * jv (rhs, recover; may be NULL): the J values [nnz_jac] the sweep wrote at the
 *   same x; with them the J products read J (mpopf_vjp_jv / mpopf_jvp_jv)
 *   instead of recomputing its branch rows, with identical results.
 * Values follow a fixed rounding order and equal the CPU reference bit for
 * bit.  rhs and recover use the handle's scratch (calls on one handle must
 * not overlap).  Errors: MPOPF_ERR_ARG for a NULL pointer (nothing is
 * launched), MPOPF_ERR_CUDA for a failed launch. */
int mpopf_ipm_prepare(mpopf_handle *h, const double *x, const double *s, const double *zl_x, const double *zu_x,
                      const double *zl_s, const double *zu_s, double delta_w, double delta_c, double eps_tol,
                      double *sigma_x, double *dvec, double *cvec, double *recip, void *stream);
int mpopf_ipm_rhs(mpopf_handle *h, const double *x, const double *jv, const double *s, const double *y,
                  const double *grad, const double *c, const double *recip, const double *dvec, const double *cvec,
                  double mu, double *rhs, void *stream);
int mpopf_ipm_recover(mpopf_handle *h, const double *x, const double *jv, const double *s, const double *y,
                      const double *zl_x, const double *zu_x, const double *zl_s, const double *zu_s,
                      const double *c, const double *recip, const double *cvec, const double *dx, double mu,
                      double delta_w, double delta_c, double *ds, double *dy, double *dzl_x, double *dzu_x,
                      double *dzl_s, double *dzu_s, void *stream);

/* COO -> CSC compression of J (m x n) and of the lower-triangle W (n x n)
 * (Sec. III-A: the COO matrices may be compressed to CSC).  CSC entries are
 * ordered by column, then row; entries of the COO pattern with the same
 * (row, column) (W has them: the groups of its pattern overlap on diagonals)
 * become one CSC entry holding their sum, added in COO order starting from the
 * first.  J has no duplicates, so its CSC values are a permutation.
 * mpopf_csc_pattern: fills *out with device pointers owned by the handle
 *   (valid until mpopf_destroy): colptr [n + 1] (int64), rowidx [nnz] (int32).
 *   The first call for a matrix builds the pattern (on the device: column
 *   counts, a scan, a scatter and a sort of each column by row and COO entry;
 *   device allocation, synchronous); later calls return it.
 * mpopf_coo_to_csc: csc_vals [nnz] from coo_vals [nnz_jac or nnz_hess] (the
 *   values mpopf_eval_jac / mpopf_eval_hess write), device arrays, asynchronous
 *   on the stream; MPOPF_ERR_ARG if the pattern was not built first.
 * which: MPOPF_CSC_JAC or MPOPF_CSC_HESS (MPOPF_ERR_ARG otherwise); a matrix
 * with 2^31 or more COO entries gets MPOPF_ERR_SIZE. */
enum { MPOPF_CSC_JAC = 0, MPOPF_CSC_HESS = 1 };
typedef struct {
  int64_t nnz;
  const int64_t *colptr; /* [n + 1] */
  const int32_t *rowidx; /* [nnz], ascending within a column */
} mpopf_csc;
int mpopf_csc_pattern(mpopf_handle *h, int32_t which, mpopf_csc *out);
int mpopf_coo_to_csc(mpopf_handle *h, int32_t which, const double *coo_vals, double *csc_vals, void *stream);

/* Factorisation and solve of the condensed matrix M (Sec. III-B: the paper
 * factorises M with the sparse direct solver cuDSS; cuDSS is not available
 * here, so cuSOLVER's sparse Cholesky stands in: a library step, not one of
 * this library's kernels).
 * mpopf_kkt_factor: kv [nnz_kkt] are the lower CSR values of M on the device
 *   (mpopf_assemble_kkt / mpopf_sweep).  The first call orders the symmetrised
 *   pattern (METIS nested dissection, host), builds the permuted full pattern
 *   and runs the symbolic analysis (synchronous, allocates); every call
 *   gathers the values (one kernel) and runs the numeric Cholesky
 *   factorisation on the device, then checks for a zero pivot (synchronous).
 *   Returns MPOPF_ERR_NUMERIC when M is not positive definite (the caller
 *   raises delta_w, as an interior-point inertia correction does); then
 *   *zero_pivot (if not NULL) is the row of M where it was found, else -1.
 * mpopf_kkt_solve: dx [n] = M^{-1} rhs [n] with the last successful
 *   factorisation (MPOPF_ERR_ARG if there is none); asynchronous.
 * Values are the library's (within its rounding; not bitwise against the CPU
 * reference). */
int mpopf_kkt_factor(mpopf_handle *h, const double *kv, int64_t *zero_pivot, void *stream);
int mpopf_kkt_solve(mpopf_handle *h, const double *rhs, double *dx, void *stream);

/* Batched full sweeps of many independent instances (uneven sizes and
 * horizons) in one CUDA graph: one or two persistent kernel launches over a
 * work list of every instance's tiles, or the instances' plain sweeps on
 * parallel branches of the graph (the schedule decides).  The
 * paper evaluates one model per solver; this runs many, e.g. scenario or
 * rolling-horizon instances, with the same values as mpopf_sweep on each.
 *
 * mpopf_batch_create: the handles (same device, each at most once, kept alive
 *   by the caller until mpopf_batch_destroy) become one batch; allocates the
 *   work list and the graph (setup time); MPOPF_ERR_ARG for a NULL, repeated
 *   or shard handle.
 * mpopf_batch_set_io: per-instance DEVICE pointers (host array of k
 *   descriptors, copied; synchronises `stream`).
 * mpopf_batch_sweep: one graph launch on `stream`: every instance's f, grad, c,
 *   J, W and M, bitwise equal to mpopf_sweep on that instance.
 * mpopf_batch_set_schedule / _get_schedule: instance order in the work list
 *   (0 as given, 1 largest first), tile size (CTA-sized chunks per work item,
 *   1..64), persistent CTAs per SM (0 = the occupancy maximum), periods per
 *   dependency chunk (0 = the whole horizon; with P > 0 the bus work of a chunk
 *   of P periods waits only for that chunk's branch work and overlaps the
 *   next chunk's), and launches: 1 = one persistent launch (bus work waits
 *   for its branch work), 2 = two persistent launches in the graph, the first
 *   with every branch tile (the sweep's 64-thread CTAs), the second with every
 *   generator tile, bus tile and objective (bus tiles do not wait; objectives
 *   wait for their generator tiles; run at the bus work's own occupancy; CTAs
 *   per SM and P are not used), 0 = no persistent launch: each instance's
 *   plain sweep (mpopf_sweep's launches, on the handle's own side stream and
 *   schedule) on one of S parallel branches of the graph, instances dealt
 *   round-robin in the order, S = the CTAs-per-SM argument (1..64, 0 = 16),
 *   tile and P not used; the graph is captured again by mpopf_batch_set_io;
 *   sched[5] = (order, tile, CTAs per SM or S, P, launches).
 * mpopf_batch_tune: times candidate schedules (coordinate search; reps graph
 *   launches each, CUDA events on `stream`) and keeps the fastest; *best_ms its
 *   time per sweep.
 * mpopf_batch_status: synchronises the device; MPOPF_ERR_CUDA if a work item's
 *   dependency wait (bounded, ~1 s) ran out in the last launch (each launch
 *   clears the flag with the counters). */
typedef struct mpopf_batch mpopf_batch;
typedef struct {
  const double *x, *lam, *sigma_x, *dvec;   /* device, [n] [m] [n] [m] of that instance */
  double sigma, delta_w;
  double *f, *grad, *c, *jv, *hv, *kv;      /* device outputs */
} mpopf_batch_io;
int mpopf_batch_create(mpopf_handle *const *hs, int32_t k, mpopf_batch **out);
int mpopf_batch_set_io(mpopf_batch *b, const mpopf_batch_io *io, void *stream);
int mpopf_batch_sweep(mpopf_batch *b, void *stream);
int mpopf_batch_set_schedule(mpopf_batch *b, int32_t order, int32_t tile_chunks, int32_t ctas_per_sm,
                             int32_t chunk_periods, int32_t launches);
int mpopf_batch_get_schedule(const mpopf_batch *b, int32_t *sched /* [5] */, int32_t *grid, int32_t *n_items);
int mpopf_batch_tune(mpopf_batch *b, void *stream, int32_t reps, double *best_ms);
int mpopf_batch_status(mpopf_batch *b);
/* Failure-path test hook (one-launch schedules; with two launches or plain
 * sweeps nothing waits and the hook returns MPOPF_ERR_ARG).  on != 0 raises the dependency
 * target of the first bus tile that waits, so that its wait can never be met: the next sweep waits
 * out the bounded limit (about a second), sets the error flag, computes the
 * tile anyway and finishes; mpopf_batch_status then returns MPOPF_ERR_CUDA.
 * on == 0 restores the target (so do mpopf_batch_set_schedule and _tune).
 * Nothing faults or hangs; this exists to test that error path. */
int mpopf_batch_test_stall(mpopf_batch *b, int32_t on);
void mpopf_batch_destroy(mpopf_batch *b);

/* Number of kernel launches one mpopf_eval call with these output bits makes
 * under the handle's current schedule (outside per-kernel profiling, which
 * runs the unsplit launches without the programmatic dependencies). */
int mpopf_launch_count(const mpopf_handle *h, unsigned outputs);

/* Launch schedule of the evaluation calls of a handle (a performance setting;
 * the outputs are the same bit for bit under every schedule).
 * chunk_periods = 0: one branch x period launch, then one bus x period launch
 * on `stream` (the generator work on the handle's side stream).  P > 0: the
 * horizon is cut into chunks of P periods (at most 64 chunks; P grows when T
 * needs more); the branch kernel of each chunk runs on `stream` and the bus
 * kernel of the same chunk on a second internal stream, behind an event
 * recorded after that branch launch, so the bus work of one chunk overlaps
 * the branch work of the next while the chunk's intermediate per-branch
 * records are still in L2.  flags: MPOPF_SCHED_BUS_PRIORITY puts the second
 * stream at the device's highest stream priority (its CTAs are dispatched
 * first as SMs free up); MPOPF_SCHED_GEN_FIRST forks the generator work
 * before the first branch chunk instead of after the last.  Both streams join
 * `stream` before the call returns, so work enqueued on `stream` afterwards
 * sees every output (under stream capture they are parallel graph branches).
 * MPOPF_SCHED_PDL (with P = 0; every default schedule is P = 0 with this flag):
 * the bus kernel is launched with programmatic stream serialization, so its
 * CTAs may be scheduled while the branch kernel's last CTAs run; it waits
 * (griddepcontrol.wait) for the branch kernel's completion before reading its
 * records.
 * MPOPF_SCHED_SPLIT_BUS (with P = 0): the bus work as two kernels after the
 * branch kernel, side by side: the balance rows with their J rows, the shunt W
 * entries, the gradient zeros and the reference row on the internal second
 * stream, the va / vm rows of M on `stream`.
 * MPOPF_SCHED_BUS_TERMS (with P = 0; full sweeps): the products D8 (m2gs vm)
 * and D9 (p2bs vm) of the condensed matrix's arc rows, which the branch kernel
 * would form at both ends of every branch, are formed once per bus and period
 * by a small kernel launched before it (into a 2 T N-double scratch of the
 * handle; the same operations, so the same values); with MPOPF_SCHED_PDL the
 * branch kernel is its programmatic dependent launch.  A new handle starts
 * with MPOPF_SCHED_PDL, plus MPOPF_SCHED_BUS_TERMS when its branch x period
 * launch has at least twice as many elements as the device holds resident
 * (2 x SMs x 768); mpopf_get_sweep_schedule reports it.
 * Per-kernel profiling (mpopf_profile_start) times unchunked, unsplit launches
 * without programmatic dependencies.
 * MPOPF_ERR_ARG for P < 0 or unknown flags. */
enum { MPOPF_SCHED_BUS_PRIORITY = 1, MPOPF_SCHED_GEN_FIRST = 2, MPOPF_SCHED_PDL = 4, MPOPF_SCHED_SPLIT_BUS = 8,
       MPOPF_SCHED_BUS_TERMS = 16 };
int mpopf_set_sweep_schedule(mpopf_handle *h, int32_t chunk_periods, int32_t flags);

/* An extra dependency of the generator work (generator x period kernel and
 * objective) of later evaluations of this handle: it also waits for `event`
 * (a cudaEvent_t passed as void*, owned and recorded by the caller; NULL
 * removes the dependency).  Only the generator work reads a period shard's
 * halo values (pg of period t0 - 1 and D of the ramp rows at t1), so a caller
 * can run the halo exchange on a stream of its own, record the event after it
 * and enqueue the evaluation at once: the branch and bus work then overlap
 * the exchange.  The event must be recorded before each evaluation is
 * enqueued; it is not meant for work recorded in a stream capture. */
int mpopf_set_gen_dependency(mpopf_handle *h, void *event);
int mpopf_get_sweep_schedule(const mpopf_handle *h, int32_t *chunk_periods, int32_t *flags);

/* Condensed-matrix assembly that allocates nothing (the paper has no
 * counterpart: this is a deployment variant of mpopf_assemble_kkt).  For
 * callers that cannot call cudaMalloc once they are running: processes that
 * reserve all device memory up front and forbid later allocation (real-time
 * controllers, serving processes with pooled memory) and plugins inside a host
 * application that owns the device's memory.
 * Same inputs, output and values as mpopf_assemble_kkt; the per-branch scratch
 * it needs lives in a fixed 32 MiB array inside the library's device image
 * (held by every GPU that loads the library until exit) instead of the
 * handle.  Limit: 12 T L <= 4 Mi doubles (T x L <= 349525 branch-periods);
 * larger problems return MPOPF_ERR_SIZE.  The handle's device must be current
 * (MPOPF_ERR_ARG otherwise).  The first call on each device looks up the
 * array's address (cudaGetSymbolAddress, no allocation) and must come before
 * any stream capture; later calls look it up again, except on a capturing
 * stream, where the address found earlier on that device is used.  All calls
 * on a device share the array, which keeps the last call's contents (every
 * record read is first rewritten, so no clearing is needed); calls that
 * overlap on the GPU race on it. */
int mpopf_assemble_kkt_noalloc(mpopf_handle *h, const double *x, const double *lam, double sigma,
                               const double *sigma_x, const double *dvec, double delta_w, double *kv, void *stream);

/* FP64 issue-rate probe (instrumentation for the roofline of the FP64-bound
 * kernels, not part of the paper's method): a kernel of eight independent
 * chains of fused multiply-adds per thread, eight 256-thread CTAs per SM, each
 * thread running `iters` iterations (8 fma each) on the current device.  One
 * warm-up launch, then the best of three timed with CUDA events.  Writes
 * *inst_per_s = FP64 thread-instructions (fma) per second and, if not NULL,
 * *seconds = the best launch's duration.  Allocates (and frees) a small output
 * buffer and a stream; synchronous.  MPOPF_ERR_ARG for iters < 1. */
int mpopf_fp64_issue_rate(int32_t iters, double *inst_per_s, double *seconds);

/* Per-kernel timing (instrumentation for benchmarks, not part of the paper's
 * method).  mpopf_profile_start creates 2 * max_launches CUDA events; every
 * later kernel launch of mpopf_eval on the caller's stream (up to
 * max_launches) is bracketed by an event pair on that stream; the generator
 * kernels, when they run on the handle's side stream, are not timed.  mpopf_profile_stop synchronises on those events,
 * writes the summed milliseconds and launch counts per kernel kind
 * (ms_sum[4], launches[4]: 0 branch x period, 1 bus x period,
 * 2 generator x period, 3 objective reduction; either may be NULL) and
 * releases the events. */
int mpopf_profile_start(mpopf_handle *h, int32_t max_launches);
int mpopf_profile_stop(mpopf_handle *h, double *ms_sum, int32_t *launches);

void mpopf_destroy(mpopf_handle *h);
const char *mpopf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MPOPF_H */
