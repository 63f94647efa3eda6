// Internal layout shared by the setup and the evaluation kernels of libmpopf.
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "mpopf.h"

namespace mpopf {

// Per-branch constants (structure of arrays, [BC_COUNT][L]).
enum {
  BC_GFF, BC_BFF, BC_GFT, BC_BFT, BC_GTF, BC_BTF, BC_GTT, BC_BTT,  // pi-model terms
  BC_G2FF, BC_B2FF, BC_G2TT, BC_B2TT,                              // 2 x self terms
  BC_SMAX2,                                                        // smax^2
  BC_COUNT
};

// Everything a kernel needs, passed by value.
struct Dev {
  int32_t N, L, G, D, T, ref;
  int64_t n, m;
  // variable block starts (va at 0)
  int64_t x_vm, x_pg, x_qg, x_p, x_q;
  // constraint block starts (K0 at 0, K_k (1..7) at T + (k-1) T L)
  int64_t c_k8, c_k9, c_k10;
  // J value starts (K0 at 0, K_k (1..4) at T + 5 (k-1) T L)
  int64_t j_k5, j_k6, j_k7, j_k8, j_k9, j_k10, jk8_per;
  // W value starts (objective at 0)
  int64_t h_br, h_th, h_sh;
  // M: region start of each variable kind and per-period block sizes
  int64_t m_va, m_vm, m_pg, m_qg, m_p, m_q;
  int64_t mb_va, mb_vm, mb_pg0, mb_pg1, mb_qg, mb_p, mb_q;
  int64_t nnz_jac, nnz_hess, nnz_kkt;
  // network
  const int32_t *br_f, *br_t;
  const double *bc;         // [BC_COUNT][L]
  const uint8_t *br_sym;    // 1 if gtf == gft and btf == bft bitwise
  const double *bus_m2gs, *bus_p2bs, *bus_mgs, *bus_bs;
  const int32_t *bgen_ptr, *bgen_idx;    // generators of a bus, ascending
  const int32_t *barc_ptr, *barc_idx;    // arcs of a bus, ascending arc index
  const int32_t *bload_ptr, *bload_idx;  // loads of a bus, ascending
  const int32_t *inc_ptr, *inc_code;     // slots of the bus at position p of bus_order: [inc_ptr[p], inc_ptr[p+1]),
                                         // in branch order; code = 2 l + end (0 from, 1 to)
  const int32_t *nbr_ptr, *nbr_bus, *nbr_grp;  // distinct neighbours ascending; nbr_grp[k]..[k+1] into grp_code
  const int32_t *grp_code;               // branches joining the bus to a neighbour, ascending: 2 l + end
  const int32_t *bus_nd, *bus_ndlt;      // distinct neighbours; those with a smaller index
  const int32_t *gen_bus, *gen_rank;     // rank = position among the generators of its bus
  const double *gen_c2, *gen_c1, *gen_c0, *gen_c2x2;
  const int32_t *arc_rank;               // position among the arcs of its bus
  const int32_t *jk8_off;                // offset of the K8 (and K9) J row of bus n inside a period block
  // M row offsets inside a period block
  const int32_t *mo_va, *mo_vm, *mo_pg0, *mo_pg1, *mo_qg, *mo_p, *mo_q;
  // loads [T][D]
  const double *pd, *qd;
  // Incidence slots: slot of branch l's from / to end in its bus's incident
  // list (branch order), [2][L]; per slot: neighbour position in the bus's
  // distinct-neighbour list (bits 0..27), group leader (bit 30: first branch to
  // that neighbour in branch order), neighbour index below the bus's (bit 29);
  // next slot of the same group or -1.
  const int32_t *br_slot, *slot_info, *slot_next;
  // Buses in the order the bus kernel processes them, and each bus's
  // incidence slots in ascending arc index (from ends, then to ends).
  const int32_t *bus_order, *arc_perm;
  // scratch: one record per incidence slot and period, [T][2L][kRec]:
  // (S_dd, S_vd, S_vv, S_vtvf, p_arc, q_arc) -- the branch element's local
  // values seen from that end plus the arc's flow variables; objective partials
  double *S;
  double *fpart;
  int32_t fpart_n;
  // Reactive ramp rows K11 (present iff qramp): row and J starts; the qg rows
  // of M at t >= 1 then use their own template (block size, row offsets).
  int32_t qramp;
  int64_t c_k11, j_k11, mb_qg1;
  const int32_t *mo_qg1;
  // The branch kernel's per-branch integers packed for 16-byte loads
  // (structure of quads, so a warp's load stays one contiguous run), [BRP_COUNT][L].
  const int4 *brp;
  // Owned periods [w0, w1) that the evaluation launches cover: [0, T) for a
  // model of its own; a period shard's local model has a halo period before
  // (w0 = 1) and / or after (w1 = T - 1) the periods it owns.
  int32_t w0, w1;
  // 1 if every branch is symmetric (br_sym all 1: no tap ratio or phase
  // shift asymmetry); the branch kernel then runs an instantiation without the
  // per-branch test
  int32_t all_sym;
  // [2][T][N]: w8 = D8 (m2gs vm) and w9 = D9 (p2bs vm) of every bus and
  // period, formed by k_bw before the branch kernel reads them at both ends
  // of each branch (SCHED_BUS_TERMS)
  double *bw;
};

// A period shard's handle evaluates only the periods it owns.
inline bool is_shard(const Dev &d) { return d.w0 != 0 || d.w1 != d.T; }

// Quads of brp: (f, t, slot of the from end, slot of the to end), (M row
// offsets of p_f, p_t, q_f, q_t inside a period block), (arc ranks of the from
// and to ends, generators at the from bus, generators at the to bus).
enum { BRP_ENDS, BRP_MROW, BRP_RANK, BRP_COUNT };

inline constexpr int kBlock = 256;
inline constexpr int kRec = 6;  // doubles per incidence record

// Optional per-kernel CUDA-event timing of the evaluation launches.
enum { KIND_BRANCH = 0, KIND_BUS = 1, KIND_GEN = 2, KIND_FSUM = 3, KIND_COUNT = 4 };
struct Prof {
  int cap = 0, next = 0;
  cudaEvent_t *ev = nullptr;  // [2 cap]
  int *kind = nullptr;        // [cap]
};

// A side stream and two events of a handle: the generator work of an
// evaluation runs on the side stream, forked from and joined back into the
// caller's stream, alongside the branch and bus work (it reads none of their
// outputs and writes disjoint ranges).
// Period chunks (chunk > 0): the branch kernel runs chunk by chunk on the
// caller's stream and the bus kernel of each chunk on a second stream `bus`,
// after an event recorded behind that chunk's branch launch, so that the bus
// work of chunk c overlaps the branch work of chunk c + 1 while the chunk's
// incidence records are still in L2.
constexpr int kMaxChunks = 64;
enum { SCHED_BUS_PRIORITY = MPOPF_SCHED_BUS_PRIORITY, SCHED_GEN_FIRST = MPOPF_SCHED_GEN_FIRST,
       SCHED_PDL = MPOPF_SCHED_PDL, SCHED_SPLIT_BUS = MPOPF_SCHED_SPLIT_BUS,
       SCHED_BUS_TERMS = MPOPF_SCHED_BUS_TERMS };
struct Fork {
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t bus = nullptr;          // bus kernels of a chunked evaluation
  cudaEvent_t ev_bus = nullptr;        // end of the bus stream's work
  cudaEvent_t ev_chunk[kMaxChunks] = {};
  int32_t chunk = 0;                   // periods per chunk; 0: one launch per kernel
  int32_t flags = 0;                   // SCHED_*: bus stream at the highest priority; generator work forked first
  cudaEvent_t gen_after = nullptr;     // the caller's event the generator work also waits for (or none)
  int32_t sms = 148;                   // SMs of the handle's device (launch shapes)
};

// The number of SMs of `device` (148 if the query fails), and the launch
// schedule (SCHED_* flags) a new handle starts with, from its branch launch's
// size on a device of `sms` SMs (mpopf_kernels.cu).
int32_t device_sms(int device);
int32_t default_schedule_flags(const Dev &d, int32_t sms);

// Kernel launchers (mpopf_kernels.cu).  With fork == nullptr every launch goes
// to s in order.
cudaError_t launch_eval(const Dev &d, unsigned outputs, const double *x, const double *lam, double sigma,
                        const double *sx, const double *dv, double dw, double *f, double *grad, double *c,
                        double *jv, double *hv, double *kv, cudaStream_t s, Prof *prof,
                        const Fork *fork = nullptr);
int eval_launch_count(const Dev &d, unsigned outputs, const Fork *fork = nullptr);
// Creates (or re-creates, for a new priority) the bus stream and the chunk
// events of a fork (mpopf_kernels.cu).
cudaError_t fork_bus_stream(Fork *fork, bool high_priority);
// Pattern expansion (mpopf_setup.cu).
cudaError_t launch_patterns(const Dev &d, int32_t *jrow, int32_t *jcol, int32_t *hrow, int32_t *hcol,
                            int64_t *krowptr, int32_t *kcol, double *xl, double *xu, double *gl, double *gu,
                            const double *vmin, const double *vmax, const double *pmin, const double *pmax,
                            const double *qmin, const double *qmax, const double *angmin, const double *angmax,
                            const double *ramp, const double *qramp, cudaStream_t s);

void set_error(const std::string &msg);

// Batched evaluation: many instances in one persistent launch.
struct BatchIO {
  const double *x, *lam, *sx, *dv;
  double *f, *grad, *c, *jv, *hv, *kv;
  double sigma, dw;
};
enum { ITEM_BRANCH = 0, ITEM_GEN = 1, ITEM_BUS = 2, ITEM_FSUM = 3 };
struct BatchItem {
  int32_t inst, kind, first, count;  // units [first, first + count) of that kind of that instance
  int32_t wait, signal;              // dependency counter waited on / incremented when done (-1: none)
};
// ctl layout: [0] next item of the (first) launch, [1] wait-limit flag,
// [2 + c] dependency counter c, [2 + n_counters] next item of the second
// launch of a two-launch schedule; need[c] = number of items that signal
// counter c.  phase: 0 one launch with every item, 1 / 2 the two launches.
cudaError_t batch_kernel_node(cudaKernelNodeParams *p, void **args, int32_t grid, int phase);
int batch_max_ctas_per_sm(int phase);
int batch_block_threads(int phase);  // CTA size of each launch form

}  // namespace mpopf

// The handle (opaque to callers).
namespace mpopf {
constexpr int kMaxBlocks = 128;
// CSC compression of J (0) or W (1), built on first request.
struct CscState {
  bool built;
  int64_t nnz;
  int64_t *colptr;  // [n + 1]
  int32_t *rowidx;  // [nnz]
  int32_t *src;     // COO entry of each sorted position
  int64_t *seg;     // [nnz + 1] run starts into src (W with duplicates); NULL: one entry per slot
};
}  // namespace mpopf

namespace mpopf {
struct KktSolver;
// Streams and events of the pipelined host-buffer sweep (created on first use).
constexpr int kHostWindows = 8;
struct HostPipe {
  cudaStream_t in, out;
  cudaEvent_t start, gen, ev_in[kHostWindows], ev_c[kHostWindows];
};
}  // namespace mpopf

struct mpopf_handle {
  mpopf::Dev d;
  mpopf_pattern pat;
  void *blocks[mpopf::kMaxBlocks];  // device allocations owned by the handle
  int nblocks;
  // staging for mpopf_sweep_host (allocated on first use)
  double *stage;
  size_t stage_bytes;
  mpopf::Prof prof;
  double *work;  // [m] row vector of the condensed right-hand side
  mpopf::CscState csc[2];
  mpopf::HostPipe *pipe;
  mpopf::KktSolver *solver;  // library factorisation of M (built on first use)
  mpopf::Fork fork;          // side stream of the evaluations (created at setup)
  int device;                // CUDA device current at setup (holds every allocation above)
  // incidence records and objective partials of mpopf_sweep_points (grown on use)
  double *pts;
  size_t pts_bytes;
};

namespace mpopf {
// Makes the handle's scratch of the many-point / many-vector calls at least
// `need` bytes (a device-wide synchronisation before a smaller one is
// replaced); MPOPF_OK or an error code with the message set for `who`
// (MPOPF_ERR_ARG when it would have to grow while `s` is being captured).
int grow_points_scratch(mpopf_handle *h, size_t need, const char *who, cudaStream_t s);
// Branch and bus work of periods [t0, t1) of a full sweep, and the generator
// work with the objective over the whole horizon; together, over a partition
// of the horizon, exactly the launches of a full sweep (mpopf_kernels.cu).
void launch_window(const Dev &d, int32_t t0, int32_t t1, const double *x, const double *lam, const double *sx,
                   const double *dv, double dw, double *grad, double *c, double *jv, double *hv, double *kv,
                   cudaStream_t s);
void launch_gen_obj(const Dev &d, const double *x, double sigma, const double *sx, const double *dv, double dw,
                    double *f, double *grad, double *c, double *jv, double *hv, double *kv, cudaStream_t s);
void hostpipe_destroy(mpopf_handle *h);
void kkt_solver_destroy(mpopf_handle *h);
}  // namespace mpopf
