"""Thin ctypes binding of ``libmpopf.so`` (declared in ``include/mpopf.h``).

Argument marshalling only: every step of the evaluation runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (float64, contiguous);
PyTorch supplies device memory and the current stream.  The library must be
built (``python -m paper_2405_14032_b300.build``); loading fails loudly
otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpopf.so")

OUT_OBJ, OUT_GRAD, OUT_CONS, OUT_JAC, OUT_HESS, OUT_KKT = 1, 2, 4, 8, 16, 32
OUT_ALL = 63
CSC_JAC, CSC_HESS = 0, 1

_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_U = ctypes.c_uint


class _Network(ctypes.Structure):
    _fields_ = [("n_bus", _I32), ("n_branch", _I32), ("n_gen", _I32), ("n_load", _I32), ("ref_bus", _I32)] + [
        (name, _P) for name in (
            "bus_gs", "bus_bs", "bus_vmin", "bus_vmax", "br_f", "br_t", "br_r", "br_x", "br_b", "br_tap",
            "br_shift", "br_smax", "br_angmin", "br_angmax", "gen_bus", "gen_c2", "gen_c1", "gen_c0",
            "gen_pmin", "gen_pmax", "gen_qmin", "gen_qmax", "gen_ramp", "load_bus", "gen_qramp")]


class _Csc(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("colptr", _P), ("rowidx", _P)]


class _Pattern(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz_jac", ctypes.c_int64),
                ("nnz_hess", ctypes.c_int64), ("nnz_kkt", ctypes.c_int64),
                ("n_bus", _I32), ("n_branch", _I32), ("n_gen", _I32), ("n_load", _I32), ("n_periods", _I32)] + [
        (name, _P) for name in ("jac_row", "jac_col", "hess_row", "hess_col", "kkt_rowptr", "kkt_col",
                                "xl", "xu", "gl", "gu")]


class _Range(ctypes.Structure):
    _fields_ = [("what", _I32), ("reserved", _I32), ("local", ctypes.c_int64), ("global_", ctypes.c_int64),
                ("count", ctypes.c_int64)]


SHARD_MAX_RANGES = 64
RANGE_X, RANGE_XALL, RANGE_ROWS, RANGE_JAC, RANGE_HESS, RANGE_KKT = 0, 1, 2, 3, 4, 5
RANGE_NAMES = {RANGE_X: "x", RANGE_XALL: "xall", RANGE_ROWS: "rows", RANGE_JAC: "jac", RANGE_HESS: "hess",
               RANGE_KKT: "kkt"}


class _ShardLayout(ctypes.Structure):
    _fields_ = [(k, _I32) for k in ("n_periods", "t0", "t1", "local_periods", "own0", "own1", "halo_len",
                                    "halo_blocks")] + \
               [(k, ctypes.c_int64) for k in ("n", "m", "nnz_jac", "nnz_hess", "nnz_kkt")] + \
               [(k, ctypes.c_int64 * 2) for k in ("x_recv", "x_send", "d_recv", "d_send")] + \
               [("n_ranges", _I32), ("reserved", _I32), ("ranges", _Range * SHARD_MAX_RANGES)]


class _BatchIO(ctypes.Structure):
    _fields_ = [("x", _P), ("lam", _P), ("sigma_x", _P), ("dvec", _P), ("sigma", _D), ("delta_w", _D),
                ("f", _P), ("grad", _P), ("c", _P), ("jv", _P), ("hv", _P), ("kv", _P)]


_lib = None


def _ensure_built():
    """Rebuild libmpopf.so when a source is newer than it (a stale library
    would not match the kernels' scratch layout).  Raises if the library is
    missing and cannot be built: there is no CPU fallback."""
    from . import build as _build
    srcs = _build.sources()
    if os.path.exists(LIB_PATH) and srcs and os.path.getmtime(LIB_PATH) >= max(
            os.path.getmtime(p) for p in srcs + [os.path.join(_build.ROOT, "include", "mpopf.h")]):
        return
    try:
        _build.build()
    except Exception as exc:  # nvcc missing or failing
        raise RuntimeError(f"libmpopf.so is missing or stale at {LIB_PATH} and could not be built ({exc}); "
                           "there is no CPU fallback") from exc


def lib():
    """Load libmpopf.so (rebuilt first if stale; raises if unavailable)."""
    global _lib
    if _lib is None:
        _ensure_built()
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "mpopf_setup": (ctypes.c_int, [ctypes.POINTER(_Network), _I32, _P, _P, ctypes.POINTER(_P),
                                           ctypes.POINTER(_Pattern)]),
            "mpopf_shard_plan": (ctypes.c_int, [ctypes.POINTER(_Network), _I32, _I32, _I32,
                                                ctypes.POINTER(_ShardLayout)]),
            "mpopf_shard_setup": (ctypes.c_int, [ctypes.POINTER(_Network), _I32, _I32, _I32, _P, _P,
                                                 ctypes.POINTER(_P), ctypes.POINTER(_Pattern)]),
            "mpopf_get_pattern": (ctypes.c_int, [_P, ctypes.POINTER(_Pattern)]),
            "mpopf_set_loads": (ctypes.c_int, [_P, _P, _P, _P]),
            "mpopf_eval": (ctypes.c_int, [_P, _U, _P, _P, _D, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P]),
            "mpopf_eval_obj": (ctypes.c_int, [_P, _P, _P, _P]),
            "mpopf_eval_grad": (ctypes.c_int, [_P, _P, _P, _P]),
            "mpopf_eval_cons": (ctypes.c_int, [_P, _P, _P, _P]),
            "mpopf_eval_jac": (ctypes.c_int, [_P, _P, _P, _P]),
            "mpopf_eval_hess": (ctypes.c_int, [_P, _P, _P, _D, _P, _P]),
            "mpopf_assemble_kkt": (ctypes.c_int, [_P, _P, _P, _D, _P, _P, _D, _P, _P]),
            "mpopf_sweep": (ctypes.c_int, [_P, _P, _P, _D, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P]),
            "mpopf_sweep_host": (ctypes.c_int, [_P, _P, _P, _D, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P]),
            "mpopf_sweep_points": (ctypes.c_int, [_P, _I32, _P, _P, _D, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P]),
            "mpopf_assemble_kkt_noalloc": (ctypes.c_int, [_P, _P, _P, _D, _P, _P, _D, _P, _P]),
            "mpopf_vjp": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
            "mpopf_jvp": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
            "mpopf_hvp": (ctypes.c_int, [_P, _P, _P, _D, _P, _P, _P]),
            "mpopf_kkt_factor": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64), _P]),
            "mpopf_kkt_solve": (ctypes.c_int, [_P, _P, _P, _P]),
            "mpopf_csc_pattern": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_Csc)]),
            "mpopf_coo_to_csc": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
            "mpopf_ipm_prepare": (ctypes.c_int, [_P] * 7 + [_D] * 3 + [_P] * 5),
            "mpopf_ipm_rhs": (ctypes.c_int, [_P] * 10 + [_D] + [_P, _P]),
            "mpopf_ipm_recover": (ctypes.c_int, [_P] * 13 + [_D] * 3 + [_P] * 7),
            "mpopf_vjp_jv": (ctypes.c_int, [_P] * 8),
            "mpopf_vjp_many": (ctypes.c_int, [_P, _I32] + [_P] * 7),
            "mpopf_jvp_many": (ctypes.c_int, [_P, _I32] + [_P] * 7),
            "mpopf_hvp_many": (ctypes.c_int, [_P, _I32, _P, _P, _D, _P, _P, _P, _P]),
            "mpopf_jvp_jv": (ctypes.c_int, [_P] * 8),
            "mpopf_batch_create": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_P)]),
            "mpopf_batch_set_io": (ctypes.c_int, [_P, _P, _P]),
            "mpopf_batch_sweep": (ctypes.c_int, [_P, _P]),
            "mpopf_batch_set_schedule": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32]),
            "mpopf_batch_get_schedule": (ctypes.c_int, [_P, _P, _P, _P]),
            "mpopf_batch_tune": (ctypes.c_int, [_P, _P, _I32, _P]),
            "mpopf_batch_status": (ctypes.c_int, [_P]),
            "mpopf_batch_test_stall": (ctypes.c_int, [_P, _I32]),
            "mpopf_batch_destroy": (None, [_P]),
            "mpopf_launch_count": (ctypes.c_int, [_P, _U]),
            "mpopf_set_sweep_schedule": (ctypes.c_int, [_P, _I32, _I32]),
            "mpopf_get_sweep_schedule": (ctypes.c_int, [_P, _P, _P]),
            "mpopf_set_gen_dependency": (ctypes.c_int, [_P, _P]),
            "mpopf_fp64_issue_rate": (ctypes.c_int, [_I32, _P, _P]),
            "mpopf_profile_start": (ctypes.c_int, [_P, _I32]),
            "mpopf_profile_stop": (ctypes.c_int, [_P, _P, _P]),
            "mpopf_destroy": (None, [_P]),
            "mpopf_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names the header declares (for the load/export check)."""
    return ["mpopf_setup", "mpopf_shard_plan", "mpopf_shard_setup", "mpopf_get_pattern", "mpopf_set_loads", "mpopf_eval", "mpopf_eval_obj",
            "mpopf_eval_grad", "mpopf_eval_cons", "mpopf_eval_jac", "mpopf_eval_hess", "mpopf_assemble_kkt",
            "mpopf_sweep", "mpopf_sweep_host", "mpopf_sweep_points", "mpopf_assemble_kkt_noalloc", "mpopf_vjp", "mpopf_jvp", "mpopf_hvp",
            "mpopf_vjp_jv", "mpopf_jvp_jv", "mpopf_vjp_many", "mpopf_jvp_many", "mpopf_hvp_many", "mpopf_kkt_factor", "mpopf_kkt_solve", "mpopf_csc_pattern",
            "mpopf_coo_to_csc", "mpopf_ipm_prepare", "mpopf_ipm_rhs", "mpopf_ipm_recover", "mpopf_batch_create",
            "mpopf_batch_set_io", "mpopf_batch_sweep", "mpopf_batch_set_schedule", "mpopf_batch_get_schedule",
            "mpopf_batch_tune", "mpopf_batch_status", "mpopf_batch_test_stall", "mpopf_batch_destroy",
            "mpopf_launch_count", "mpopf_set_sweep_schedule", "mpopf_get_sweep_schedule", "mpopf_set_gen_dependency",
            "mpopf_fp64_issue_rate", "mpopf_profile_start", "mpopf_profile_stop", "mpopf_destroy", "mpopf_last_error"]


class MpopfError(RuntimeError):
    pass


def fp64_issue_rate(iters=4096, stream=None):
    """(FP64 thread-instructions per second, seconds) of the library's DFMA-chain
    probe on the current device (mpopf_fp64_issue_rate; synchronous)."""
    rate = np.zeros(1)
    secs = np.zeros(1)
    _check(lib().mpopf_fp64_issue_rate(int(iters), rate.ctypes.data, secs.ctypes.data), "mpopf_fp64_issue_rate")
    return float(rate[0]), float(secs[0])


def _check(rc, what):
    if rc != 0:
        raise MpopfError(f"{what} failed ({rc}): {lib().mpopf_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


class _DeviceArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _network_struct(net, keep):
    """The C network descriptor of a synth.Network; `keep` holds the arrays
    it points to."""

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data if a.size else None

    f64, i32 = np.float64, np.int32
    return _Network(
        n_bus=net.n_bus, n_branch=net.n_branch, n_gen=net.n_gen, n_load=net.n_load, ref_bus=net.ref_bus,
        bus_gs=arr(net.bus_gs, f64), bus_bs=arr(net.bus_bs, f64), bus_vmin=arr(net.bus_vmin, f64),
        bus_vmax=arr(net.bus_vmax, f64), br_f=arr(net.br_f, i32), br_t=arr(net.br_t, i32),
        br_r=arr(net.br_r, f64), br_x=arr(net.br_x, f64), br_b=arr(net.br_b, f64), br_tap=arr(net.br_tap, f64),
        br_shift=arr(net.br_shift, f64), br_smax=arr(net.br_smax, f64), br_angmin=arr(net.br_angmin, f64),
        br_angmax=arr(net.br_angmax, f64), gen_bus=arr(net.gen_bus, i32), gen_c2=arr(net.gen_c2, f64),
        gen_c1=arr(net.gen_c1, f64), gen_c0=arr(net.gen_c0, f64), gen_pmin=arr(net.gen_pmin, f64),
        gen_pmax=arr(net.gen_pmax, f64), gen_qmin=arr(net.gen_qmin, f64), gen_qmax=arr(net.gen_qmax, f64),
        gen_ramp=arr(net.gen_ramp, f64), load_bus=arr(net.load_bus, i32),
        gen_qramp=None if net.gen_qramp is None else arr(net.gen_qramp, f64))


def shard_plan(net, T, t0, t1):
    """Layout of the period shard [t0, t1) of a T-period model (host only, no
    device): dict with the local sizes, the halo offsets (x_recv, x_send,
    d_recv, d_send: lists per block, -1 where there is no neighbour) and the
    local <-> global ranges {name: [(local, global, count), ...]}."""
    keep = []
    c = _network_struct(net, keep)
    lay = _ShardLayout()
    _check(lib().mpopf_shard_plan(ctypes.byref(c), int(T), int(t0), int(t1), ctypes.byref(lay)), "mpopf_shard_plan")
    out = {k: int(getattr(lay, k)) for k in ("n_periods", "t0", "t1", "local_periods", "own0", "own1", "halo_len",
                                             "halo_blocks", "n", "m", "nnz_jac", "nnz_hess", "nnz_kkt")}
    for k in ("x_recv", "x_send", "d_recv", "d_send"):
        out[k] = [int(v) for v in getattr(lay, k)][:out["halo_blocks"]]
    ranges = {name: [] for name in RANGE_NAMES.values()}
    for i in range(lay.n_ranges):
        r = lay.ranges[i]
        ranges[RANGE_NAMES[r.what]].append((int(r.local), int(r.global_), int(r.count)))
    out["ranges"] = ranges
    return out


class Handle:
    """A multi-period AC OPF model on the GPU (``mpopf_setup`` once); with
    shard=(t0, t1) the period shard [t0, t1) of it (``mpopf_shard_setup``)."""

    def __init__(self, inst, shard=None):
        net = inst.net
        self._keep = []
        c = _network_struct(net, self._keep)
        pd = np.ascontiguousarray(inst.pd, dtype=np.float64)
        qd = np.ascontiguousarray(inst.qd, dtype=np.float64)
        pdp = pd.ctypes.data if pd.size else None
        qdp = qd.ctypes.data if qd.size else None
        h = ctypes.c_void_p()
        pat = _Pattern()
        if shard is None:
            _check(lib().mpopf_setup(ctypes.byref(c), int(inst.T), pdp, qdp, ctypes.byref(h), ctypes.byref(pat)),
                   "mpopf_setup")
        else:
            t0, t1 = (int(v) for v in shard)
            _check(lib().mpopf_shard_setup(ctypes.byref(c), int(inst.T), t0, t1, pdp, qdp, ctypes.byref(h),
                                           ctypes.byref(pat)), "mpopf_shard_setup")
        self._keep = []
        self.h = h
        self.pat = pat
        self.shard = None if shard is None else (t0, t1)
        self.T = int(pat.n_periods)
        self.n_load = int(inst.net.n_load)
        self.n, self.m = int(pat.n), int(pat.m)
        self.nnz_jac, self.nnz_hess, self.nnz_kkt = int(pat.nnz_jac), int(pat.nnz_hess), int(pat.nnz_kkt)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().mpopf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- patterns (zero-copy torch views of handle-owned device memory) ------
    def pattern(self):
        import torch
        p = self.pat
        t = lambda ptr, k, ty: torch.as_tensor(_DeviceArray(ptr, k, ty), device="cuda")
        return dict(
            jac_row=t(p.jac_row, self.nnz_jac, "<i4"), jac_col=t(p.jac_col, self.nnz_jac, "<i4"),
            hess_row=t(p.hess_row, self.nnz_hess, "<i4"), hess_col=t(p.hess_col, self.nnz_hess, "<i4"),
            kkt_rowptr=t(p.kkt_rowptr, self.n + 1, "<i8"), kkt_col=t(p.kkt_col, self.nnz_kkt, "<i4"),
            xl=t(p.xl, self.n, "<f8"), xu=t(p.xu, self.n, "<f8"), gl=t(p.gl, self.m, "<f8"),
            gu=t(p.gu, self.m, "<f8"))

    def launch_count(self, outputs=OUT_ALL):
        return int(lib().mpopf_launch_count(self.h, outputs))

    SCHED_BUS_PRIORITY, SCHED_GEN_FIRST, SCHED_PDL, SCHED_SPLIT_BUS = 1, 2, 4, 8
    SCHED_BUS_TERMS = 16

    def set_sweep_schedule(self, chunk_periods, flags=0):
        """Period chunks of the evaluation launches (0: one launch per kernel);
        flags SCHED_BUS_PRIORITY, SCHED_GEN_FIRST, SCHED_PDL, SCHED_SPLIT_BUS,
        SCHED_BUS_TERMS (see mpopf_set_sweep_schedule)."""
        _check(lib().mpopf_set_sweep_schedule(self.h, int(chunk_periods), int(flags)), "mpopf_set_sweep_schedule")

    def set_gen_dependency(self, event):
        """Later evaluations' generator work also waits for `event` (a
        torch.cuda.Event recorded by the caller before each evaluation, e.g.
        after a shard's halo exchange on another stream); None removes it."""
        self._gen_event = event  # kept alive while the handle may use it
        _check(lib().mpopf_set_gen_dependency(self.h, None if event is None else ctypes.c_void_p(event.cuda_event)),
               "mpopf_set_gen_dependency")

    def sweep_schedule(self):
        p = np.zeros(1, np.int32)
        f = np.zeros(1, np.int32)
        _check(lib().mpopf_get_sweep_schedule(self.h, p.ctypes.data, f.ctypes.data), "mpopf_get_sweep_schedule")
        return int(p[0]), int(f[0])

    KERNEL_KINDS = ("branch", "bus", "gen", "fsum")

    def profile_start(self, max_launches):
        _check(lib().mpopf_profile_start(self.h, int(max_launches)), "mpopf_profile_start")

    def profile_stop(self):
        """{kind: (summed ms, launches)} of the launches since profile_start."""
        ms = np.zeros(4)
        cnt = np.zeros(4, np.int32)
        _check(lib().mpopf_profile_stop(self.h, ms.ctypes.data, cnt.ctypes.data), "mpopf_profile_stop")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KERNEL_KINDS)}

    # -- evaluation -----------------------------------------------------------
    def new_outputs(self, outputs=OUT_ALL):
        import torch
        kw = dict(dtype=torch.float64, device="cuda")
        e = lambda k: torch.empty(k, **kw)
        return dict(f=e(1) if outputs & OUT_OBJ else None, grad=e(self.n) if outputs & OUT_GRAD else None,
                    c=e(self.m) if outputs & OUT_CONS else None, jv=e(self.nnz_jac) if outputs & OUT_JAC else None,
                    hv=e(self.nnz_hess) if outputs & OUT_HESS else None,
                    kv=e(self.nnz_kkt) if outputs & OUT_KKT else None)

    def eval(self, outputs, x, lam=None, sigma=1.0, sigma_x=None, dvec=None, delta_w=0.0, out=None, stream=None):
        out = self.new_outputs(outputs) if out is None else out
        _check(lib().mpopf_eval(self.h, outputs, _ptr(x), _ptr(lam), float(sigma), _ptr(sigma_x), _ptr(dvec),
                                float(delta_w), _ptr(out.get("f")), _ptr(out.get("grad")), _ptr(out.get("c")),
                                _ptr(out.get("jv")), _ptr(out.get("hv")), _ptr(out.get("kv")),
                                _stream_ptr(stream)), "mpopf_eval")
        return out

    def sweep(self, x, lam, sigma, sigma_x, dvec, delta_w, out=None, stream=None):
        out = self.new_outputs(OUT_ALL) if out is None else out
        _check(lib().mpopf_sweep(self.h, _ptr(x), _ptr(lam), float(sigma), _ptr(sigma_x), _ptr(dvec),
                                 float(delta_w), _ptr(out["f"]), _ptr(out["grad"]), _ptr(out["c"]), _ptr(out["jv"]),
                                 _ptr(out["hv"]), _ptr(out["kv"]), _stream_ptr(stream)), "mpopf_sweep")
        return out

    def new_point_outputs(self, k):
        """Outputs of mpopf_sweep_points at k points: [k, size] tensors."""
        import torch
        kw = dict(dtype=torch.float64, device="cuda")
        return dict(f=torch.empty(k, **kw), grad=torch.empty(k, self.n, **kw), c=torch.empty(k, self.m, **kw),
                    jv=torch.empty(k, self.nnz_jac, **kw), hv=torch.empty(k, self.nnz_hess, **kw),
                    kv=torch.empty(k, self.nnz_kkt, **kw))

    def sweep_points(self, x, lam, sigma, sigma_x, dvec, delta_w, out=None, stream=None):
        """Full sweeps at k points in one launch per kernel (mpopf_sweep_points):
        x, sigma_x [k, n] and lam, dvec [k, m] contiguous device tensors;
        sigma and delta_w shared.  Returns [k, size] outputs (f [k])."""
        k = int(x.shape[0])
        for name, a, w in (("x", x, self.n), ("lam", lam, self.m), ("sigma_x", sigma_x, self.n),
                           ("dvec", dvec, self.m)):
            if tuple(a.shape) != (k, w) or not a.is_contiguous():
                raise ValueError(f"sweep_points: {name} must be a contiguous [{k}, {w}] tensor")
        out = self.new_point_outputs(k) if out is None else out
        _check(lib().mpopf_sweep_points(self.h, k, _ptr(x), _ptr(lam), float(sigma), _ptr(sigma_x), _ptr(dvec),
                                        float(delta_w), _ptr(out["f"]), _ptr(out["grad"]), _ptr(out["c"]),
                                        _ptr(out["jv"]), _ptr(out["hv"]), _ptr(out["kv"]), _stream_ptr(stream)),
               "mpopf_sweep_points")
        return out

    def sweep_host(self, x, lam, sigma, sigma_x, dvec, delta_w, out, stream=None):
        """All inputs and outputs are host arrays (numpy or pinned torch CPU tensors)."""
        _check(lib().mpopf_sweep_host(self.h, _ptr(x), _ptr(lam), float(sigma), _ptr(sigma_x), _ptr(dvec),
                                      float(delta_w), _ptr(out["f"]), _ptr(out["grad"]), _ptr(out["c"]),
                                      _ptr(out["jv"]), _ptr(out["hv"]), _ptr(out["kv"]), _stream_ptr(stream)),
               "mpopf_sweep_host")
        return out

    def assemble_kkt_noalloc(self, x, lam, sigma, sigma_x, dvec, delta_w, kv, stream=None):
        """M values into the caller's `kv` with no device allocation by the
        call: the scratch is a fixed array inside the library (for callers
        that cannot allocate once they are running, e.g. processes that
        reserve all device memory up front).  Raises MpopfError (code -2)
        when 12 T L exceeds that array."""
        _check(lib().mpopf_assemble_kkt_noalloc(self.h, _ptr(x), _ptr(lam), float(sigma), _ptr(sigma_x),
                                                _ptr(dvec), float(delta_w), _ptr(kv), _stream_ptr(stream)),
               "mpopf_assemble_kkt_noalloc")
        return kv

    # -- matrix-free derivative products -------------------------------------
    def vjp(self, x, y, gx=None, loads=True, jv=None, stream=None):
        """(J^T y, (dc/dPd)^T y, (dc/dQd)^T y); the load parts are None when
        loads is False; jv: J values at x (optional: read instead of recomputed)."""
        import torch
        gx = torch.empty(self.n, dtype=torch.float64, device="cuda") if gx is None else gx
        gpd = gqd = None
        if loads:
            gpd = torch.empty(self.T * self.n_load, dtype=torch.float64, device="cuda")
            gqd = torch.empty_like(gpd)
        _check(lib().mpopf_vjp_jv(self.h, _ptr(x), _ptr(jv), _ptr(y), _ptr(gx), _ptr(gpd), _ptr(gqd),
                                  _stream_ptr(stream)), "mpopf_vjp")
        return gx, gpd, gqd

    def jvp(self, x, v, dpd=None, dqd=None, out=None, jv=None, stream=None):
        """J v [m]; jv: J values at x (optional: read instead of recomputed)."""
        import torch
        out = torch.empty(self.m, dtype=torch.float64, device="cuda") if out is None else out
        _check(lib().mpopf_jvp_jv(self.h, _ptr(x), _ptr(jv), _ptr(v), _ptr(dpd), _ptr(dqd), _ptr(out),
                                  _stream_ptr(stream)), "mpopf_jvp")
        return out

    def hvp(self, x, lam, sigma, v, out=None, stream=None):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device="cuda") if out is None else out
        _check(lib().mpopf_hvp(self.h, _ptr(x), _ptr(lam), float(sigma), _ptr(v), _ptr(out), _stream_ptr(stream)),
               "mpopf_hvp")
        return out

    def _many(self, name, a, width):
        if a.dim() != 2 or a.shape[1] != width or not a.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous [k, {width}] tensor")
        return int(a.shape[0])

    def vjp_many(self, x, Y, loads=True, jv=None, stream=None):
        """J^T y for the k rows of Y [k, m] at one point: (GX [k, n], GPD, GQD
        [k, T D] or None); jv: J values at x (optional)."""
        import torch
        k = self._many("vjp_many", Y, self.m)
        gx = torch.empty(k, self.n, dtype=torch.float64, device="cuda")
        gpd = gqd = None
        if loads:
            gpd = torch.empty(k, self.T * self.n_load, dtype=torch.float64, device="cuda")
            gqd = torch.empty_like(gpd)
        _check(lib().mpopf_vjp_many(self.h, k, _ptr(x), _ptr(jv), _ptr(Y), _ptr(gx), _ptr(gpd), _ptr(gqd),
                                    _stream_ptr(stream)), "mpopf_vjp_many")
        return gx, gpd, gqd

    def jvp_many(self, x, V, dpd=None, dqd=None, jv=None, stream=None):
        """J v for the k rows of V [k, n] (load tangents dpd, dqd [k, T D]) -> [k, m]."""
        import torch
        k = self._many("jvp_many", V, self.n)
        out = torch.empty(k, self.m, dtype=torch.float64, device="cuda")
        _check(lib().mpopf_jvp_many(self.h, k, _ptr(x), _ptr(jv), _ptr(V), _ptr(dpd), _ptr(dqd), _ptr(out),
                                    _stream_ptr(stream)), "mpopf_jvp_many")
        return out

    def hvp_many(self, x, lam, sigma, V, hw=None, stream=None):
        """W v for the k rows of V [k, n] -> [k, n]; hw: W values at (x, lam,
        sigma) (optional)."""
        import torch
        k = self._many("hvp_many", V, self.n)
        out = torch.empty(k, self.n, dtype=torch.float64, device="cuda")
        _check(lib().mpopf_hvp_many(self.h, k, _ptr(x), _ptr(lam), float(sigma), _ptr(hw), _ptr(V), _ptr(out),
                                    _stream_ptr(stream)), "mpopf_hvp_many")
        return out

    # -- library factorisation of M ---------------------------------------------
    def kkt_factor(self, kv, stream=None):
        """Cholesky factorisation of M from its lower CSR values; returns -1, or
        the row of a zero / negative pivot when M is not positive definite."""
        zp = ctypes.c_int64(-1)
        rc = lib().mpopf_kkt_factor(self.h, _ptr(kv), ctypes.byref(zp), _stream_ptr(stream))
        if rc == -5:
            return int(zp.value)
        _check(rc, "mpopf_kkt_factor")
        return -1

    def kkt_solve(self, rhs, out=None, stream=None):
        """M^{-1} rhs with the last factorisation."""
        out = self._dvec(self.n) if out is None else out
        _check(lib().mpopf_kkt_solve(self.h, _ptr(rhs), _ptr(out), _stream_ptr(stream)), "mpopf_kkt_solve")
        return out

    # -- COO -> CSC compression -------------------------------------------------
    def csc_pattern(self, which):
        """dict(colptr [n + 1] int64, rowidx [nnz] int32) of J (CSC_JAC) or the
        lower W (CSC_HESS), zero-copy views of handle-owned device memory
        (built on the first call)."""
        import torch
        c = _Csc()
        _check(lib().mpopf_csc_pattern(self.h, int(which), ctypes.byref(c)), "mpopf_csc_pattern")
        self._csc_nnz = getattr(self, "_csc_nnz", {})
        self._csc_nnz[int(which)] = int(c.nnz)
        return dict(colptr=torch.as_tensor(_DeviceArray(c.colptr, self.n + 1, "<i8"), device="cuda"),
                    rowidx=torch.as_tensor(_DeviceArray(c.rowidx, c.nnz, "<i4"), device="cuda"), nnz=int(c.nnz))

    def coo_to_csc(self, which, coo_vals, out=None, stream=None):
        """CSC values of J or W from their COO values (csc_pattern first)."""
        nnz = getattr(self, "_csc_nnz", {}).get(int(which))
        if nnz is None:
            nnz = self.csc_pattern(which)["nnz"]
        out = self._dvec(nnz) if out is None else out
        _check(lib().mpopf_coo_to_csc(self.h, int(which), _ptr(coo_vals), _ptr(out), _stream_ptr(stream)),
               "mpopf_coo_to_csc")
        return out

    # -- interior-point algebra around the condensed matrix -------------------
    def _dvec(self, k):
        import torch
        return torch.empty(k, dtype=torch.float64, device="cuda")

    def ipm_prepare(self, x, s, zl_x, zu_x, zl_s, zu_s, delta_w, delta_c, eps_tol, recip=None, stream=None):
        """(Sigma_x [n], D [m], C [m], recip [2n + 2m]) from the bounds and bound
        duals; recip (the reciprocals 1/(v - lo), 1/(hi - v)) feeds ipm_rhs and
        ipm_recover at the same point."""
        sigx, dvec, cvec = self._dvec(self.n), self._dvec(self.m), self._dvec(self.m)
        recip = self._dvec(2 * (self.n + self.m)) if recip is None else recip
        _check(lib().mpopf_ipm_prepare(self.h, _ptr(x), _ptr(s), _ptr(zl_x), _ptr(zu_x), _ptr(zl_s), _ptr(zu_s),
                                       float(delta_w), float(delta_c), float(eps_tol), _ptr(sigx), _ptr(dvec),
                                       _ptr(cvec), _ptr(recip), _stream_ptr(stream)), "mpopf_ipm_prepare")
        return sigx, dvec, cvec, recip

    def ipm_rhs(self, x, s, y, grad, c, recip, dvec, cvec, mu, out=None, jv=None, stream=None):
        """Condensed right-hand side q_x + J^T (C q_s + D q_y) [n]; jv: J values
        at x from the sweep (optional: read instead of recomputed)."""
        out = self._dvec(self.n) if out is None else out
        _check(lib().mpopf_ipm_rhs(self.h, _ptr(x), _ptr(jv), _ptr(s), _ptr(y), _ptr(grad), _ptr(c),
                                   _ptr(recip), _ptr(dvec), _ptr(cvec), float(mu), _ptr(out), _stream_ptr(stream)),
               "mpopf_ipm_rhs")
        return out

    def ipm_recover(self, x, s, y, zl_x, zu_x, zl_s, zu_s, c, recip, cvec, dx, mu, delta_w, delta_c, out=None,
                    jv=None, stream=None):
        """dict ds, dy, dzl_s, dzu_s [m] and dzl_x, dzu_x [n] from dx; jv as in
        ipm_rhs."""
        r = out if out is not None else dict(
            ds=self._dvec(self.m), dy=self._dvec(self.m), dzl_x=self._dvec(self.n), dzu_x=self._dvec(self.n),
            dzl_s=self._dvec(self.m), dzu_s=self._dvec(self.m))
        _check(lib().mpopf_ipm_recover(self.h, _ptr(x), _ptr(jv), _ptr(s), _ptr(y), _ptr(zl_x), _ptr(zu_x),
                                       _ptr(zl_s), _ptr(zu_s), _ptr(c), _ptr(recip), _ptr(cvec), _ptr(dx), float(mu),
                                       float(delta_w), float(delta_c), _ptr(r["ds"]), _ptr(r["dy"]),
                                       _ptr(r["dzl_x"]), _ptr(r["dzu_x"]), _ptr(r["dzl_s"]), _ptr(r["dzu_s"]),
                                       _stream_ptr(stream)), "mpopf_ipm_recover")
        return r

    def set_loads(self, pd, qd, stream=None):
        _check(lib().mpopf_set_loads(self.h, _ptr(pd), _ptr(qd), _stream_ptr(stream)), "mpopf_set_loads")


class Batch:
    """Many handles swept together by one persistent launch (CUDA graph)."""

    def __init__(self, handles):
        self.handles = list(handles)
        arr = (_P * len(self.handles))(*[h.h.value for h in self.handles])
        b = ctypes.c_void_p()
        _check(lib().mpopf_batch_create(arr, len(self.handles), ctypes.byref(b)), "mpopf_batch_create")
        self.b = b
        self._io = None

    def set_io(self, ios, stream=None):
        """ios: per instance a dict with x, lam, sigma, sigma_x, dvec, delta_w and
        output tensors f, grad, c, jv, hv, kv (all CUDA float64)."""
        arr = (_BatchIO * len(ios))()
        for i, io in enumerate(ios):
            arr[i] = _BatchIO(_ptr(io["x"]), _ptr(io["lam"]), _ptr(io["sigma_x"]), _ptr(io["dvec"]),
                              float(io["sigma"]), float(io["delta_w"]), _ptr(io["f"]), _ptr(io["grad"]),
                              _ptr(io["c"]), _ptr(io["jv"]), _ptr(io["hv"]), _ptr(io["kv"]))
        self._io = ios  # keep the tensors alive
        _check(lib().mpopf_batch_set_io(self.b, arr, _stream_ptr(stream)), "mpopf_batch_set_io")

    def sweep(self, stream=None):
        _check(lib().mpopf_batch_sweep(self.b, _stream_ptr(stream)), "mpopf_batch_sweep")

    def set_schedule(self, order, tile_chunks, ctas_per_sm, chunk_periods=0, launches=1):
        _check(lib().mpopf_batch_set_schedule(self.b, order, tile_chunks, ctas_per_sm, chunk_periods, launches),
               "mpopf_batch_set_schedule")

    def schedule(self):
        s = np.zeros(5, np.int32)
        g = np.zeros(1, np.int32)
        k = np.zeros(1, np.int32)
        _check(lib().mpopf_batch_get_schedule(self.b, s.ctypes.data, g.ctypes.data, k.ctypes.data),
               "mpopf_batch_get_schedule")
        return dict(order=int(s[0]), tile_chunks=int(s[1]), ctas_per_sm=int(s[2]), chunk_periods=int(s[3]),
                    launches=int(s[4]), grid=int(g[0]), items=int(k[0]))

    def tune(self, reps=5, stream=None):
        best = np.zeros(1)
        _check(lib().mpopf_batch_tune(self.b, _stream_ptr(stream), int(reps), best.ctypes.data), "mpopf_batch_tune")
        return float(best[0])

    def test_stall(self, on):
        """Failure-path test hook (see mpopf_batch_test_stall)."""
        _check(lib().mpopf_batch_test_stall(self.b, int(bool(on))), "mpopf_batch_test_stall")

    def status(self):
        _check(lib().mpopf_batch_status(self.b), "mpopf_batch_status")

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            lib().mpopf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
