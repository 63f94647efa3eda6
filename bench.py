#!/usr/bin/env python
"""Benchmark of the per-iteration hot path of the multi-period AC OPF method
(arXiv 2405.14032): one full derivative sweep = f, grad f, c, J (COO), W (lower
COO) and the condensed KKT matrix M = W + diag(Sigma_x + delta_w) + J^T D J
(lower CSR), all FP64, on the 10,000-bus / 16,000-branch / 2,000-generator /
6,000-load network with T = 168 hourly periods (seeded synthetic data).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  Under torchrun (N > 1) the horizon is split into N
contiguous blocks of periods, one per GPU (strong scaling): before each sweep
every rank exchanges two G-vectors with its neighbours (pg of the period
before its block, D of the ramp rows after it; NCCL point-to-point) and after
it the partial objectives are summed (all-reduce); --mode replicas instead
evaluates one independent copy per rank (weak scaling).  The timing is the max
over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "full derivative sweeps/s + HBM GB/s (10k-bus T=168); batched & adjoint vs plain"
UNIT = "sweeps/s"
WORKLOAD = dict(n_bus=10000, n_branch=16000, n_gen=2000, n_load=6000, seed=3)
# FP64 operations of one branch x period instance of the full sweep (k_branch,
# ALL outputs): angle difference 1, sin/cos 15, flow terms 14, constraint values
# 14, Jacobian 8, W block 16, condensed-matrix contributions 75.  (Exact
# doublings and sign flips are integer operations and are not counted.)
FP64_OPS_PER_BRANCH_PERIOD = 143
# The FP64 pipe issues 2 thread-instructions (fma, add or mul) per cycle per SM
# (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 296
# for 148 SMs); with the maximum SM clock that is the ALU roofline of the path.
FP64_PER_CYCLE_PER_SM = 2
SM_MAX_MHZ = 2032.0


def fp64_issue_peak(sms, sm_max_mhz):
    """FP64 operations per second (in G) the GPU's FP64 pipes can issue."""
    return FP64_PER_CYCLE_PER_SM * sms * sm_max_mhz * 1e6 / 1e9


FP64_OPS_PER_BUS_PERIOD = 33   # hand counts of the bus and generator kernels (their
FP64_OPS_PER_GEN_PERIOD = 17   # loops vary with the degree; these are averages)
# With the bus-term launch in the schedule (MPOPF_SCHED_BUS_TERMS), the branch
# kernel reads the products D8 (m2gs vm) and D9 (p2bs vm) at both ends of its
# branch (8 operations fewer per element) and k_bw forms them once per bus and
# period (4 operations).
FP64_OPS_BUS_TERMS_PER_BRANCH_PERIOD = 8
FP64_OPS_BUS_TERMS_PER_BUS_PERIOD = 4
SCHED_BUS_TERMS = 16


def branch_ops_per_element(bus_terms):
    return FP64_OPS_PER_BRANCH_PERIOD - (FP64_OPS_BUS_TERMS_PER_BRANCH_PERIOD if bus_terms else 0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--periods", type=int, default=168, help="horizon T (168 is the benchmark workload)")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--dist-backend", choices=["nccl", "gloo"], default="nccl",
                    help="process-group backend for N > 1 (gloo stages the halo through host memory)")
    ap.add_argument("--mode", choices=["single", "replicas", "shards"], default=None,
                    help="N > 1: 'shards' (default; the horizon split into contiguous period blocks, one per "
                         "GPU, halo exchange and f all-reduce; strong scaling) or 'replicas' (one independent "
                         "copy of the instance per GPU; weak scaling)")
    return ap.parse_args()


def algorithmic_bytes(n, m, nnz_jac, nnz_hess, nnz_kkt, D, T):
    """Each array touched once: reads x, Sigma_x (n), lambda, D (m), loads
    (2 D T); writes grad (n), c (m), J, W, M values."""
    return 8 * (2 * n + 2 * m + 2 * D * T) + 8 * (n + m + nnz_jac + nnz_hess + nnz_kkt)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


BRANCH_KERNEL_END = "// The branch kernel over elements [first, end) on stream s"
DESCRIPTOR_END = "// Optional per-kernel CUDA-event timing of the evaluation launches."


def kernel_source_hash():
    """Hash of the code the branch kernel is compiled from: the device
    descriptor and constants of the internal header (up to the launch-side
    declarations that follow them), the device helpers, and the kernels file
    up to the end of k_branch (its helpers, branch_body and the kernel itself;
    the launchers and the other kernels follow), comments and whitespace
    removed, so that a comment edit or a change elsewhere keeps the counters
    valid."""
    h = hashlib.sha256()
    for name in ("mpopf_internal.cuh", "mpopf_device.cuh", "mpopf_kernels.cu"):
        with open(os.path.join(ROOT, "paper_2405_14032_b300", "csrc", name)) as fh:
            text = fh.read()
        if name == "mpopf_kernels.cu":
            text = text[:text.index(BRANCH_KERNEL_END)]
        if name == "mpopf_internal.cuh":
            text = text[:text.index(DESCRIPTOR_END)]
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def link_rates(torch, nbytes=1 << 30):
    """The host link's rates for plain pinned copies of 1 GB (one direction at a
    time, CUDA events on the current stream): the bound of the host-buffer
    sweep, whose traffic is mostly device-to-host."""
    k = nbytes // 8
    d = torch.ones(k, dtype=torch.float64, device="cuda")
    hbuf = torch.empty(k, dtype=torch.float64, pin_memory=True)
    rates = {}
    for name, fn in (("link_d2h_gbs", lambda: hbuf.copy_(d, non_blocking=True)),
                     ("link_h2d_gbs", lambda: d.copy_(hbuf, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fn()
        e1.record()
        torch.cuda.synchronize()
        rates[name] = 3 * nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del d, hbuf
    return rates


def ncu_traffic(periods):
    """DRAM bytes of one launch of the dominant kernel over `periods` periods,
    scaled from the committed ncu capture of a shorter horizon (the kernel's
    traffic is proportional to the branch x period elements it processes), or
    None when the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "k_branch_traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)
    except OSError:
        return None
    if rec.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    per = rec.get("dram_bytes_per_launch")
    if per is None or not rec.get("captured_periods"):
        return None
    return per * periods / rec["captured_periods"]


# ---------------------------------------------------------------------------
# Clocks (NVML, read-only) sampled during the timed region.
# ---------------------------------------------------------------------------
class NvmlLite:
    """The few read-only NVML queries the clock sampler makes, through ctypes
    on the driver's libnvidia-ml.so.1 (for hosts without the pynvml module).
    Same names as pynvml's."""
    NVML_CLOCK_SM = 1

    def __init__(self):
        import ctypes
        self._c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"NVML {what}: error {rc}")

    def nvmlInit(self):
        self._check(self.lib.nvmlInit_v2(), "init")

    def nvmlDeviceGetHandleByUUID(self, uuid):
        h = self._c.c_void_p()
        uuid = uuid if isinstance(uuid, bytes) else uuid.encode()
        self._check(self.lib.nvmlDeviceGetHandleByUUID(self._c.c_char_p(uuid), self._c.byref(h)), "handle by UUID")
        return h

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self._c.c_void_p()
        self._check(self.lib.nvmlDeviceGetHandleByIndex_v2(self._c.c_uint(i), self._c.byref(h)), "handle by index")
        return h

    def _uint(self, fn, h, *args):
        v = self._c.c_uint()
        self._check(fn(h, *args, self._c.byref(v)), fn.__name__)
        return v.value

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._uint(self.lib.nvmlDeviceGetMaxClockInfo, h, self._c.c_int(kind))

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._uint(self.lib.nvmlDeviceGetClockInfo, h, self._c.c_int(kind))

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self._c.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._check(fn(h, self._c.byref(v)), "clock event reasons")
        return v.value


class ClockSampler:
    REASONS = {
        "gpu_idle": 0x1, "applications_clocks_setting": 0x2, "sw_power_cap": 0x4, "hw_slowdown": 0x8,
        "sync_boost": 0x10, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
        "hw_power_brake_slowdown": 0x80, "display_clock_setting": 0x100,
    }

    def __init__(self, index, period_s=0.002):
        self.index, self.period = index, period_s
        self.samples, self.reasons = [], 0
        self.max_mhz = None
        self._stop = threading.Event()
        self._t = None
        self.ok = False
        self.error = None

    def _handle(self, nv):
        """NVML handle of the CUDA device (by UUID; NVML and CUDA number
        devices differently when CUDA_VISIBLE_DEVICES is set)."""
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.index).uuid)
            name = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            return nv.nvmlDeviceGetHandleByUUID(name.encode())
        except Exception:
            pass
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if ids and ids[min(self.index, len(ids) - 1)].isdigit():
            return nv.nvmlDeviceGetHandleByIndex(int(ids[min(self.index, len(ids) - 1)]))
        return nv.nvmlDeviceGetHandleByIndex(self.index)

    def start(self):
        try:
            try:
                import pynvml as nv
                self.api = "pynvml"
            except ImportError:
                nv = NvmlLite()
                self.api = "libnvidia-ml.so.1 via ctypes"
            nv.nvmlInit()
            self._nv = nv
            self._h = self._handle(nv)
            self.max_mhz = nv.nvmlDeviceGetMaxClockInfo(self._h, nv.NVML_CLOCK_SM)
            self.ok = True
        except Exception as exc:
            self.error = repr(exc)[:200]
            return self._start_smi()
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def _start_smi(self):
        """Fallback when NVML cannot be used from Python: nvidia-smi every 50 ms."""
        import subprocess
        sel = []
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            pass
        try:
            self._proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                           "-lms", "50"] + sel, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                          text=True)
            self.ok = "smi"
        except Exception as exc:
            self.error = (self.error or "") + " / " + repr(exc)[:200]
        return self

    def _stop_smi(self):
        self._proc.terminate()
        out, _ = self._proc.communicate(timeout=10)
        mhz, reasons = [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.splitlines():
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                self.max_mhz = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": self.max_mhz,
                "samples": len(mhz), "reasons": sorted(reasons),
                "source": "nvidia-smi every 50 ms during the timed region",
                "nvml_error": self.error}

    def _run(self):
        nv = self._nv
        while not self._stop.is_set():
            try:
                self.samples.append(nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM))
                self.reasons |= nv.nvmlDeviceGetCurrentClocksEventReasons(self._h)
            except Exception:
                pass
            time.sleep(self.period)

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join()
        if self.ok == "smi":
            return self._stop_smi()
        if not self.ok:
            return {"error": self.error}
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                "sm_max_mhz": self.max_mhz, "samples": len(self.samples),
                "reasons": [k for k, v in self.REASONS.items() if self.reasons & v],
                "source": f"NVML ({self.api}), read-only, every 2 ms during the timed region"}


# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device=None):
    """Max of a float over the ranks of the default process group (identity
    for one rank).  Timing only; no data-path collective."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "gloo":
        device = None  # gloo reduces host tensors
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def fp64_gemm_peak(torch, n=8192, reps=3):
    """Measured FP64 FMA rate (ops/s, one fused multiply-add = one op) of a
    cuBLAS FP64 GEMM on this GPU, best of `reps`."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, n ** 3 / (e0.elapsed_time(e1) * 1e-3))
    del a, b
    torch.cuda.empty_cache()
    return best


def cpu_baseline(inst, pt, budget_s=15.0):
    """The CPU oracle as it stands on a bounded sample of the same workload:
    all callbacks and the condensed-matrix rows of whole periods, one period
    at a time, until about `budget_s` of CPU work; single thread."""
    import oracle
    o = oracle.Oracle(inst)
    out = dict(f=np.empty(1), g=np.empty(o.n), c=np.empty(o.m), jv=np.empty(o.nnz_jac), hv=np.empty(o.nnz_hess))
    done, t0 = 0, time.perf_counter()
    while True:
        t = done % inst.T
        o.eval(pt.x, pt.lam, pt.sigma, t, t + 1, out=out)
        o.kkt(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w, t, t + 1)
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or done >= inst.T:
            break
    per_sweep = el / done * inst.T
    return {"value": 1.0 / per_sweep, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} of {inst.T} periods (all callbacks + M rows of each period), "
                      f"{el:.1f} s, extrapolated to the full horizon"}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def adjoint_comparison(torch, vectors=256):
    """The differentiation workload (2,000-bus network, T = 24, seed 5; 256
    (y, v) vectors): matrix-free J^T y (+ load adjoint) and W v against the
    plain form, which materialises J (W) with the callback and multiplies with
    cuSPARSE (torch.sparse CSR): per vector at a fresh point, and amortised
    over the 256 vectors at one point."""
    from paper_2405_14032_b300 import mpopf, synth
    inst = synth.make_instance(5, 2000, 3200, 400, 1200, 24)
    pt = synth.make_point(5, inst)
    h = mpopf.Handle(inst)
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    x, lam = dev(pt.x), dev(pt.lam)
    Y = dev(synth.uniform(5, 5000, vectors * h.m, -1.0, 1.0).reshape(vectors, h.m))
    V = dev(synth.normal(5, 9000, vectors * h.n).reshape(vectors, h.n))
    pat = h.pattern()
    # J^T as CSR: rows = J columns; permutation of the COO values (setup, untimed)
    jr, jc = pat["jac_row"].long(), pat["jac_col"].long()
    order = torch.argsort(jc * h.m + jr)
    jt_crow = torch.zeros(h.n + 1, dtype=torch.int64, device="cuda")
    jt_crow[1:] = torch.cumsum(torch.bincount(jc, minlength=h.n), 0)
    jt_col = jr[order]
    # W symmetric expansion as CSR (duplicates kept; SpMV sums them)
    hr, hc = pat["hess_row"].long(), pat["hess_col"].long()
    off = hr != hc
    er = torch.cat([hr, hc[off]])
    ec = torch.cat([hc, hr[off]])
    src = torch.cat([torch.arange(h.nnz_hess, device="cuda"), torch.nonzero(off).squeeze(1)])
    ho = torch.argsort(er * h.n + ec)
    w_crow = torch.zeros(h.n + 1, dtype=torch.int64, device="cuda")
    w_crow[1:] = torch.cumsum(torch.bincount(er, minlength=h.n), 0)
    w_col, w_src = ec[ho], src[ho]
    jv = torch.empty(h.nnz_jac, dtype=torch.float64, device="cuda")
    hv = torch.empty(h.nnz_hess, dtype=torch.float64, device="cuda")
    gx = torch.empty(h.n, dtype=torch.float64, device="cuda")

    def plain_vjp(y, fresh):
        if fresh:
            h.eval(mpopf.OUT_JAC, x, out=dict(jv=jv))
        A = torch.sparse_csr_tensor(jt_crow, jt_col, jv[order], size=(h.n, h.m))
        return torch.mv(A, y)

    def plain_hvp(v, fresh):
        if fresh:
            h.eval(mpopf.OUT_HESS, x, lam, pt.sigma, out=dict(hv=hv))
        A = torch.sparse_csr_tensor(w_crow, w_col, hv[w_src], size=(h.n, h.n))
        return torch.mv(A, v)

    def timed(fn):
        for k in range(3):
            fn(k)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for k in range(vectors):
            fn(k)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / vectors

    # correctness of the plain form against the matrix-free kernels
    h.eval(mpopf.OUT_JAC, x, out=dict(jv=jv))
    h.eval(mpopf.OUT_HESS, x, lam, pt.sigma, out=dict(hv=hv))
    ref_v = h.vjp(x, Y[0], gx=gx, loads=False)[0].clone()
    pv = plain_vjp(Y[0], False)
    err_v = float((pv - ref_v).abs().max() / ref_v.abs().max())
    ref_h = h.hvp(x, lam, pt.sigma, V[0])
    err_h = float((plain_hvp(V[0], False) - ref_h).abs().max() / ref_h.abs().max())
    gpd = torch.empty(inst.T * inst.net.n_load, dtype=torch.float64, device="cuda")
    gqd = torch.empty_like(gpd)
    res = {
        "workload": "2000-bus / 3200-branch / 400-gen / 1200-load network, T = 24, 256 vectors",
        "vjp_matrix_free_ms": timed(lambda k: lib_vjp(h, x, Y[k], gx, gpd, gqd)),
        "vjp_plain_fresh_ms": timed(lambda k: plain_vjp(Y[k], True)),
        "vjp_plain_amortised_ms": timed(lambda k: plain_vjp(Y[k], False)),
        "hvp_matrix_free_ms": timed(lambda k: h.hvp(x, lam, pt.sigma, V[k], out=gx)),
        "hvp_plain_fresh_ms": timed(lambda k: plain_hvp(V[k], True)),
        "hvp_plain_amortised_ms": timed(lambda k: plain_hvp(V[k], False)),
        "plain_vs_matrix_free_max_rel_diff": max(err_v, err_h),
        "plain": "callback (eval_jac / eval_hess) + cuSPARSE CSR SpMV via torch.sparse",
    }
    res["vjp_speedup_vs_fresh"] = res["vjp_plain_fresh_ms"] / res["vjp_matrix_free_ms"]
    res["hvp_speedup_vs_fresh"] = res["hvp_plain_fresh_ms"] / res["hvp_matrix_free_ms"]

    # All 256 vectors at once: mpopf_vjp_many / mpopf_hvp_many (branch rows
    # recomputed, or read from the J / W the sweep wrote at this point) against
    # the plain form's sparse-times-dense product (J or W formed once,
    # torch.sparse.mm over the 256 columns).
    def timed_once(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(10):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 10 / vectors

    out = h.sweep(x, lam, pt.sigma, dev(pt.sigma_x), dev(pt.dvec), pt.delta_w)
    A_j = torch.sparse_csr_tensor(jt_crow, jt_col, out["jv"][order], size=(h.n, h.m))
    A_w = torch.sparse_csr_tensor(w_crow, w_col, out["hv"][w_src], size=(h.n, h.n))
    YT, VT = Y.t().contiguous(), V.t().contiguous()
    err_many = max(float((h.vjp_many(x, Y, loads=False)[0][5] - h.vjp(x, Y[5], loads=False)[0]).abs().max()),
                   float((h.hvp_many(x, lam, pt.sigma, V)[9] - h.hvp(x, lam, pt.sigma, V[9])).abs().max()))
    res["many"] = {
        "what": "all 256 vectors in one call at one point; ms per vector",
        "vjp_ms": timed_once(lambda: h.vjp_many(x, Y)),
        "vjp_stored_j_ms": timed_once(lambda: h.vjp_many(x, Y, jv=out["jv"])),
        "hvp_ms": timed_once(lambda: h.hvp_many(x, lam, pt.sigma, V)),
        "hvp_stored_w_ms": timed_once(lambda: h.hvp_many(x, lam, pt.sigma, V, hw=out["hv"])),
        "vjp_plain_spmm_ms": timed_once(lambda: torch.sparse.mm(A_j, YT)),
        "hvp_plain_spmm_ms": timed_once(lambda: torch.sparse.mm(A_w, VT)),
        "max_abs_diff_vs_single_products": err_many,
        "plain": "J / W formed once (untimed), cuSPARSE SpMM over the 256 columns via torch.sparse.mm",
    }
    h.close()
    return res


def batched_comparison(torch, reps=20, fp64_peak=None):
    """The batched workload: 64 instances (buses log-uniform in [500, 5000],
    L = 1.6 N, G = 0.2 N, D = 0.6 N, T in {12, 24, 48, 96}; instance k uses seed
    1000 + k) swept through the batch API (one CUDA graph, autotuned schedule)
    against 64 sequential plain sweeps (mpopf_sweep with each handle's default
    schedule: four launches, five for the instances large enough for the
    bus-term launch)."""
    from paper_2405_14032_b300 import mpopf, synth
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    hs, ios = [], []
    units = 0
    alg_bytes = 0
    fp64_ops = 0
    for s in synth.batch_shapes(64):
        inst = synth.make_instance(s["seed"], s["n_bus"], s["n_branch"], s["n_gen"], s["n_load"], s["T"])
        pt = synth.make_point(s["seed"], inst)
        h = mpopf.Handle(inst)
        io = dict(x=dev(pt.x), lam=dev(pt.lam), sigma=pt.sigma, sigma_x=dev(pt.sigma_x), dvec=dev(pt.dvec),
                  delta_w=pt.delta_w)
        io.update(h.new_outputs())
        hs.append(h)
        ios.append(io)
        units += s["T"] * (s["n_bus"] + s["n_branch"] + s["n_gen"])
        alg_bytes += algorithmic_bytes(h.n, h.m, h.nnz_jac, h.nnz_hess, h.nnz_kkt, s["n_load"], s["T"])
        fp64_ops += fp64_ops_per_sweep(s["n_bus"], s["n_branch"], s["n_gen"], s["T"],
                                       bool(h.sweep_schedule()[1] & SCHED_BUS_TERMS))

    def sequential():
        for h, io in zip(hs, ios):
            h.sweep(io["x"], io["lam"], io["sigma"], io["sigma_x"], io["dvec"], io["delta_w"], out=io)

    b = mpopf.Batch(hs)
    b.set_io(ios)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    seq_ms = timed(sequential)
    untuned_ms = timed(b.sweep)
    b.tune(reps=3)
    bat_ms = timed(b.sweep)
    b.status()
    res = {"workload": "64 uneven instances (N log-uniform [500, 5000], T in {12, 24, 48, 96}), all six outputs",
           "instances": 64, "component_periods": units,
           "sequential_ms": seq_ms, "batched_ms": bat_ms, "batched_untuned_ms": untuned_ms,
           "sequential_launches": sum(h.launch_count() for h in hs), "batched_graph_launches": 1,
           "speedup": seq_ms / bat_ms, "schedule": b.schedule(),
           "instance_sweeps_per_s_batched": 64 / (bat_ms * 1e-3),
           "instance_sweeps_per_s_sequential": 64 / (seq_ms * 1e-3),
           "algorithmic_bytes": alg_bytes, "gbs_batched": alg_bytes / (bat_ms * 1e-3) / 1e9,
           "fp64_ops_hand_count": fp64_ops,
           "fp64_gops_batched": fp64_ops / (bat_ms * 1e-3) / 1e9}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    res["schedule_kind"] = ("plain sweeps on parallel graph branches" if res["schedule"]["launches"] == 0 else
                            f"{res['schedule']['launches']} persistent launch(es)")
    res["fp64_frac_of_issue_peak"] = res["fp64_gops_batched"] / fp64_issue_peak(
        sms, measured_peaks().get("sm_max_mhz") or SM_MAX_MHZ)
    if fp64_peak:
        res["fp64_frac_of_dgemm_rate"] = res["fp64_gops_batched"] / (fp64_peak / 1e9)
    b.close()
    for h in hs:
        h.close()
    return res


def graph_sweeps(torch, count=1000):
    """Small sweeps are launch-bound, so they are replayed as one CUDA graph of
    `count` sweeps at perturbed iterates (x_k = x + 1e-3 N(0, 1), drawn on the
    device from a seeded generator), against the same sweeps launched one by
    one: the 2,000-bus, T = 24 network and the single-period (T = 1) 10k-bus
    network."""
    from paper_2405_14032_b300 import mpopf, synth
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    res = {}
    for name, (N, L, G, D, T, seed) in (("2000_bus_T24", (2000, 3200, 400, 1200, 24, 2)),
                                         ("10k_bus_T1", (10000, 16000, 2000, 6000, 1, 3))):
        inst = synth.make_instance(seed, N, L, G, D, T)
        pt = synth.make_point(seed, inst)
        h = mpopf.Handle(inst)
        gen = torch.Generator(device="cuda").manual_seed(seed)
        X = dev(pt.x) + 1e-3 * torch.randn((count, h.n), generator=gen, device="cuda", dtype=torch.float64)
        lam, sx, dv = dev(pt.lam), dev(pt.sigma_x), dev(pt.dvec)
        out = h.new_outputs()
        sweep = lambda k: h.sweep(X[k], lam, pt.sigma, sx, dv, pt.delta_w, out=out)
        for k in range(3):
            sweep(k)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for k in range(count):
            sweep(k)
        e1.record()
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            sweep(0)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for k in range(count):
                sweep(k)
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_ms = e0.elapsed_time(e1)
        alg = algorithmic_bytes(h.n, h.m, h.nnz_jac, h.nnz_hess, h.nnz_kkt, D, T)
        cpu = cpu_baseline(inst, pt, budget_s=4.0)
        res[name] = {"sweeps": count, "n": h.n, "m": h.m, "graph_ms_per_sweep": graph_ms / count,
                     "cpu_oracle": cpu,
                     "plain_ms_per_sweep": plain_ms / count, "sweeps_per_s_graph": count / (graph_ms * 1e-3),
                     "sweeps_per_s_plain": count / (plain_ms * 1e-3),
                     "algorithmic_bytes_per_sweep": alg, "gbs_graph": alg * count / (graph_ms * 1e-3) / 1e9}
        del g
        h.close()
    return res


def point_sweeps(torch, k=40, launches=25):
    """Many sweeps of one network at independent points through
    mpopf_sweep_points: k perturbed iterates (x_j = x + 1e-3 N(0, 1), drawn on
    the device from a seeded generator; lam, sigma_x and dvec the same at every
    point) per call, `launches` calls = k x launches sweeps, for the 2,000-bus
    T = 24 network (1,000 sweeps at the default k and launches) and the 10k-bus
    T = 1 network.  Each call launches the sweep's four kernels once over all
    k points."""
    from paper_2405_14032_b300 import mpopf, synth
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    res = {}
    for name, (N, L, G, D, T, seed) in (("2000_bus_T24", (2000, 3200, 400, 1200, 24, 2)),
                                         ("10k_bus_T1", (10000, 16000, 2000, 6000, 1, 3))):
        inst = synth.make_instance(seed, N, L, G, D, T)
        pt = synth.make_point(seed, inst)
        h = mpopf.Handle(inst)
        gen = torch.Generator(device="cuda").manual_seed(seed)
        X = dev(pt.x) + 1e-3 * torch.randn((k, h.n), generator=gen, device="cuda", dtype=torch.float64)
        rep = lambda a: dev(a).unsqueeze(0).repeat(k, 1).contiguous()
        lam, sx, dv = rep(pt.lam), rep(pt.sigma_x), rep(pt.dvec)
        out = h.new_point_outputs(k)
        sweep = lambda: h.sweep_points(X, lam, pt.sigma, sx, dv, pt.delta_w, out=out)
        for _ in range(3):
            sweep()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(launches):
            sweep()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        alg = algorithmic_bytes(h.n, h.m, h.nnz_jac, h.nnz_hess, h.nnz_kkt, D, T)
        res[name] = {"points_per_call": k, "calls": launches, "sweeps": k * launches,
                     "ms_per_sweep": ms / (k * launches), "sweeps_per_s": k * launches / (ms * 1e-3),
                     "algorithmic_bytes_per_sweep": alg, "gbs": alg * k * launches / (ms * 1e-3) / 1e9}
        del X, lam, sx, dv, out
        h.close()
    return res


def batched_iterates(torch, k=32, launches=32):
    """Throughput of many independent sweeps of the 2,000-bus, T = 24 network
    (seed 2): k handles of the same network at k perturbed iterates, one
    batched sweep (mpopf_batch_sweep, tuned schedule) evaluating all k;
    `launches` batched sweeps = k x launches sweeps.  For evaluations that do
    not depend on each other (scenarios, line searches over several trial
    points); an interior-point iteration's sweeps are sequential and are the
    graph-replayed figures of small_sweeps."""
    from paper_2405_14032_b300 import mpopf, synth
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    inst = synth.config_instance("cfg2")
    pt = synth.make_point(2, inst)
    gen = torch.Generator(device="cuda").manual_seed(2)
    hs, ios = [], []
    for j in range(k):
        h = mpopf.Handle(inst)
        x = dev(pt.x) + 1e-3 * torch.randn(h.n, generator=gen, device="cuda", dtype=torch.float64)
        io = dict(x=x, lam=dev(pt.lam), sigma=pt.sigma, sigma_x=dev(pt.sigma_x), dvec=dev(pt.dvec),
                  delta_w=pt.delta_w)
        io.update(h.new_outputs())
        hs.append(h)
        ios.append(io)
    b = mpopf.Batch(hs)
    b.set_io(ios)
    b.tune(reps=5)
    for _ in range(3):
        b.sweep()
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(launches):
        b.sweep()
    e1.record()
    torch.cuda.synchronize()
    b.status()
    ms = e0.elapsed_time(e1)
    h = hs[0]
    alg = algorithmic_bytes(h.n, h.m, h.nnz_jac, h.nnz_hess, h.nnz_kkt, inst.net.n_load, inst.T)
    res = {"workload": f"2,000-bus network, T = 24: {k} iterates per batched sweep, {launches} batched sweeps",
           "sweeps": k * launches, "ms_per_sweep": ms / (k * launches), "sweeps_per_s": k * launches / (ms * 1e-3),
           "algorithmic_bytes_per_sweep": alg, "gbs": alg * k * launches / (ms * 1e-3) / 1e9,
           "schedule": b.schedule()}
    b.close()
    for h in hs:
        h.close()
    return res


# Synthetic networks with the sizes of the benchmark cases of the paper's
# Table II (bus counts from the case names; branch and generator counts the
# commonly reported sizes of those public cases; loads at 0.6 of the buses, as
# in every synthetic network here) and the horizons the paper runs them with.
TABLE2_SHAPES = [("case30", 30, 41, 6, 30), ("case118", 118, 186, 54, 168), ("case118", 118, 186, 54, 10080),
                 ("case1354", 1354, 1991, 260, 30), ("case9241", 9241, 16049, 1445, 30),
                 ("case9241", 9241, 16049, 1445, 180)]


def table2_shapes(torch, reps=10):
    """The full sweep on seeded synthetic networks shaped like the paper's
    Table II cases (the case files themselves are not available): time per
    sweep (CUDA events, mean of `reps` after 3 warm-ups) and algorithmic
    bandwidth."""
    from paper_2405_14032_b300 import mpopf, synth
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    peak = measured_peaks().get("hbm_gbs")
    out = {}
    for k, (case, N, L, G, T) in enumerate(TABLE2_SHAPES):
        D = round(0.6 * N)
        inst = synth.make_instance(50 + k, N, L, G, D, T)
        pt = synth.make_point(50 + k, inst)
        h = mpopf.Handle(inst)
        x, lam, sx, dv = dev(pt.x), dev(pt.lam), dev(pt.sigma_x), dev(pt.dvec)
        res = h.new_outputs()
        for _ in range(3):
            h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=res)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(reps):
            h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=res)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        alg = algorithmic_bytes(h.n, h.m, h.nnz_jac, h.nnz_hess, h.nnz_kkt, D, T)
        gbs = alg / (ms * 1e-3) / 1e9
        out[f"{case}_T{T}"] = {"n_bus": N, "n_branch": L, "n_gen": G, "n_load": D, "T": T, "n": h.n, "m": h.m,
                               "ms_per_sweep": ms, "sweeps_per_s": 1e3 / ms, "gbs": gbs,
                               "hbm_frac": gbs / peak if peak else None}
        del res, x, lam, sx, dv
        h.close()
    return out


def ipm_step_timing(torch, reps=5):
    """One whole interior-point step on the 2,000-bus, T = 24 network (seed 2)
    at an interior point (interval midpoints, unit duals, delta_w = 50 so that M
    is positive definite): Sigma/D/C, the sweep, the condensed right-hand side,
    the library Cholesky factorisation of M (cuSOLVER, standing in for cuDSS)
    and solve, and the step recovery."""
    from paper_2405_14032_b300 import mpopf, synth
    inst = synth.config_instance("cfg2")
    h = mpopf.Handle(inst)
    pat = h.pattern()
    eps, mu, dw, dc = 1e-2, 0.05, 50.0, 1e-4
    xl, xu, gl, gu = (pat[k] for k in ("xl", "xu", "gl", "gu"))

    def interior(lo, hi, other):
        fl, fu = torch.isfinite(lo), torch.isfinite(hi)
        v = torch.where(fl & fu, 0.5 * (lo + hi), other)
        v = torch.where(fl & ~fu, lo + 0.5, v)
        return torch.where(~fl & fu, hi - 0.5, v)

    eq = gl == gu
    sl, su = torch.where(eq, gl - eps, gl), torch.where(eq, gu + eps, gu)
    pt = synth.make_point(2, inst)
    x = interior(xl, xu, torch.as_tensor(pt.x, device="cuda"))
    s = interior(sl, su, torch.zeros_like(sl))
    one = lambda b: torch.where(torch.isfinite(b), 1.0, 0.0).double()
    z = [one(xl), one(xu), one(sl), one(su)]
    y = torch.as_tensor(pt.lam, device="cuda")
    neg_y = -y
    out = h.new_outputs()
    sigx, dvec, cvec, recip = h.ipm_prepare(x, s, *z, dw, dc, eps)
    h.sweep(x, neg_y, 1.0, sigx, dvec, dw, out=out)
    rhs = h.ipm_rhs(x, s, y, out["grad"], out["c"], recip, dvec, cvec, mu)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pivot = h.kkt_factor(out["kv"])  # first call: ordering and symbolic analysis
    first_s = time.perf_counter() - t0
    if pivot >= 0:
        h.close()
        return {"error": f"M not positive definite (pivot row {pivot})"}
    dx = h.kkt_solve(rhs)
    rec = h.ipm_recover(x, s, y, *z, out["c"], recip, cvec, dx, mu, dw, dc)
    parts = {k: 0.0 for k in ("prepare", "sweep", "rhs", "factor", "solve", "recover")}
    torch.cuda.synchronize()
    for _ in range(reps):
        marks = [time.perf_counter()]
        h.ipm_prepare(x, s, *z, dw, dc, eps, recip=recip)
        torch.cuda.synchronize(); marks.append(time.perf_counter())
        h.sweep(x, neg_y, 1.0, sigx, dvec, dw, out=out)
        torch.cuda.synchronize(); marks.append(time.perf_counter())
        h.ipm_rhs(x, s, y, out["grad"], out["c"], recip, dvec, cvec, mu, out=rhs)
        torch.cuda.synchronize(); marks.append(time.perf_counter())
        h.kkt_factor(out["kv"])
        torch.cuda.synchronize(); marks.append(time.perf_counter())
        h.kkt_solve(rhs, out=dx)
        torch.cuda.synchronize(); marks.append(time.perf_counter())
        h.ipm_recover(x, s, y, *z, out["c"], recip, cvec, dx, mu, dw, dc, out=rec)
        torch.cuda.synchronize(); marks.append(time.perf_counter())
        for k, a, b in zip(parts, marks[:-1], marks[1:]):
            parts[k] += (b - a) * 1e3 / reps
    h.close()
    return {"kind": ("functional check of one whole interior-point step through the library factorisation "
                     "(a stand-in for the paper's cuDSS), not a performance figure of this library's kernels"),
            "workload": "2000-bus / 3200-branch / 400-gen / 1200-load network, T = 24 (n = 422,400)",
            "ordering_and_analysis_s": first_s, "ms": parts, "step_ms": sum(parts.values()),
            "timing": "host clock around each synchronised call (the factorisation synchronises itself)",
            "factorisation": "cuSOLVER sparse Cholesky (csrchol), METIS nested-dissection ordering"}


def unfused_timing(torch, h, x, lam, sigma, sx, dv, dw, out, reps=20):
    """The six callbacks called one by one (f, grad f, c, J, W, then M, which
    recomputes the branch derivatives), as an NLP solver without the fused
    sweep would call them, against the one fused sweep."""
    from paper_2405_14032_b300 import mpopf

    def seq():
        for bit in (mpopf.OUT_OBJ, mpopf.OUT_GRAD, mpopf.OUT_CONS, mpopf.OUT_JAC, mpopf.OUT_HESS, mpopf.OUT_KKT):
            h.eval(bit, x, lam, sigma, sx, dv, dw, out=out)

    for _ in range(3):
        seq()
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(reps):
        seq()
    e1.record()
    torch.cuda.synchronize()
    return {"unfused_ms": e0.elapsed_time(e1) / reps,
            "calls": "mpopf_eval with one output bit each: OBJ, GRAD, CONS, JAC, HESS, KKT"}


def csc_timing(torch, h, out, reps=20):
    """COO -> CSC compression of the benchmark instance's J and W values (the
    pattern built once on the host, untimed; each compression one kernel)."""
    from paper_2405_14032_b300 import mpopf
    res = {}
    for which, key, nnz_coo in ((mpopf.CSC_JAC, "jv", h.nnz_jac), (mpopf.CSC_HESS, "hv", h.nnz_hess)):
        t0 = time.perf_counter()
        nnz = h.csc_pattern(which)["nnz"]
        build_s = time.perf_counter() - t0
        dst = torch.empty(nnz, dtype=torch.float64, device="cuda")
        for _ in range(3):
            h.coo_to_csc(which, out[key], out=dst)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(reps):
            h.coo_to_csc(which, out[key], out=dst)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        # COO values read once, source index read once, CSC values written once (+ run starts for W)
        alg = 8 * nnz_coo + 4 * nnz_coo + 8 * nnz + (8 * (nnz + 1) if nnz != nnz_coo else 0)
        res["jac" if which == mpopf.CSC_JAC else "hess"] = {
            "nnz_coo": nnz_coo, "nnz_csc": nnz, "ms": ms, "gbs": alg / (ms * 1e-3) / 1e9,
            "pattern_build_s": build_s}
    return res


def ipm_timing(torch, h, reps=50, eps=1e-2, mu=0.05, dw=1e-3, dc=1e-4):
    """The interior-point algebra around M (Sec. III-B) on the benchmark
    instance: mpopf_ipm_prepare, mpopf_ipm_rhs and mpopf_ipm_recover at an
    interior point built from the pattern's bounds (midpoints of finite
    intervals, 0.5 inside one-sided bounds, duals 1 on finite bounds), each
    timed alone with CUDA events over reps calls."""
    pat = h.pattern()
    xl, xu, gl, gu = (pat[k] for k in ("xl", "xu", "gl", "gu"))
    inf = float("inf")

    def interior(lo, hi, other):
        fl, fu = torch.isfinite(lo), torch.isfinite(hi)
        v = torch.where(fl & fu, 0.5 * (lo + hi), other)
        v = torch.where(fl & ~fu, lo + 0.5, v)
        return torch.where(~fl & fu, hi - 0.5, v)

    eq = gl == gu
    sl, su = torch.where(eq, gl - eps, gl), torch.where(eq, gu + eps, gu)
    x = interior(xl, xu, torch.zeros_like(xl))
    s = interior(sl, su, torch.zeros_like(sl))
    one = lambda b: torch.where(torch.isfinite(b), 1.0, 0.0).double()
    zlx, zux, zls, zus = one(xl), one(xu), one(sl), one(su)
    y = torch.full_like(s, 0.25)
    from paper_2405_14032_b300 import mpopf
    out = h.eval(mpopf.OUT_OBJ | mpopf.OUT_GRAD | mpopf.OUT_CONS, x)
    sigx, dvec, cvec, recip = h.ipm_prepare(x, s, zlx, zux, zls, zus, dw, dc, eps)
    rhs = h.ipm_rhs(x, s, y, out["grad"], out["c"], recip, dvec, cvec, mu)
    dx = rhs.clone()
    rec = h.ipm_recover(x, s, y, zlx, zux, zls, zus, out["c"], recip, cvec, dx, mu, dw, dc)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    n, m = h.n, h.m
    t_prep = timed(lambda: h.ipm_prepare(x, s, zlx, zux, zls, zus, dw, dc, eps, recip=recip))
    t_rhs = timed(lambda: h.ipm_rhs(x, s, y, out["grad"], out["c"], recip, dvec, cvec, mu, out=rhs))
    t_rec = timed(lambda: h.ipm_recover(x, s, y, zlx, zux, zls, zus, out["c"], recip, cvec, dx, mu, dw, dc, out=rec))
    # one interior-point iteration without the factorisation: Sigma/D/C, the
    # full sweep at lambda = -y (W, J, M, grad f, c), the condensed right-hand
    # side and the step recovery (dx stands in for the solve's result)
    neg_y = -y
    sw = h.new_outputs()

    def iteration(stored):
        sx_, dv_, cv_, rc_ = h.ipm_prepare(x, s, zlx, zux, zls, zus, dw, dc, eps, recip=recip)
        h.sweep(x, neg_y, 1.0, sx_, dv_, dw, out=sw)
        jv = sw["jv"] if stored else None
        h.ipm_rhs(x, s, y, sw["grad"], sw["c"], rc_, dv_, cv_, mu, out=rhs, jv=jv)
        h.ipm_recover(x, s, y, zlx, zux, zls, zus, sw["c"], rc_, cv_, dx, mu, dw, dc, out=rec, jv=jv)

    t_iter = timed(lambda: iteration(False))
    t_iter_jv = timed(lambda: iteration(True))
    jvs = sw["jv"]  # J at x from the last sweep
    t_rhs_jv = timed(lambda: h.ipm_rhs(x, s, y, out["grad"], out["c"], recip, dvec, cvec, mu, out=rhs, jv=jvs))
    t_rec_jv = timed(lambda: h.ipm_recover(x, s, y, zlx, zux, zls, zus, out["c"], recip, cvec, dx, mu, dw, dc,
                                           out=rec, jv=jvs))
    gx = torch.empty_like(x)
    t_vjp = timed(lambda: h.vjp(x, y, gx=gx, loads=False))
    jvo = torch.empty_like(y)
    t_jvp = timed(lambda: h.jvp(x, dx, out=jvo))
    t_vjp_jv = timed(lambda: h.vjp(x, y, gx=gx, loads=False, jv=jvs))
    t_jvp_jv = timed(lambda: h.jvp(x, dx, out=jvo, jv=jvs))
    # each array read or written once (the J products: x, the vector and the result)
    b_prep = 8 * (8 * n + 9 * m)
    b_rhs = 8 * (8 * m + (n + m + n) + 5 * n)
    b_rec = 8 * ((n + n + m) + 13 * m + 7 * n)
    g = lambda b, t: b / (t * 1e-3) / 1e9
    return {"prepare_ms": t_prep, "rhs_ms": t_rhs, "recover_ms": t_rec, "vjp_ms": t_vjp, "jvp_ms": t_jvp,
            "iteration_ms_without_factorisation": t_iter, "iteration_ms_stored_j": t_iter_jv,
            "rhs_stored_j_ms": t_rhs_jv, "recover_stored_j_ms": t_rec_jv, "vjp_stored_j_ms": t_vjp_jv,
            "jvp_stored_j_ms": t_jvp_jv,
            "prepare_gbs": g(b_prep, t_prep), "rhs_gbs": g(b_rhs, t_rhs), "recover_gbs": g(b_rec, t_rec),
            "algorithmic_bytes": {"prepare": b_prep, "rhs": b_rhs, "recover": b_rec},
            "note": "rhs and recover include one matrix-free J product each (J^T w, J dx; timed alone as "
                    "vjp_ms / jvp_ms); all divisions in prepare"}


def lib_vjp(h, x, y, gx, gpd, gqd):
    from paper_2405_14032_b300 import mpopf
    import torch
    s = mpopf._stream_ptr(None)
    mpopf._check(mpopf.lib().mpopf_vjp(h.h, x.data_ptr(), y.data_ptr(), gx.data_ptr(), gpd.data_ptr(),
                                       gqd.data_ptr(), s), "mpopf_vjp")


# ---------------------------------------------------------------------------
PARALLELISM = {"single": "single", "replicas": "replicas{n}", "shards": "period-shards{n} (halo + f all-reduce)"}
L2_NOTE = "inputs + outputs 2.7 GB per step > 126 MB L2; no flush"


def workload_config(T, world, mode):
    """The `config` object of both arms: the workload and how it is spread over
    the GPUs."""
    return {"workload": f"mpopf_sweep_10k_bus_T{T}", **WORKLOAD, "n_periods": T,
            "parallelism": PARALLELISM[mode].format(n=world), "l2": L2_NOTE}


def run_mode(args, world):
    return (args.mode or "shards") if world > 1 else "single"


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle on this workload, timed on the host
    cores; each step evaluates every callback and the M rows of one period
    (a bounded sample), steps rotate over the periods."""
    if rank != 0:
        return 0
    from paper_2405_14032_b300 import synth
    import oracle
    inst = synth.make_instance(WORKLOAD["seed"], WORKLOAD["n_bus"], WORKLOAD["n_branch"], WORKLOAD["n_gen"],
                               WORKLOAD["n_load"], args.periods)
    pt = synth.make_point(WORKLOAD["seed"], inst)
    o = oracle.Oracle(inst)
    out = dict(f=np.empty(1), g=np.empty(o.n), c=np.empty(o.m), jv=np.empty(o.nnz_jac), hv=np.empty(o.nnz_hess))

    def step(k):
        t = k % inst.T
        o.eval(pt.x, pt.lam, pt.sigma, t, t + 1, out=out)
        o.kkt(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w, t, t + 1)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    el = time.perf_counter() - t0
    sweeps = args.steps / inst.T
    value = sweeps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "strong" if run_mode(args, world) == "shards" else "weak",
            "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(inst.T, world, run_mode(args, world)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: all callbacks + M rows of one period of the horizon"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def fp64_ops_per_sweep(N, L, G, T, bus_terms=False):
    """Hand count of the FP64 operations of one full sweep over T periods
    (bus_terms: the schedule forms the bus-end products in their own launch)."""
    bus = FP64_OPS_PER_BUS_PERIOD + (FP64_OPS_BUS_TERMS_PER_BUS_PERIOD if bus_terms else 0)
    return branch_ops_per_element(bus_terms) * T * L + bus * T * N + FP64_OPS_PER_GEN_PERIOD * T * G


def run_ours(args, world, rank, local):
    import torch
    local = local % max(torch.cuda.device_count(), 1)  # ranks beyond the visible GPUs share them
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(args.dist_backend)
        dist.barrier()  # a collective of every rank first: the halo exchanges' batched P2P calls never are
    dev = torch.device("cuda", local)
    from paper_2405_14032_b300 import mpopf, shard, synth

    mode = run_mode(args, world)
    T = args.periods
    inst = synth.make_instance(WORKLOAD["seed"], WORKLOAD["n_bus"], WORKLOAD["n_branch"], WORKLOAD["n_gen"],
                               WORKLOAD["n_load"], T)
    pt = synth.make_point(WORKLOAD["seed"], inst)
    span = shard.split(T, world)[rank] if mode == "shards" else None
    plan = mpopf.shard_plan(inst.net, T, *span) if span else None
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    h = mpopf.Handle(inst, shard=span)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    n, m = h.n, h.m
    D = inst.net.n_load
    todev = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)
    # two perturbed iterates, alternated step by step
    xs_whole = [pt.x, synth.perturb(WORKLOAD["seed"], pt.x, 0)]
    if plan:
        local = lambda a, what, k: shard.scatter(plan, what, a, np.zeros(k))
        xs = [todev(local(x, "x", n)) for x in xs_whole]
        lam, sx, dv = todev(local(pt.lam, "rows", m)), todev(local(pt.sigma_x, "x", n)), todev(local(pt.dvec, "rows", m))
    else:
        xs = [todev(x) for x in xs_whole]
        lam, sx, dv = todev(pt.lam), todev(pt.sigma_x), todev(pt.dvec)
    out = h.new_outputs()
    launches = h.launch_count()
    W = (span[1] - span[0]) if span else T   # periods this rank evaluates
    whole = mpopf.shard_plan(inst.net, T, 0, T)  # sizes of the whole-horizon model (host only)
    alg_whole = algorithmic_bytes(whole["n"], whole["m"], whole["nnz_jac"], whole["nnz_hess"], whole["nnz_kkt"], D, T)

    # shards: the halo exchange runs on a stream of its own, overlapping the
    # branch and bus kernels (only the generator work waits for it); the sum
    # of the partial objectives runs on that stream too, after the sweep,
    # without holding the next sweep back
    halo_stream = torch.cuda.Stream() if plan else None
    halo_event = torch.cuda.Event() if plan else None
    f_whole = torch.zeros(1, dtype=torch.float64, device=dev) if plan else None

    def step(k):
        x = xs[k % 2]
        if plan:
            shard.exchange_halos_async(plan, x, dv, rank, world, halo_stream, halo_event)
            if k == 0:
                h.set_gen_dependency(halo_event)
        h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=out)
        if plan:
            shard.reduce_objective_async(out["f"], f_whole, halo_stream)

    def drain():
        if plan:  # the timed region ends after the last sum of the objective
            torch.cuda.current_stream().wait_stream(halo_stream)

    fp64_peak = fp64_gemm_peak(torch) if rank == 0 else None
    probe_rate, _ = mpopf.fp64_issue_rate(16384)

    for k in range(args.warmup):
        step(k)
    drain()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local).start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(k)
    drain()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world, dev)
    ms_step = ms / args.steps
    # whole-job sweeps per second: N replicas make N sweeps per step; N shards
    # make one sweep of the whole horizon per step
    value = (world if mode == "replicas" else 1) * args.steps / (ms * 1e-3)

    # per-kernel times: a separate pass with a CUDA-event pair around every
    # launch on the caller's stream (not inside the timed region)
    h.profile_start(args.steps * launches)
    for k in range(args.steps):
        h.sweep(xs[k % 2], lam, pt.sigma, sx, dv, pt.delta_w, out=out)
    torch.cuda.synchronize()
    prof = h.profile_stop()

    # dominant kernel and its roofline
    top = max(prof, key=lambda k: prof[k][0])
    top_ms = prof[top][0] / max(prof[top][1], 1)
    roof = None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    derived = fp64_issue_peak(sms, measured_peaks().get("sm_max_mhz") or SM_MAX_MHZ)
    peak = probe_rate / 1e9
    bus_terms = bool(h.sweep_schedule()[1] & SCHED_BUS_TERMS)
    if top == "branch":
        ops = branch_ops_per_element(bus_terms) * W * inst.net.n_branch
        achieved = ops / (top_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "kernel": "k_branch (branch x period)", "achieved": achieved, "peak": peak,
                "unit": "Gop/s (FP64 fma/add/mul)", "frac": achieved / peak,
                "traffic": ncu_traffic(W), "ops_per_launch": ops, "avg_launch_ms": top_ms,
                "peak_source": ("measured: the library's DFMA-chain probe (mpopf_fp64_issue_rate), "
                                "FP64 thread-instructions per second, same run"),
                "peak_derived": derived,
                "peak_derived_source": (f"{FP64_PER_CYCLE_PER_SM} FP64 thread-instructions per cycle per SM x "
                                        f"{sms} SMs x max SM clock"),
                "peak_measured_dgemm": fp64_peak / 1e9 if fp64_peak else None,
                "frac_of_measured_dgemm": achieved / (fp64_peak / 1e9) if fp64_peak else None}
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    gbs = alg_whole / (ms_step * 1e-3) / 1e9 * (world if mode == "replicas" else 1)
    floor_ms = fp64_ops_per_sweep(inst.net.n_bus, inst.net.n_branch, inst.net.n_gen, W, bus_terms) / probe_rate * 1e3
    hbm = {"algorithmic_bytes_per_sweep": alg_whole, "gbs": gbs, "peak_gbs": hbm_peak,
           "frac": gbs / hbm_peak if hbm_peak else None, "peak_source": "MEASURED_PEAKS.json",
           "nominal_gbs": 7700.0, "frac_nominal": gbs / 7700.0}
    if mode != "shards":
        # the FP64 work alone bounds the sweep from below; at that floor the
        # algorithmic bytes would move at this fraction of the HBM peak
        hbm.update({"fp64_ops_per_sweep": fp64_ops_per_sweep(inst.net.n_bus, inst.net.n_branch, inst.net.n_gen, T,
                                                             bus_terms),
                    "fp64_floor_ms": floor_ms,
                    "attainable_frac": (alg_whole / (floor_ms * 1e-3) / 1e9) / hbm_peak if hbm_peak else None,
                    "frac_of_fp64_floor": floor_ms / ms_step})

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if mode == "shards" else "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(T, world, mode),
            "sizes": {"n": whole["n"], "m": whole["m"], "nnz_jac": whole["nnz_jac"], "nnz_hess": whole["nnz_hess"],
                      "nnz_kkt": whole["nnz_kkt"]},
            "inputs": "two perturbed iterates alternated step by step, resident in HBM",
            "hbm": hbm,
            "roofline": roof,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1] > 0},
            "kernels_note": ("a separate pass after the timed region, CUDA events around every launch on the "
                             "caller's stream; k_gen and k_fsum run on the handle's side stream, overlapped with "
                             "k_bus, and are not timed per kernel (see the ncu launch list for their serialised "
                             "durations)"),
            "clocks": clk,
            "gpu_launches": launches * args.steps,
            "setup": {"seconds": setup_s,
                      "what": ("mpopf_setup once per handle: layout, templates and incidence lists on the host, "
                               "the J / W / M patterns and bounds expanded on the GPU")}}
    if plan:
        line["shards"] = {"periods_per_rank": [b - a for a, b in shard.split(T, world)],
                          "halo_doubles_each_way": plan["halo_len"] * plan["halo_blocks"],
                          "exchange": "torch.distributed batch_isend_irecv (NCCL) on a stream of its own, "
                                      "overlapping the branch and bus kernels (the generator work waits "
                                      "for it); f summed by an all_reduce on that stream after the sweep, "
                                      "not holding the next sweep back"}

    line["e2e"] = e2e_host(torch, args, world, rank, dev, h, plan, pt, inst, mode)
    if rank == 0:
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(inst, pt)
            line["adjoint"] = adjoint_comparison(torch)
            line["batched"] = batched_comparison(torch, fp64_peak=fp64_peak)
            line["ipm"] = ipm_timing(torch, h)
            line["small_sweeps"] = graph_sweeps(torch)
            line["small_sweeps"]["2000_bus_T24_batched_iterates"] = batched_iterates(torch)
            line["small_sweeps"]["points"] = point_sweeps(torch)
            line["csc"] = csc_timing(torch, h, out)
            line["unfused"] = unfused_timing(torch, h, xs[0], lam, pt.sigma, sx, dv, pt.delta_w, out)
            line["unfused"]["fused_ms"] = ms_step
            line["unfused"]["speedup_fused"] = line["unfused"]["unfused_ms"] / ms_step
            line["ipm_step"] = ipm_step_timing(torch)
            line["table2_shapes"] = table2_shapes(torch)
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def e2e_host(torch, args, world, rank, dev, h, plan, pt, inst, mode):
    """End to end through the public API with host buffers: every step copies
    that step's inputs in from pinned host memory and all outputs back.  One
    rank (or replicas): mpopf_sweep_host (pipelined copies inside the call).
    Shards: each rank copies its local inputs in, exchanges the halo, sweeps
    its shard (mpopf_sweep), sums f and copies its owned outputs out."""
    from paper_2405_14032_b300 import shard
    pin = lambda k: torch.empty(k, dtype=torch.float64, pin_memory=True)
    n, m = h.n, h.m
    stream = torch.cuda.current_stream()
    hout = dict(f=pin(1), grad=pin(n), c=pin(m), jv=pin(h.nnz_jac), hv=pin(h.nnz_hess), kv=pin(h.nnz_kkt))
    if plan is None:
        hx, hl, hs, hd = pin(n), pin(m), pin(n), pin(m)
        hx.numpy()[:], hl.numpy()[:], hs.numpy()[:], hd.numpy()[:] = pt.x, pt.lam, pt.sigma_x, pt.dvec
        hostnp = {k: v.numpy() for k, v in hout.items()}
        run = lambda: h.sweep_host(hx.numpy(), hl.numpy(), pt.sigma, hs.numpy(), hd.numpy(), pt.delta_w, hostnp,
                                   stream=stream)
        h2d, d2h = 8 * (2 * n + 2 * m), 8 * (1 + n + m + h.nnz_jac + h.nnz_hess + h.nnz_kkt)
        api = "mpopf_sweep_host (pinned host buffers, all inputs in, all outputs out; every rank)"
    else:
        loc = lambda a, what, k: torch.from_numpy(shard.scatter(plan, what, a, np.zeros(k)))
        hx, hl, hs, hd = (loc(pt.x, "x", n), loc(pt.lam, "rows", m), loc(pt.sigma_x, "x", n),
                          loc(pt.dvec, "rows", m))
        hx, hl, hs, hd = (t.pin_memory() for t in (hx, hl, hs, hd))
        dx, dl, ds, dd = (torch.empty(t.numel(), dtype=torch.float64, device=dev) for t in (hx, hl, hs, hd))
        dout = h.new_outputs()

        def run():
            for d_, h_ in ((dx, hx), (dl, hl), (ds, hs), (dd, hd)):
                d_.copy_(h_, non_blocking=True)
            shard.exchange_halos(plan, dx, dd, rank, world)
            h.sweep(dx, dl, pt.sigma, ds, dd, pt.delta_w, out=dout)
            shard.reduce_objective(dout["f"])
            for k, v in dout.items():
                hout[k].copy_(v, non_blocking=True)
            torch.cuda.synchronize()
        h2d = 8 * (2 * n + 2 * m)
        d2h = 8 * (1 + n + m + h.nnz_jac + h.nnz_hess + h.nnz_kkt)
        api = ("shard handle: pinned host -> device copies of the shard's inputs, halo exchange, mpopf_sweep, "
               "f all-reduce, device -> pinned host copies of its outputs; every rank")
    run()
    torch.cuda.synchronize()
    ke = max(1, args.e2e_steps)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        run()
    el = max_over_ranks(time.perf_counter() - t0, world, dev)
    per = world if mode == "replicas" else 1
    e2e = {"value": per * ke / el, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "d2h_gbs": d2h * ke / el / 1e9, "h2d_gbs": h2d * ke / el / 1e9,
           "bytes_note": "per rank" if world > 1 else "",
           "steps": ke, "ranks": world, "api": api}
    del hout
    e2e.update(link_rates(torch))
    if e2e.get("link_d2h_gbs"):
        e2e["d2h_frac_of_link"] = e2e["d2h_gbs"] / e2e["link_d2h_gbs"]
    return e2e


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
