"""ctypes front of the plain FP64 CPU oracle (``mpopf_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports it.
The oracle shares no code with the CUDA library; both are fed by the seeded
input generator :mod:`paper_2405_14032_b300.synth`.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpopf_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_mpopf.so")
_FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]

_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["g++", *_FLAGS, "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Set the ctypes signatures of an oracle library."""
    sigs = {
        "orc_new": (_P, [_P] * 10),
        "orc_free": (None, [_P]),
        "orc_sizes": (None, [_P, _P]),
        "orc_bounds": (None, [_P, _P, _P, _P, _P]),
        "orc_jac_pattern": (None, [_P, _P, _P]),
        "orc_hess_pattern": (None, [_P, _P, _P]),
        "orc_jac_rowptr": (None, [_P, _P]),
        "orc_eval": (None, [_P, _I64, _I64, _P, _P, _D, _P, _P, _P, _P, _P]),
        "orc_kkt_new": (_P, [_P, _I64, _I64, _P, _P, _D, _P, _P, _D]),
        "orc_kkt_sizes": (None, [_P, _P]),
        "orc_kkt_copy": (None, [_P, _P, _P, _P, _P]),
        "orc_kkt_free": (None, [_P]),
        "orc_window_rows": (_I64, [_P, _I64, _I64]),
        "orc_vjp": (None, [_P, _I64, _I64, _P, _P, _P, _P, _P]),
        "orc_hvp": (None, [_P, _I64, _I64, _P, _P, _D, _P, _P]),
        "orc_jvp": (None, [_P, _I64, _I64, _P, _P, _P, _P, _P]),
        "orc_sincos": (None, [_P, _I64, _P, _P]),
        "orc_gradlag": (None, [_P, _P, _P, _D, _P]),
        "orc_gradlag_cstep": (None, [_P, _P, _P, _D, _P, _D, _P]),
        "orc_cons_textbook": (None, [_P, _P, _P]),
        "orc_cons_cstep": (None, [_P, _P, _P, _D, _P]),
        "orc_obj_textbook": (_D, [_P, _P]),
        "orc_branch_terms": (None, [_P, _P]),
        "orc_csc_nnz": (ctypes.c_int64, [_P, ctypes.c_int32]),
        "orc_csc": (None, [_P, ctypes.c_int32, _P, _P, _P, _P]),
        "orc_ipm_prepare": (None, [_P] * 7 + [_D, _D, _D] + [_P] * 5),
        "orc_ipm_rhs": (None, [_P] * 10 + [_D, _D, _D, _D, _P, _P]),
        "orc_ipm_recover": (None, [_P] * 10 + [_D, _D, _D, _D] + [_P] * 6),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def build_variant(source: str, directory: str) -> str:
    """Compile a modified copy of the oracle source (the tests plant mistakes in
    it to show that the pins catch them); returns the library path."""
    src = os.path.join(directory, "oracle_variant.cpp")
    out = os.path.join(directory, "liboracle_variant.so")
    with open(src, "w") as fh:
        fh.write(source)
    subprocess.check_call(["g++", *_FLAGS, "-o", out, src])
    return out


@contextlib.contextmanager
def using(path: str):
    """Oracle objects created inside use the library at `path`."""
    global _lib
    saved = load()
    _lib = _bind(ctypes.CDLL(path))
    try:
        yield _lib
    finally:
        _lib = saved


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One model (network, horizon, loads) held by the C++ oracle."""

    def __init__(self, inst):
        lib = load()
        self._lib = lib  # the library this object's handle belongs to
        net = inst.net
        self.inst = inst
        self.T = inst.T
        self._keep = [
            np.array([net.n_bus, net.n_branch, net.n_gen, net.n_load, net.ref_bus, inst.T], dtype=np.int64),
            _f64(np.concatenate([net.bus_gs, net.bus_bs, net.bus_vmin, net.bus_vmax])),
            np.ascontiguousarray(np.concatenate([net.br_f, net.br_t]), dtype=np.int32),
            _f64(np.concatenate([net.br_r, net.br_x, net.br_b, net.br_tap, net.br_shift, net.br_smax,
                                 net.br_angmin, net.br_angmax])),
            np.ascontiguousarray(net.gen_bus, dtype=np.int32),
            _f64(np.concatenate([net.gen_c2, net.gen_c1, net.gen_c0, net.gen_pmin, net.gen_pmax,
                                 net.gen_qmin, net.gen_qmax, net.gen_ramp])),
            np.ascontiguousarray(net.load_bus, dtype=np.int32),
            _f64(inst.pd), _f64(inst.qd),
            None if net.gen_qramp is None else _f64(net.gen_qramp),
        ]
        self.h = lib.orc_new(*[_ptr(a) for a in self._keep])
        out = np.zeros(4, np.int64)
        lib.orc_sizes(self.h, _ptr(out))
        self.n, self.m, self.nnz_jac, self.nnz_hess = (int(v) for v in out)

    def __del__(self):
        if getattr(self, "h", None) and getattr(self, "_lib", None) is not None:
            self._lib.orc_free(self.h)
            self.h = None

    # -- patterns ---------------------------------------------------------
    def bounds(self):
        xl, xu = np.empty(self.n), np.empty(self.n)
        gl, gu = np.empty(self.m), np.empty(self.m)
        self._lib.orc_bounds(self.h, _ptr(xl), _ptr(xu), _ptr(gl), _ptr(gu))
        return xl, xu, gl, gu

    def jac_pattern(self):
        r = np.empty(self.nnz_jac, np.int32)
        c = np.empty(self.nnz_jac, np.int32)
        self._lib.orc_jac_pattern(self.h, _ptr(r), _ptr(c))
        return r, c

    def hess_pattern(self):
        r = np.empty(self.nnz_hess, np.int32)
        c = np.empty(self.nnz_hess, np.int32)
        self._lib.orc_hess_pattern(self.h, _ptr(r), _ptr(c))
        return r, c

    def jac_rowptr(self):
        rp = np.empty(self.m + 1, np.int64)
        self._lib.orc_jac_rowptr(self.h, _ptr(rp))
        return rp

    # -- callbacks --------------------------------------------------------
    def eval(self, x, lam, sigma, t0=0, t1=None, want=("f", "g", "c", "jv", "hv"), out=None):
        """Outputs restricted to periods [t0, t1); entries outside stay NaN
        (or keep whatever `out`, a dict of preallocated arrays, held)."""
        t1 = self.T if t1 is None else t1
        x, lam = _f64(x), _f64(lam)
        if out is not None:
            f, g, c, jv, hv = (out.get(k) for k in ("f", "g", "c", "jv", "hv"))
        else:
            f = np.full(1, np.nan) if "f" in want else None
            g = np.full(self.n, np.nan) if "g" in want else None
            c = np.full(self.m, np.nan) if "c" in want else None
            jv = np.full(self.nnz_jac, np.nan) if "jv" in want else None
            hv = np.full(self.nnz_hess, np.nan) if "hv" in want else None
        self._lib.orc_eval(self.h, t0, t1, _ptr(x), _ptr(lam), float(sigma),
                      _ptr(f), _ptr(g), _ptr(c), _ptr(jv), _ptr(hv))
        return dict(f=None if f is None else float(f[0]), g=g, c=c, jv=jv, hv=hv)

    def kkt(self, x, lam, sigma, sigma_x, dvec, delta_w, t0=0, t1=None):
        """Rows of M for the variables of periods [t0, t1):
        (global row ids, row lengths, columns, values)."""
        t1 = self.T if t1 is None else t1
        x, lam, sx, dv = _f64(x), _f64(lam), _f64(sigma_x), _f64(dvec)
        res = self._lib.orc_kkt_new(self.h, t0, t1, _ptr(x), _ptr(lam), float(sigma), _ptr(sx), _ptr(dv),
                                    float(delta_w))
        try:
            sizes = np.zeros(2, np.int64)
            self._lib.orc_kkt_sizes(res, _ptr(sizes))
            nr, nnz = int(sizes[0]), int(sizes[1])
            assert nr == self._lib.orc_window_rows(self.h, t0, t1)
            rows = np.empty(nr, np.int64)
            rowlen = np.empty(nr, np.int64)
            cols = np.empty(nnz, np.int32)
            vals = np.empty(nnz, np.float64)
            self._lib.orc_kkt_copy(res, _ptr(rows), _ptr(rowlen), _ptr(cols), _ptr(vals))
        finally:
            self._lib.orc_kkt_free(res)
        return rows, rowlen, cols, vals

    def kkt_csr(self, x, lam, sigma, sigma_x, dvec, delta_w):
        rows, rowlen, cols, vals = self.kkt(x, lam, sigma, sigma_x, dvec, delta_w)
        assert np.array_equal(rows, np.arange(self.n))
        rowptr = np.zeros(self.n + 1, np.int64)
        np.cumsum(rowlen, out=rowptr[1:])
        return rowptr, cols, vals

    def vjp(self, x, y, t0=0, t1=None):
        t1 = self.T if t1 is None else t1
        x, y = _f64(x), _f64(y)
        gx = np.full(self.n, np.nan)
        D = self.inst.net.n_load
        gpd = np.full(self.T * D, np.nan)
        gqd = np.full(self.T * D, np.nan)
        self._lib.orc_vjp(self.h, t0, t1, _ptr(x), _ptr(y), _ptr(gx), _ptr(gpd), _ptr(gqd))
        return gx, gpd, gqd

    def hvp(self, x, lam, sigma, v, t0=0, t1=None):
        t1 = self.T if t1 is None else t1
        out = np.full(self.n, np.nan)
        self._lib.orc_hvp(self.h, t0, t1, _ptr(_f64(x)), _ptr(_f64(lam)), float(sigma), _ptr(_f64(v)), _ptr(out))
        return out

    def jvp(self, x, v, t0=0, t1=None, dpd=None, dqd=None):
        """J v (plus the load terms -sum dpd, -sum dqd on the balance rows)."""
        t1 = self.T if t1 is None else t1
        out = np.full(self.m, np.nan)
        dpd = None if dpd is None else _f64(dpd)
        dqd = None if dqd is None else _f64(dqd)
        self._lib.orc_jvp(self.h, t0, t1, _ptr(_f64(x)), _ptr(_f64(v)), _ptr(dpd), _ptr(dqd), _ptr(out))
        return out

    # -- pins -------------------------------------------------------------
    def cons_textbook(self, x):
        c = np.empty(self.m)
        self._lib.orc_cons_textbook(self.h, _ptr(_f64(x)), _ptr(c))
        return c

    def cons_cstep(self, x, dx, h=1e-30):
        dc = np.empty(self.m)
        self._lib.orc_cons_cstep(self.h, _ptr(_f64(x)), _ptr(_f64(dx)), float(h), _ptr(dc))
        return dc

    def gradlag(self, x, lam, sigma):
        out = np.empty(self.n)
        self._lib.orc_gradlag(self.h, _ptr(_f64(x)), _ptr(_f64(lam)), float(sigma), _ptr(out))
        return out

    def gradlag_cstep(self, x, lam, sigma, dx, h=1e-30):
        out = np.empty(self.n)
        self._lib.orc_gradlag_cstep(self.h, _ptr(_f64(x)), _ptr(_f64(lam)), float(sigma), _ptr(_f64(dx)),
                               float(h), _ptr(out))
        return out

    def obj_textbook(self, x):
        return float(self._lib.orc_obj_textbook(self.h, _ptr(_f64(x))))

    # -- COO -> CSC compression (Sec. III-A) ----------------------------------
    def csc(self, which, coo=None):
        """(colptr [n + 1], rowidx, vals or None) of J (which = 0) or the lower W
        (which = 1); duplicates summed in COO order."""
        nnz = int(self._lib.orc_csc_nnz(self.h, int(which)))
        colptr = np.empty(self.n + 1, np.int64)
        rowidx = np.empty(nnz, np.int32)
        vals = None if coo is None else np.empty(nnz)
        self._lib.orc_csc(self.h, int(which), None if coo is None else _ptr(_f64(coo)), _ptr(colptr), _ptr(rowidx),
                     None if vals is None else _ptr(vals))
        return colptr, rowidx, vals

    # -- interior-point algebra around M (Sec. III-B) ------------------------
    def ipm_prepare(self, x, s, zlx, zux, zls, zus, delta_w, delta_c, eps):
        """(Sigma_x, D, C, Sigma_s, recip) with recip = [rl_x, ru_x, rl_s, ru_s]."""
        sigx, dvec, cvec, sigs = np.empty(self.n), np.empty(self.m), np.empty(self.m), np.empty(self.m)
        recip = np.empty(2 * self.n + 2 * self.m)
        self._lib.orc_ipm_prepare(self.h, *[_ptr(_f64(a)) for a in (x, s, zlx, zux, zls, zus)], float(delta_w),
                             float(delta_c), float(eps), _ptr(sigx), _ptr(dvec), _ptr(cvec), _ptr(sigs),
                             _ptr(recip))
        return sigx, dvec, cvec, sigs, recip

    def ipm_rhs(self, x, s, y, zlx, zux, zls, zus, grad, c, mu, delta_w, delta_c, eps):
        rhs, w = np.empty(self.n), np.empty(self.m)
        self._lib.orc_ipm_rhs(self.h, *[_ptr(_f64(a)) for a in (x, s, y, zlx, zux, zls, zus, grad, c)], float(mu),
                         float(delta_w), float(delta_c), float(eps), _ptr(rhs), _ptr(w))
        return rhs, w

    def ipm_recover(self, x, s, y, zlx, zux, zls, zus, c, dx, mu, delta_w, delta_c, eps):
        outs = [np.empty(self.m), np.empty(self.m), np.empty(self.n), np.empty(self.n), np.empty(self.m),
                np.empty(self.m)]
        self._lib.orc_ipm_recover(self.h, *[_ptr(_f64(a)) for a in (x, s, y, zlx, zux, zls, zus, c, dx)], float(mu),
                             float(delta_w), float(delta_c), float(eps), *[_ptr(a) for a in outs])
        ds, dy, dzlx, dzux, dzls, dzus = outs
        return dict(ds=ds, dy=dy, dzlx=dzlx, dzux=dzux, dzls=dzls, dzus=dzus)

    def branch_terms(self):
        L = self.inst.net.n_branch
        out = np.empty(8 * L)
        self._lib.orc_branch_terms(self.h, _ptr(out))
        return out.reshape(8, L)


def sincos(x):
    lib = load()
    x = _f64(x)
    s, c = np.empty_like(x), np.empty_like(x)
    lib.orc_sincos(_ptr(x), x.size, _ptr(s), _ptr(c))
    return s, c
