"""The C-ABI library loads, exports every symbol include/mpopf.h declares, and
rejects bad arguments on the host before any device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2405_14032_b300 import mpopf, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mpopf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mpopf_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = mpopf.lib()
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(mpopf.exported_symbols())


def _prototypes():
    """{name: [parameter types]} from the header's declarations."""
    txt = open(os.path.join(ROOT, "include", "mpopf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(mpopf_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", txt):
        params = " ".join(m.group(2).split())
        if params in ("", "void"):
            out[m.group(1)] = []
            continue
        kinds = []
        for prm in params.split(","):
            prm = prm.strip()
            if "*" in prm:
                kinds.append("ptr")
            elif re.match(r"(const\s+)?double\b", prm):
                kinds.append("double")
            else:
                kinds.append("int")
        out[m.group(1)] = kinds
    return out


def test_binding_signatures_match_header():
    """Every ctypes prototype has the header's parameter count and kinds
    (pointer / double / integer), so a marshalling slip fails here, on the host."""
    lib = mpopf.lib()
    protos = _prototypes()
    assert set(protos) == set(_declared())

    def kind(t):
        if t is ctypes.c_double:
            return "double"
        if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and not isinstance(t._type_, str):
            return "ptr"
        return "int"

    for name, want in protos.items():
        got = [kind(t) for t in getattr(lib, name).argtypes]
        assert got == want, (name, got, want)


def _setup_rc(net, T=2, pd=None, qd=None):
    lib = mpopf.lib()
    h = ctypes.c_void_p()
    pat = mpopf._Pattern()
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data if a.size else None

    c = mpopf._Network(
        n_bus=net.n_bus, n_branch=net.n_branch, n_gen=net.n_gen, n_load=net.n_load, ref_bus=net.ref_bus,
        **{k: arr(getattr(net, k), np.int32 if k in ("br_f", "br_t", "gen_bus", "load_bus") else np.float64)
           for k, _ in mpopf._Network._fields_[5:] if getattr(net, k) is not None})
    pd = np.zeros((T, net.n_load)) if pd is None else pd
    qd = np.zeros((T, net.n_load)) if qd is None else qd
    rc = lib.mpopf_setup(ctypes.byref(c), T, arr(pd, np.float64), arr(qd, np.float64), ctypes.byref(h),
                         ctypes.byref(pat))
    if rc == 0:
        lib.mpopf_destroy(h)
    return rc, lib.mpopf_last_error().decode()


def test_rejects_bad_arguments_on_host():
    net = synth.make_network(3, 10, 14, 2, 3)
    rc, msg = _setup_rc(net, T=0)
    assert rc == -1 and "n_periods" in msg
    bad = synth.make_network(3, 10, 14, 2, 3)
    bad.br_t = bad.br_f.copy()
    rc, msg = _setup_rc(bad)
    assert rc == -1 and "self-loop" in msg
    bad = synth.make_network(3, 10, 14, 2, 3)
    bad.gen_bus = np.array([0, 11], np.int32)
    rc, msg = _setup_rc(bad)
    assert rc == -1 and "generator bus" in msg
    bad = synth.make_network(3, 10, 14, 2, 3)
    bad.ref_bus = 10
    rc, msg = _setup_rc(bad)
    assert rc == -1
    bad = synth.make_network(3, 10, 14, 2, 3)
    bad.br_tap = np.zeros(14)
    rc, msg = _setup_rc(bad)
    assert rc == -1 and "tap" in msg
    bad = synth.make_network(3, 10, 14, 2, 3)
    bad.gen_qramp = np.array([0.1, -0.2])
    rc, msg = _setup_rc(bad)
    assert rc == -1 and "reactive ramp" in msg


def test_rejects_oversized_problem_before_allocation():
    """n = T (2N + 2G + 4L) >= 2^31 is refused with MPOPF_ERR_SIZE before any
    array is read (the arrays here are NULL)."""
    lib = mpopf.lib()
    c = mpopf._Network(n_bus=600_000_000, n_branch=0, n_gen=0, n_load=0, ref_bus=0)
    h = ctypes.c_void_p()
    rc = lib.mpopf_setup(ctypes.byref(c), 2, None, None, ctypes.byref(h), None)
    assert rc == -2
    assert "2^31" in lib.mpopf_last_error().decode()


def test_null_handle_calls_fail_cleanly():
    lib = mpopf.lib()
    assert lib.mpopf_eval(None, 63, None, None, 1.0, None, None, 0.0, None, None, None, None, None, None,
                          None) == -1
    assert lib.mpopf_launch_count(None, 63) == -1
    lib.mpopf_destroy(None)


def test_no_device_is_an_error_not_a_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, msg = _setup_rc(synth.make_network(3, 10, 14, 2, 3))
    assert rc == -3 and "CUDA" in msg


def test_last_error_is_per_thread():
    """Threads that fail concurrently for different reasons each read their own
    message (the error text is thread-local)."""
    import threading
    lib = mpopf.lib()
    results = {}
    barrier = threading.Barrier(8)

    def worker(k):
        net = synth.make_network(3, 10, 14, 2, 3)
        if k % 2:
            net.br_t = net.br_f.copy()  # self-loops
            want = "self-loop"
        else:
            net.gen_bus = np.array([0, 99], np.int32)  # generator bus out of range
            want = "generator bus"
        barrier.wait()
        for _ in range(50):
            rc, msg = _setup_rc(net)
            if rc != -1 or want not in msg:
                results[k] = (rc, msg)
                return
            if want not in lib.mpopf_last_error().decode():
                results[k] = ("reread", lib.mpopf_last_error().decode())
                return
        results[k] = "ok"

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert all(v == "ok" for v in results.values()), results
