"""The C boundary from C: include/mpopf.h compiles as strict C99, and a plain C
program (tests/c/sweep_host_example.c: a 3-bus network with a tapped and a
phase-shifting branch, T = 2) drives the library through mpopf_setup and the
host-buffer sweep with no CUDA calls of its own.  Without a GPU it fails with
the library's error; on a GPU its outputs equal the CPU reference bit for bit
(the objective within 1e-12)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import build, synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "sweep_host_example.c")
SHARD_SRC = os.path.join(HERE, "c", "shard_plan_example.c")
GCC = shutil.which("gcc")


def _compile(tmp_path, src=SRC):
    exe = str(tmp_path / os.path.splitext(os.path.basename(src))[0])
    build.build()
    subprocess.run([GCC, "-std=c99", "-Wall", "-Wextra", "-Werror", "-ffp-contract=off", "-I",
                    os.path.join(build.ROOT, "include"), src, "-o", exe, "-L", build.HERE, "-lmpopf",
                    "-Wl,-rpath," + build.HERE], check=True, capture_output=True, text=True)
    return exe


def _instance():
    net = synth.Network(
        n_bus=3, n_branch=3, n_gen=1, n_load=1, ref_bus=0,
        bus_gs=np.array([0.0, 0.02, 0.0]), bus_bs=np.array([0.0, 0.1, 0.0]),
        bus_vmin=np.full(3, 0.9), bus_vmax=np.full(3, 1.1),
        br_f=np.array([0, 1, 0], np.int32), br_t=np.array([1, 2, 2], np.int32),
        br_r=np.array([0.01, 0.02, 0.015]), br_x=np.array([0.1, 0.12, 0.08]), br_b=np.array([0.02, 0.01, 0.0]),
        br_tap=np.array([1.0, 1.03, 1.0]), br_shift=np.array([0.0, 0.0, 0.05]),
        br_smax=np.array([1.5, 1.2, 1.0]), br_angmin=np.full(3, -0.5), br_angmax=np.full(3, 0.5),
        gen_bus=np.array([0], np.int32), gen_c2=np.array([0.05]), gen_c1=np.array([20.0]), gen_c0=np.array([1.0]),
        gen_pmin=np.array([0.0]), gen_pmax=np.array([3.0]), gen_qmin=np.array([-1.5]), gen_qmax=np.array([1.5]),
        gen_ramp=np.array([0.6]), load_bus=np.array([2], np.int32))
    return synth.Instance(net=net, T=2, pd=np.array([[0.8], [0.9]]), qd=np.array([[0.2], [0.25]]))


@pytest.mark.skipif(GCC is None, reason="gcc not available")
def test_header_and_example_compile_as_c99(tmp_path):
    _compile(tmp_path)


@pytest.mark.skipif(GCC is None, reason="gcc not available")
def test_without_a_device_the_c_caller_gets_the_error(tmp_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([_compile(tmp_path)], capture_output=True, text=True)
    assert r.returncode == 1 and "no CUDA device" in r.stderr


@pytest.mark.gpu
@pytest.mark.skipif(GCC is None, reason="gcc not available")
def test_c_caller_outputs_equal_the_reference(tmp_path):
    r = subprocess.run([_compile(tmp_path)], capture_output=True, text=True, check=True)
    lines = r.stdout.split("\n")
    n, m, nj, nh, nk = (int(v) for v in lines[0].split())
    vals = np.array([float(v) for v in lines[1:] if v.strip()])
    inst = _instance()
    o = oracle.Oracle(inst)
    assert (n, m, nj, nh) == (o.n, o.m, o.nnz_jac, o.nnz_hess)
    i = np.arange(n)
    x = 1.0 + 0.01 * (((i * 7) % 11) - 5).astype(np.float64)
    sx = 0.5 + 0.25 * (i % 3).astype(np.float64)
    k = np.arange(m)
    lam = 0.1 * (((k * 5) % 9) - 4).astype(np.float64)
    dv = 1.0 + 0.5 * (k % 4).astype(np.float64)
    ref = o.eval(x, lam, 1.0)
    _, _, kv = o.kkt_csr(x, lam, 1.0, sx, dv, 1e-8)
    assert nk == kv.size
    f, rest = vals[0], vals[1:]
    assert abs(f - ref["f"]) <= 1e-12 * abs(ref["f"])
    parts = np.split(rest, np.cumsum([n, m, nj, nh]))
    for got, want in zip(parts, (ref["g"], ref["c"], ref["jv"], ref["hv"], kv)):
        assert np.array_equal(got, want)


@pytest.mark.skipif(GCC is None, reason="gcc not available")
def test_shard_plan_from_c_matches_the_binding(tmp_path):
    """tests/c/shard_plan_example.c asks for the layout of three period
    shards (no device needed); sizes, halo offsets and ranges equal the
    Python binding's, and a split with t0 = t1 is refused."""
    from paper_2405_14032_b300 import mpopf
    r = subprocess.run([_compile(tmp_path, SHARD_SRC)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lines = [list(map(int, ln.split())) for ln in r.stdout.split("\n") if ln.strip()]
    inst = _instance()
    net = inst.net
    pos = 0
    for t0, t1 in ((0, 2), (2, 3), (3, 5)):
        head = lines[pos]
        p = mpopf.shard_plan(net, 5, t0, t1)
        assert head[:5] == [t0, t1, p["local_periods"], p["own0"], p["own1"]]
        assert head[5:10] == [p["n"], p["m"], p["nnz_jac"], p["nnz_hess"], p["nnz_kkt"]]
        assert head[10:14] == [p["x_recv"][0], p["x_send"][0], p["d_recv"][0], p["d_send"][0]]
        n = head[14]
        got = {}
        for what, lo, gl, cnt in lines[pos + 1:pos + 1 + n]:
            got.setdefault(mpopf.RANGE_NAMES[what], []).append((lo, gl, cnt))
        assert got == {k: v for k, v in p["ranges"].items() if v}
        pos += 1 + n
    assert pos == len(lines)
