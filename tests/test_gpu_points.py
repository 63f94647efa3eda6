"""Sweeps of one network at several points in one launch per kernel
(mpopf_sweep_points): every point's outputs equal the single sweep's at that
point bit for bit, the first point's equal the oracle's within the parity
tolerance, on the parity networks (ragged sizes, parallel branches, an isolated
bus, no generators, the reactive ramp rows, T = 1) and on the 2,000-bus x 24
network.  Each point has its own x, lam, sigma_x and dvec, so a wrong point
offset in any input or output shows."""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests.test_gpu_parity import CASES, Case, assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _points(inst, seed, k):
    return [synth.make_point(seed, inst, stream_offset=100 * j) for j in range(k)]


def _stack(pts, key):
    return torch.as_tensor(np.stack([getattr(p, key) for p in pts]), dtype=torch.float64, device="cuda").contiguous()


def _np(t):
    return t.detach().cpu().numpy()


def _check(h, pts, out, o=None, name=""):
    sigma, dw = pts[0].sigma, pts[0].delta_w
    got = {k: _np(v) for k, v in out.items()}
    for j, p in enumerate(pts):
        dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
        one = h.sweep(dev(p.x), dev(p.lam), sigma, dev(p.sigma_x), dev(p.dvec), dw)
        torch.cuda.synchronize()
        for k, v in one.items():
            assert np.array_equal(got[k][j], _np(v).reshape(got[k][j].shape)), (name, j, k)
    if o is not None:
        p = pts[0]
        ref = o.eval(p.x, p.lam, sigma)
        _, _, kv = o.kkt_csr(p.x, p.lam, sigma, p.sigma_x, p.dvec, dw)
        for k, r in (("grad", ref["g"]), ("c", ref["c"]), ("jv", ref["jv"]), ("hv", ref["hv"]), ("kv", kv)):
            assert_close(f"{name}:{k}", got[k][0], r)
        assert abs(got["f"][0] - ref["f"]) <= max(1e-12 * abs(ref["f"]), 1e-14)


def _sweep_points(h, pts, stream=None):
    return h.sweep_points(_stack(pts, "x"), _stack(pts, "lam"), pts[0].sigma, _stack(pts, "sigma_x"),
                          _stack(pts, "dvec"), pts[0].delta_w, stream=stream)


@pytest.mark.parametrize("name", sorted(CASES))
def test_points_equal_single_sweeps(name):
    cs = CASES[name]()
    pts = _points(cs.inst, 61, 3)
    out = _sweep_points(cs.h, pts)
    torch.cuda.synchronize()
    _check(cs.h, pts, out, cs.o, name)
    cs.h.close()


def test_points_cfg2_scratch_growth_and_schedules():
    """2,000 buses x 24: 2, then 5 (the scratch grows), then 3 points (it is
    reused); with the bus kernel launched programmatically (default) and
    plainly; on a side stream."""
    cs = Case(synth.config_instance("cfg2"), 2)
    h = cs.h
    pts = _points(cs.inst, 62, 5)
    out = _sweep_points(h, pts[:2])
    torch.cuda.synchronize()
    _check(h, pts[:2], out, cs.o, "cfg2 k=2")
    out = _sweep_points(h, pts)
    torch.cuda.synchronize()
    _check(h, pts, out, None, "cfg2 k=5")
    default = h.sweep_schedule()
    try:
        h.set_sweep_schedule(0, 0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            out = _sweep_points(h, pts[2:], stream=s)
        s.synchronize()
        _check(h, pts[2:], out, None, "cfg2 k=3 plain launches")
    finally:
        h.set_sweep_schedule(*default)
    h.close()


def test_points_single_point_and_errors():
    import paper_2405_14032_b300.mpopf as mp
    inst = synth.config_instance("cfg1")
    h = mp.Handle(inst)
    pts = _points(inst, 63, 1)
    out = _sweep_points(h, pts)
    torch.cuda.synchronize()
    _check(h, pts, out, oracle.Oracle(inst), "cfg1 k=1")
    x = _stack(pts, "x")
    with pytest.raises(ValueError):  # shapes are checked by the binding
        h.sweep_points(x[:, :-1].contiguous(), _stack(pts, "lam"), 1.0, _stack(pts, "sigma_x"),
                       _stack(pts, "dvec"), 0.0)
    o = h.new_point_outputs(1)
    lib = mp.lib()
    p = lambda t: t.data_ptr()
    args = [p(x), p(_stack(pts, "lam")), 1.0, p(_stack(pts, "sigma_x")), p(_stack(pts, "dvec")), 0.0,
            p(o["f"]), p(o["grad"]), p(o["c"]), p(o["jv"]), p(o["hv"]), p(o["kv"]), None]
    assert lib.mpopf_sweep_points(h.h, 0, *args) == -1  # MPOPF_ERR_ARG: no points
    assert lib.mpopf_sweep_points(h.h, 65536, *args) == -1
    bad = list(args)
    bad[7] = None  # grad
    assert lib.mpopf_sweep_points(h.h, 1, *bad) == -1
    h.close()
    T = inst.T
    hs = mp.Handle(inst, shard=(0, T // 2))
    assert lib.mpopf_sweep_points(hs.h, 1, *args) == -1  # not on a period shard
    hs.close()


NEED_POINTS_BYTES = 100 * 2**30


def test_points_offsets_beyond_2_31():
    """The 10k-bus network at T = 168 (nnz of M 96.1M) at 24 points in one
    call: the later points' J, W and M start past 2^31 entries of their
    arrays (point 23's M at 2.2e9), so the kernels' point offsets are 64-bit
    wherever they must be.  The first and last points against single sweeps
    at the same points, on the device.  About 75 GB of device memory: skipped
    when less than 100 GB is free."""
    free, _ = torch.cuda.mem_get_info()
    if free < NEED_POINTS_BYTES:
        pytest.skip(f"needs {NEED_POINTS_BYTES / 2**30:.0f} GB free on the device, {free / 2**30:.0f} GB free")
    from paper_2405_14032_b300 import mpopf
    inst = synth.config_instance("cfg3")
    pt = synth.make_point(3, inst)
    h = mpopf.Handle(inst)
    k = 24
    assert (k - 1) * h.nnz_kkt > 2**31
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(24)
    X = dev(pt.x).unsqueeze(0) + 1e-3 * torch.randn(k, h.n, generator=gen, device="cuda", dtype=torch.float64)
    rep = lambda a: dev(a).unsqueeze(0).expand(k, -1).contiguous()
    LAM, SX, DV = rep(pt.lam), rep(pt.sigma_x), rep(pt.dvec)
    out = h.sweep_points(X, LAM, pt.sigma, SX, DV, pt.delta_w)
    torch.cuda.synchronize()
    del LAM, SX, DV
    for j in (0, k - 1):
        one = h.sweep(X[j], dev(pt.lam), pt.sigma, dev(pt.sigma_x), dev(pt.dvec), pt.delta_w)
        torch.cuda.synchronize()
        for key, v in one.items():
            assert torch.equal(out[key][j], v.reshape(out[key][j].shape)), (j, key)
        del one
    del out, X
    h.close()
    torch.cuda.empty_cache()
