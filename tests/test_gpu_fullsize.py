"""Parity at the full benchmark size: the 10k-bus network with 168 periods
(seed 3), evaluated through mpopf_sweep exactly as bench.py times it.  The
oracle evaluates sampled periods (the first two, one in the middle, the last
two: ramp rows at both ends of the horizon) on their own; every output entry
of those periods -- c, grad f, J, W and the rows of M -- must equal the GPU's
bit for bit.  The objective (a sum over the whole horizon, a tree on the GPU)
is compared with the textbook sum within 1e-12 relative; the derivative
products are compared on the same sampled periods; the host-buffer entry point
(pipelined copies) must return the device sweep's outputs bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, L, G, D, T, SEED = 10000, 16000, 2000, 6000, 168, 3
PERIODS = (0, 1, 84, 166, 167)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def full():
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(SEED, N, L, G, D, T)
    pt = synth.make_point(SEED, inst)
    h = mpopf.Handle(inst)
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    d = dict(x=dev(pt.x), lam=dev(pt.lam), sx=dev(pt.sigma_x), dv=dev(pt.dvec))
    out = h.sweep(d["x"], d["lam"], pt.sigma, d["sx"], d["dv"], pt.delta_w)
    torch.cuda.synchronize()
    host = {k: _np(v) for k, v in out.items()}
    pat = {k: _np(v) for k, v in h.pattern().items()}
    yield inst, pt, h, d, host, pat, oracle.Oracle(inst)
    h.close()


def test_default_schedule_has_the_bus_term_launch(full):
    """The benchmark-size handle starts with the bus-end products in a launch
    of their own (its branch launch spans far more than two waves), so the
    parity tests of this file check that schedule; a sweep with it turned off
    gives the same outputs bit for bit."""
    from paper_2405_14032_b300 import mpopf
    inst, pt, h, d, host, pat, o = full
    assert h.sweep_schedule() == (0, mpopf.Handle.SCHED_PDL | mpopf.Handle.SCHED_BUS_TERMS)
    h.set_sweep_schedule(0, mpopf.Handle.SCHED_PDL)
    try:
        out = h.sweep(d["x"], d["lam"], pt.sigma, d["sx"], d["dv"], pt.delta_w)
        torch.cuda.synchronize()
        for k, v in out.items():
            assert np.array_equal(_np(v), host[k]), k
    finally:
        h.set_sweep_schedule(0, mpopf.Handle.SCHED_PDL | mpopf.Handle.SCHED_BUS_TERMS)


@pytest.mark.parametrize("t", PERIODS)
def test_sampled_period_bitwise(full, t):
    inst, pt, h, d, host, pat, o = full
    ref = o.eval(pt.x, pt.lam, pt.sigma, t0=t, t1=t + 1)
    for key, gkey in (("c", "c"), ("g", "grad"), ("jv", "jv"), ("hv", "hv")):
        mask = ~np.isnan(ref[key])
        assert mask.sum() > 0, (t, key)
        assert np.array_equal(host[gkey][mask], ref[key][mask]), (t, key)
    rows, rowlen, cols, vals = o.kkt(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w, t0=t, t1=t + 1)
    rp = pat["kkt_rowptr"]
    assert np.array_equal(rp[rows + 1] - rp[rows], rowlen), t
    pos = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    assert np.array_equal(pat["kkt_col"][pos], cols), t
    assert np.array_equal(host["kv"][pos], vals), t


def test_objective_full_horizon(full):
    inst, pt, h, d, host, pat, o = full
    ref = o.obj_textbook(pt.x)
    assert abs(host["f"][0] - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("t", (0, 167))
def test_products_sampled_period(full, t):
    inst, pt, h, d, host, pat, o = full
    rng = np.random.default_rng(31 + t)
    y, v = rng.standard_normal(o.m), rng.standard_normal(o.n)
    gx = _np(h.vjp(d["x"], torch.as_tensor(y, device="cuda"), loads=False)[0])
    rgx = o.vjp(pt.x, y, t0=t, t1=t + 1)[0]
    mask = ~np.isnan(rgx)
    assert mask.sum() > 0 and np.array_equal(gx[mask], rgx[mask])
    jvv = _np(h.jvp(d["x"], torch.as_tensor(v, device="cuda")))
    rjv = o.jvp(pt.x, v, t0=t, t1=t + 1)
    mask = ~np.isnan(rjv)
    assert mask.sum() > 0 and np.array_equal(jvv[mask], rjv[mask])


def test_host_buffer_sweep_full_size(full):
    inst, pt, h, d, host, pat, o = full
    out = dict(f=np.empty(1), grad=np.empty(h.n), c=np.empty(h.m), jv=np.empty(h.nnz_jac),
               hv=np.empty(h.nnz_hess), kv=np.empty(h.nnz_kkt))
    h.sweep_host(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w, out)
    for k in out:
        assert np.array_equal(out[k], host[k]), k
