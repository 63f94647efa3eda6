"""GPU parity: every callback and the assembled KKT matrix, through the C-ABI,
against the CPU oracle on the same seeded inputs.

Index arrays must be identical; values must satisfy
|gpu - ref| <= max(1e-12 |ref|, 1e-14) elementwise (the tolerance the benchmark spec
states for FP64 values).  Both sides follow the same written rounding order,
so in practice the values agree bit for bit; the tests report that count.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def assert_close(name, got, ref, mask=None):
    got = np.asarray(got)
    ref = np.asarray(ref)
    if mask is not None:
        got, ref = got[mask], ref[mask]
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    err = np.abs(got - ref)
    ok = err <= np.maximum(1e-12 * np.abs(ref), 1e-14)
    if not ok.all():
        i = np.nonzero(~ok)[0][:5]
        raise AssertionError(f"{name}: {int((~ok).sum())} of {ok.size} outside tolerance; e.g. idx {i} "
                             f"gpu {got[i]} ref {ref[i]}")
    return int((got == ref).sum()), int(got.size)


class Case:
    def __init__(self, inst, seed, point=None):
        import paper_2405_14032_b300.mpopf as mp
        self.inst = inst
        self.pt = point if point is not None else synth.make_point(seed, inst)
        self.h = mp.Handle(inst)
        self.o = oracle.Oracle(inst)

    def run(self, outputs=63):
        pt = self.pt
        out = self.h.eval(outputs, _dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec),
                          pt.delta_w)
        torch.cuda.synchronize()
        return {k: (None if v is None else _np(v)) for k, v in out.items()}


def _edge_network():
    """Parallel branches, an isolated bus, several generators on one bus, a bus
    with no generator or load, tap/shift branches (asymmetric pi-model),
    nonzero cost constants."""
    f = [0, 1, 1, 2, 3, 0, 4, 2, 5]
    t = [1, 2, 2, 3, 4, 4, 5, 0, 6]
    L = len(f)
    rng = np.random.default_rng(9)
    tap = np.ones(L)
    shift = np.zeros(L)
    tap[3], shift[3] = 1.04, 0.05
    tap[6] = 0.97
    shift[8] = -0.08
    net = H.network(8, f, t, rng.uniform(0.005, 0.05, L), rng.uniform(0.02, 0.2, L), rng.uniform(0, 0.05, L),
                    gen_bus=[1, 1, 1, 4, 6, 0], load_bus=[2, 2, 3, 6, 7], ref=3, tap=tap, shift=shift,
                    gs=rng.uniform(0, 0.05, 8) * (rng.uniform(size=8) < 0.5),
                    bs=rng.uniform(0, 0.3, 8) * (rng.uniform(size=8) < 0.5),
                    c2=rng.uniform(0.01, 0.1, 6), c1=rng.uniform(10, 40, 6))
    net.gen_c0[:] = rng.uniform(-5.0, 5.0, 6)  # the synthetic networks have c0 = 0
    return net


def _cases():
    yield "cfg1", lambda: Case(synth.config_instance("cfg1"), 1)
    yield "ragged_T3", lambda: Case(synth.make_instance(41, 333, 530, 67, 200, 3), 41)
    yield "edge_T1", lambda: Case(H.instance(_edge_network(), 1), 42)
    yield "edge_T5", lambda: Case(H.instance(_edge_network(), 5), 43)
    yield "single_bus", lambda: Case(H.instance(H.network(1, [], [], [], [], [], gen_bus=[0, 0], load_bus=[0]), 3), 44)
    yield "no_gens_no_loads", lambda: Case(H.instance(H.network(
        5, [0, 1, 2, 3], [1, 2, 3, 4], [0.01] * 4, [0.1] * 4, [0.02] * 4, ref=2), 2, pd=np.zeros(0),
        qd=np.zeros(0)), 45)


def _wide_angle_case():
    inst = synth.make_instance(46, 60, 100, 12, 30, 3)
    pt = synth.make_point(46, inst)
    sl = H.var_slices(inst.net, inst.T)
    pt.x[sl["va"]] = synth.uniform(46, 999, inst.T * inst.net.n_bus, -4.0, 4.0)
    return Case(inst, 46, pt)


CASES = dict(_cases())
CASES["wide_angles"] = _wide_angle_case
# the reactive ramp rows K11 (optional variant)
CASES["qramp_T3"] = lambda: Case(synth.with_reactive_ramp(synth.make_instance(47, 200, 320, 40, 120, 3)), 47)
CASES["qramp_edge_T5"] = lambda: Case(synth.with_reactive_ramp(H.instance(_edge_network(), 5)), 48)
CASES["qramp_T1"] = lambda: Case(synth.with_reactive_ramp(H.instance(_edge_network(), 1)), 49)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    return request.param, CASES[request.param]()


def test_patterns_and_bounds(case):
    name, cs = case
    o, h = cs.o, cs.h
    assert (h.n, h.m, h.nnz_jac, h.nnz_hess) == (o.n, o.m, o.nnz_jac, o.nnz_hess)
    pat = {k: _np(v) for k, v in h.pattern().items()}
    jr, jc = o.jac_pattern()
    assert np.array_equal(pat["jac_row"], jr) and np.array_equal(pat["jac_col"], jc)
    hr, hc = o.hess_pattern()
    assert np.array_equal(pat["hess_row"], hr) and np.array_equal(pat["hess_col"], hc)
    pt = cs.pt
    rowptr, cols, _ = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    assert h.nnz_kkt == cols.size
    assert np.array_equal(pat["kkt_rowptr"], rowptr) and np.array_equal(pat["kkt_col"], cols)
    xl, xu, gl, gu = o.bounds()
    for k, r in (("xl", xl), ("xu", xu), ("gl", gl), ("gu", gu)):
        assert np.array_equal(pat[k], r), k


def test_values_match_oracle(case):
    name, cs = case
    pt, o = cs.pt, cs.o
    out = cs.run()
    ref = o.eval(pt.x, pt.lam, pt.sigma)
    _, _, kv = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    stats = {}
    for k, r in (("grad", ref["g"]), ("c", ref["c"]), ("jv", ref["jv"]), ("hv", ref["hv"]), ("kv", kv)):
        stats[k] = assert_close(f"{name}:{k}", out[k], r)
    assert abs(out["f"][0] - ref["f"]) <= max(1e-12 * abs(ref["f"]), 1e-14), (out["f"][0], ref["f"])
    print(name, {k: f"{e}/{n} bitwise" for k, (e, n) in stats.items()})


def test_single_callbacks_equal_sweep(case):
    """Each callback alone gives the sweep's values bit for bit."""
    name, cs = case
    full = cs.run()
    for bit, key in ((1, "f"), (2, "grad"), (4, "c"), (8, "jv"), (16, "hv"), (32, "kv")):
        one = cs.run(bit)
        assert np.array_equal(one[key], full[key]), (name, key)


def test_deterministic(case):
    name, cs = case
    a = cs.run()
    b = cs.run()
    for k in a:
        assert np.array_equal(a[k], b[k]), (name, k)


def test_cfg2_full():
    """2,000 buses x 24 periods: every entry of every output."""
    cs = Case(synth.config_instance("cfg2"), 2)
    pt, o = cs.pt, cs.o
    out = cs.run()
    ref = o.eval(pt.x, pt.lam, pt.sigma)
    rowptr, cols, kv = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    pat = {k: _np(v) for k, v in cs.h.pattern().items()}
    jr, jc = o.jac_pattern()
    assert np.array_equal(pat["jac_row"], jr) and np.array_equal(pat["jac_col"], jc)
    assert np.array_equal(pat["kkt_rowptr"], rowptr) and np.array_equal(pat["kkt_col"], cols)
    for k, r in (("grad", ref["g"]), ("c", ref["c"]), ("jv", ref["jv"]), ("hv", ref["hv"]), ("kv", kv)):
        e, n = assert_close(f"cfg2:{k}", out[k], r)
        print("cfg2", k, f"{e}/{n} bitwise")
    assert abs(out["f"][0] - ref["f"]) <= 1e-12 * abs(ref["f"])


HOST_CASES = {
    "cfg1": lambda: Case(synth.config_instance("cfg1"), 1),               # T = 4: four one-period windows
    "ragged_T13": lambda: Case(synth.make_instance(52, 150, 240, 30, 90, 13), 52),  # windows 1, 2, 2, 2, 2, 2, 1, 1
    "edge_T1": lambda: Case(H.instance(_edge_network(), 1), 42),          # one window, no ramp rows
    "no_gens_no_loads": CASES["no_gens_no_loads"],
    "qramp_T3": CASES["qramp_T3"],
    "cfg2": lambda: Case(synth.config_instance("cfg2"), 2),               # T = 24: windows 1, 3, 4, 4, 3, 3, 3, 3
}


@pytest.mark.parametrize("name", sorted(HOST_CASES))
def test_sweep_host_matches_device(name):
    """The host-buffer entry point (inputs and outputs copied in period
    windows, overlapped with the kernels) equals the device sweep bit for bit,
    twice in a row (the pipeline's streams and events are reused)."""
    cs = HOST_CASES[name]()
    pt = cs.pt
    dev = cs.run()
    for _ in range(2):
        out = dict(f=np.full(1, np.nan), grad=np.full(cs.h.n, np.nan), c=np.full(cs.h.m, np.nan),
                   jv=np.full(cs.h.nnz_jac, np.nan), hv=np.full(cs.h.nnz_hess, np.nan),
                   kv=np.full(cs.h.nnz_kkt, np.nan))
        cs.h.sweep_host(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w, out)
        for k in out:
            assert np.array_equal(out[k], dev[k]), (name, k)


SCHEDULES = [(1, 0), (2, 1), (3, 2), (4, 3), (5, 0), (0, 0), (0, 2), (0, 6), (0, 8), (0, 12), (0, 16), (0, 20),
             (0, 24), (2, 16)]


def test_chunked_schedules_equal_plain(case):
    """Every launch schedule (period chunks, the bus kernel of each chunk on a
    second stream, with and without its priority raised, the generator work
    forked first or last; the bus kernel as a programmatic dependent launch;
    the bus work split in two kernels side by side; the bus-end products of
    M in a launch of their own before the branch kernel, with and without the
    programmatic dependency) gives the plain sweep's
    outputs bit for bit, for
    every output and for the callbacks alone; the plain sweep matches the
    oracle (test_values_match_oracle), so these do too."""
    name, cs = case
    default = cs.h.sweep_schedule()
    # one launch per kernel, the bus kernel a programmatic dependent launch
    # (these networks' branch launches fit one wave: no bus-term launch)
    assert default == (0, 4)
    full = cs.run()
    try:
        for P, flags in SCHEDULES:
            cs.h.set_sweep_schedule(P, flags)
            assert cs.h.sweep_schedule() == (P, flags)
            got = cs.run()
            for k in full:
                assert np.array_equal(got[k], full[k]), (name, P, flags, k)
            for bit, key in ((4, "c"), (32, "kv")):
                assert np.array_equal(cs.run(bit)[key], full[key]), (name, P, flags, key)
    finally:
        cs.h.set_sweep_schedule(*default)


def test_chunked_schedule_cfg2_and_launch_count():
    """2,000 buses x 24 periods in chunks of 5 (the last one shorter): the
    outputs equal the oracle's; the launch count reports two launches per
    chunk plus the generator kernels."""
    import paper_2405_14032_b300.mpopf as mp
    cs = Case(synth.config_instance("cfg2"), 2)
    plain = cs.h.launch_count()
    assert plain == 4  # branch, bus, generator, objective
    cs.h.set_sweep_schedule(0, mp.Handle.SCHED_PDL | mp.Handle.SCHED_BUS_TERMS)
    assert cs.h.launch_count() == plain + 1  # and the bus-end products
    cs.h.set_sweep_schedule(0, mp.Handle.SCHED_SPLIT_BUS)
    assert cs.h.launch_count() == plain + 1  # the bus work as two kernels
    cs.h.set_sweep_schedule(5, mp.Handle.SCHED_BUS_PRIORITY)
    assert cs.h.launch_count() == plain - 2 + 2 * 5
    pt, o = cs.pt, cs.o
    out = cs.run()
    ref = o.eval(pt.x, pt.lam, pt.sigma)
    _, _, kv = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    for k, r in (("grad", ref["g"]), ("c", ref["c"]), ("jv", ref["jv"]), ("hv", ref["hv"]), ("kv", kv)):
        assert_close(f"cfg2 chunked:{k}", out[k], r)
    assert abs(out["f"][0] - ref["f"]) <= 1e-12 * abs(ref["f"])
    with pytest.raises(mp.MpopfError, match="bad argument"):
        cs.h.set_sweep_schedule(-1, 0)
    with pytest.raises(mp.MpopfError, match="bad argument"):
        cs.h.set_sweep_schedule(4, 1 << 10)  # a bit no schedule defines
    cs.h.close()
