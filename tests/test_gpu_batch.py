"""Batched sweeps: many uneven instances in one persistent launch (CUDA graph)
give, for every instance, the same outputs bit for bit as mpopf_sweep on that
instance alone, whatever the schedule; the autotuner keeps that property.  The
batched outputs are also compared with the CPU oracle directly: every output
of every small instance, and sampled periods of the smallest, the largest, a
T = 12 and a T = 96 instance of the 64-instance workload, with the parity
tolerance |gpu - ref| <= max(1e-12 |ref|, 1e-14)."""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("f", "grad", "c", "jv", "hv", "kv")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _setup(shapes, seeds=None, keep=None):
    """Handles, batch I/O and per-instance reference sweeps; with `keep` (a
    list) the (instance, point) pairs are appended to it."""
    from paper_2405_14032_b300 import mpopf
    hs, ios, refs = [], [], []
    for k, shape in enumerate(shapes):
        N, L, G, D, T = shape[:5]
        seed = 100 + k if seeds is None else seeds[k]
        inst = synth.make_instance(seed, N, L, G, D, T)
        if len(shape) > 5 and shape[5] == "qramp":
            inst = synth.with_reactive_ramp(inst)
        pt = synth.make_point(seed, inst)
        if keep is not None:
            keep.append((inst, pt))
        h = mpopf.Handle(inst)
        io = dict(x=_dev(pt.x), lam=_dev(pt.lam), sigma=pt.sigma, sigma_x=_dev(pt.sigma_x), dvec=_dev(pt.dvec),
                  delta_w=pt.delta_w)
        ref = h.sweep(io["x"], io["lam"], pt.sigma, io["sigma_x"], io["dvec"], pt.delta_w)
        out = {k2: torch.full_like(v, float("nan")) for k2, v in ref.items()}
        io.update(out)
        hs.append(h)
        ios.append(io)
        refs.append(ref)
    torch.cuda.synchronize()
    return hs, ios, refs


def _within(name, got, ref):
    err = np.abs(got - ref)
    ok = err <= np.maximum(1e-12 * np.abs(ref), 1e-14)
    assert ok.all(), (name, int((~ok).sum()), np.nonzero(~ok)[0][:5])


def _check_oracle(inst, pt, h, io, periods=None):
    """The batched outputs of one instance against the oracle: every output
    (periods None) or every entry of the sampled periods."""
    o = oracle.Oracle(inst)
    got = {k: io[k].cpu().numpy() for k in KEYS}
    pat = {k: v.cpu().numpy() for k, v in h.pattern().items()}
    if periods is None:
        ref = o.eval(pt.x, pt.lam, pt.sigma)
        for key, gkey in (("c", "c"), ("g", "grad"), ("jv", "jv"), ("hv", "hv")):
            _within(gkey, got[gkey], ref[key])
        rp, cols, vals = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
        assert np.array_equal(pat["kkt_rowptr"], rp) and np.array_equal(pat["kkt_col"], cols)
        _within("kv", got["kv"], vals)
    else:
        for t in periods:
            ref = o.eval(pt.x, pt.lam, pt.sigma, t0=t, t1=t + 1)
            for key, gkey in (("c", "c"), ("g", "grad"), ("jv", "jv"), ("hv", "hv")):
                mask = ~np.isnan(ref[key])
                assert mask.sum() > 0, (t, key)
                _within((t, gkey), got[gkey][mask], ref[key][mask])
            rows, rowlen, cols, vals = o.kkt(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w, t0=t, t1=t + 1)
            rp = pat["kkt_rowptr"]
            assert np.array_equal(rp[rows + 1] - rp[rows], rowlen), t
            pos = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
            assert np.array_equal(pat["kkt_col"][pos], cols), t
            _within((t, "kv"), got["kv"][pos], vals)
    f_ref = o.obj_textbook(pt.x)
    assert abs(float(got["f"][0]) - f_ref) <= 1e-12 * abs(f_ref) + 1e-14


def _check_all(b, ios, refs):
    for io in ios:
        for k in KEYS:
            io[k].fill_(float("nan"))
    b.sweep()
    b.status()
    torch.cuda.synchronize()
    for i, (io, ref) in enumerate(zip(ios, refs)):
        for k in KEYS:
            assert torch.equal(io[k], ref[k]), (i, k)


# Shapes cover both paths of the staged J and W ranges of the branch tiles
# (one bulk copy when the destination is 16-byte aligned, warp stores when not):
# T odd puts the K1 and K3 rows of J on an 8-byte boundary, and the K2 and K4
# rows too unless L is odd; T G odd does so for the W blocks.  (57, 91, 11, 30,
# 3) alternates the two paths within a warp, (161, 257, 33, 97, 2) takes only
# bulk copies.
SMALL = [(40, 64, 8, 20, 3), (73, 117, 15, 44, 2), (130, 208, 26, 78, 5), (31, 50, 6, 19, 1), (250, 400, 50, 150, 4),
         (12, 20, 0, 5, 3), (600, 960, 120, 360, 7), (90, 140, 20, 50, 4, "qramp"), (57, 91, 11, 30, 3),
         (161, 257, 33, 97, 2)]


def test_batch_equals_individual_sweeps_every_schedule():
    from paper_2405_14032_b300 import mpopf
    kept = []
    hs, ios, refs = _setup(SMALL, keep=kept)
    b = mpopf.Batch(hs)
    b.set_io(ios)
    _check_all(b, ios, refs)
    for (inst, pt), h, io in zip(kept, hs, ios):  # the batched outputs against the oracle, in full
        _check_oracle(inst, pt, h, io)
    for sched in [(0, 1, 0, 0), (1, 1, 1, 1), (0, 2, 2, 2), (1, 4, 0, 3), (0, 4, 1, 0), (1, 2, 3, 1), (0, 1, 0, 2),
                  (0, 1, 0, 0, 2), (1, 2, 1, 0, 2), (0, 4, 3, 0, 2), (0, 1, 0, 0, 0), (1, 1, 3, 0, 0),
                  (0, 1, 64, 0, 0), (1, 1, 1, 0, 0)]:
        b.set_schedule(*sched)
        _check_all(b, ios, refs)
        _check_all(b, ios, refs)  # replay of the same graph
    best = b.tune(reps=2)
    assert best > 0
    _check_all(b, ios, refs)
    for bad in [(0, 1, 65, 0, 0), (0, 1, 0, 0, 3), (2, 1, 0, 0, 1), (0, 0, 0, 0, 1), (0, 1, -1, 0, 1),
                (0, 1, 0, 0, -1)]:
        with pytest.raises(mpopf.MpopfError, match="bad argument"):
            b.set_schedule(*bad)
    _check_all(b, ios, refs)
    b.close()


def test_batch_64_uneven_instances():
    """The batched workload: 64 instances, buses log-uniform in [500, 5000],
    L = 1.6 N, G = 0.2 N, D = 0.6 N, T in {12, 24, 48, 96}."""
    from paper_2405_14032_b300 import mpopf
    spec = synth.batch_shapes(64)
    shapes = [(s["n_bus"], s["n_branch"], s["n_gen"], s["n_load"], s["T"]) for s in spec]
    kept = []
    hs, ios, refs = _setup(shapes, seeds=[s["seed"] for s in spec], keep=kept)
    b = mpopf.Batch(hs)
    b.set_io(ios)
    _check_all(b, ios, refs)
    b.tune(reps=2)
    _check_all(b, ios, refs)
    # the tuned batch's outputs against the oracle: the smallest and the
    # largest instance, and one with T = 12 and one with T = 96 (sampled
    # periods: both ends of the horizon, with their ramp rows, and the middle)
    sizes = [s["n_bus"] * s["T"] for s in spec]
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    for T in (12, 96):
        pick.append(next(k for k, s in enumerate(spec) if s["T"] == T and k not in pick))
    for k in pick:
        T = spec[k]["T"]
        inst, pt = kept[k]
        _check_oracle(inst, pt, hs[k], ios[k], periods=sorted({0, 1, T // 2, T - 2, T - 1}))
    b.close()


def test_dependency_wait_timeout_is_reported_not_hung():
    """A bus tile whose dependency target can never be met (test hook) waits out
    its bounded limit, the launch finishes, mpopf_batch_status reports the
    error, the outputs are still complete (the tile is computed after the
    wait), and once the target is restored the next launch is clean."""
    import time

    from paper_2405_14032_b300 import mpopf
    hs, ios, refs = _setup(SMALL[:3])
    b = mpopf.Batch(hs)
    b.set_io(ios)
    _check_all(b, ios, refs)
    b.test_stall(True)
    for io in ios:
        for k in KEYS:
            io[k].fill_(float("nan"))
    t0 = time.perf_counter()
    b.sweep()
    with pytest.raises(mpopf.MpopfError, match="dependency wait"):
        b.status()
    waited = time.perf_counter() - t0
    assert 0.05 < waited < 60.0
    for io, ref in zip(ios, refs):
        for k in KEYS:
            assert torch.equal(io[k], ref[k]), k
    b.test_stall(False)
    _check_all(b, ios, refs)
    # with two launches, or plain sweeps, nothing waits: the hook has no wait
    # to hold back
    for sched, launches in (((0, 1, 0, 0, 2), 2), ((1, 1, 4, 0, 0), 0)):
        b.set_schedule(*sched)
        assert b.schedule()["launches"] == launches
        with pytest.raises(mpopf.MpopfError, match="no bus tile waits"):
            b.test_stall(True)
        _check_all(b, ios, refs)
    b.close()


def test_batch_refuses_a_repeated_handle():
    """Each instance's scratch belongs to its handle, so a batch holding the
    same handle twice is refused at creation."""
    from paper_2405_14032_b300 import mpopf
    hs, ios, refs = _setup(SMALL[:2])
    with pytest.raises(mpopf.MpopfError, match="appears twice"):
        mpopf.Batch([hs[0], hs[1], hs[0]])
    b = mpopf.Batch(hs)
    b.set_io(ios)
    _check_all(b, ios, refs)
    b.close()
