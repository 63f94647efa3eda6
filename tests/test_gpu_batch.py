"""Batched sweeps: many uneven instances in one persistent launch (CUDA graph)
give, for every instance, the same outputs bit for bit as mpopf_sweep on that
instance alone, whatever the schedule; the autotuner keeps that property."""
import numpy as np
import pytest

from paper_2405_14032_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("f", "grad", "c", "jv", "hv", "kv")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _setup(shapes):
    from paper_2405_14032_b300 import mpopf
    hs, ios, refs = [], [], []
    for k, shape in enumerate(shapes):
        N, L, G, D, T = shape[:5]
        inst = synth.make_instance(100 + k, N, L, G, D, T)
        if len(shape) > 5 and shape[5] == "qramp":
            inst = synth.with_reactive_ramp(inst)
        pt = synth.make_point(100 + k, inst)
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
    hs, ios, refs = _setup(SMALL)
    b = mpopf.Batch(hs)
    b.set_io(ios)
    _check_all(b, ios, refs)
    for sched in [(0, 1, 0, 0), (1, 1, 1, 1), (0, 2, 2, 2), (1, 4, 0, 3), (0, 4, 1, 0), (1, 2, 3, 1), (0, 1, 0, 2),
                  (0, 1, 0, 0, 2), (1, 2, 1, 0, 2), (0, 4, 3, 0, 2)]:
        b.set_schedule(*sched)
        _check_all(b, ios, refs)
        _check_all(b, ios, refs)  # replay of the same graph
    best = b.tune(reps=2)
    assert best > 0
    _check_all(b, ios, refs)
    for bad in [(0, 1, 0, 0, 0), (0, 1, 0, 0, 3), (2, 1, 0, 0, 1), (0, 0, 0, 0, 1), (0, 1, -1, 0, 1)]:
        with pytest.raises(mpopf.MpopfError, match="bad argument"):
            b.set_schedule(*bad)
    _check_all(b, ios, refs)
    b.close()


def test_batch_64_uneven_instances():
    """The batched workload: 64 instances, buses log-uniform in [500, 5000],
    L = 1.6 N, G = 0.2 N, D = 0.6 N, T in {12, 24, 48, 96}."""
    from paper_2405_14032_b300 import mpopf
    shapes = [(s["n_bus"], s["n_branch"], s["n_gen"], s["n_load"], s["T"]) for s in synth.batch_shapes(64)]
    hs, ios, refs = _setup(shapes)
    b = mpopf.Batch(hs)
    b.set_io(ios)
    _check_all(b, ios, refs)
    b.tune(reps=2)
    _check_all(b, ios, refs)
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
    # with two launches nothing waits: the hook has no wait to hold back
    b.set_schedule(0, 1, 0, 0, 2)
    assert b.schedule()["launches"] == 2
    with pytest.raises(mpopf.MpopfError, match="no bus tile waits"):
        b.test_stall(True)
    _check_all(b, ios, refs)
    b.close()
