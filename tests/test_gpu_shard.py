"""Period shards through the C-ABI on one GPU: the horizon split into 2, 3 or
4 contiguous blocks (one-period shards included), one shard handle each
(mpopf_shard_setup), every halo entry of the local inputs NaN until the halo
exchange (device copies between the shards' own arrays, the protocol that
shard.exchange_halos runs across GPUs), one sweep per shard; the owned outputs
placed by the plan's ranges equal the unsharded mpopf_sweep's bit for bit (f,
the sum of the shards' partial objectives, within 1e-12), and the shards'
local patterns map onto the whole pattern."""
import numpy as np
import pytest

from paper_2405_14032_b300 import shard, synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = (("grad", "x"), ("c", "rows"), ("jv", "jac"), ("hv", "hess"), ("kv", "kkt"))


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _instances():
    yield "cfg1", synth.config_instance("cfg1"), (2, 3, 4)
    yield "ragged_T7", synth.make_instance(61, 333, 530, 67, 200, 7), (2, 3)
    yield "qramp_T6", synth.with_reactive_ramp(synth.make_instance(62, 200, 320, 40, 120, 6)), (2, 3, 6)
    yield "no_gens_T5", H.instance(H.network(5, [0, 1, 2, 3], [1, 2, 3, 4], [0.01] * 4, [0.1] * 4, [0.02] * 4,
                                             ref=2), 5, pd=np.zeros(0), qd=np.zeros(0)), (2,)
    yield "cfg2", synth.config_instance("cfg2"), (3,)


CASES = {name: (inst, parts) for name, inst, parts in _instances()}


def _exchange(plans, xs, dvs):
    """The halo exchange as device copies (k-th receive from a peer <- k-th
    send of that peer)."""
    world = len(plans)
    ops = [shard.halo_ops(plans[r], xs[r], dvs[r], r, world) for r in range(world)]
    for r in range(world):
        for peer in {p for _, p, _ in ops[r]}:
            recvs = [t for kind, p, t in ops[r] if kind == "recv" and p == peer]
            sends = [t for kind, p, t in ops[peer] if kind == "send" and p == r]
            assert len(recvs) == len(sends)
            for dst, src in zip(recvs, sends):
                dst.copy_(src)


def run_shards(inst, pt, parts, schedule=(0, 0)):
    """Whole-size outputs stitched from `parts` shard sweeps, plus the shards."""
    from paper_2405_14032_b300 import mpopf
    spans = shard.split(inst.T, parts)
    plans = [mpopf.shard_plan(inst.net, inst.T, t0, t1) for t0, t1 in spans]
    hs = [mpopf.Handle(inst, shard=s) for s in spans]
    ins = []
    for p in plans:
        nan = lambda k: torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        x, sx, lam, dv = nan(p["n"]), nan(p["n"]), nan(p["m"]), nan(p["m"])
        shard.scatter(p, "x", _dev(pt.x), x)
        shard.scatter(p, "x", _dev(pt.sigma_x), sx)
        shard.scatter(p, "rows", _dev(pt.lam), lam)
        shard.scatter(p, "rows", _dev(pt.dvec), dv)
        ins.append((x, lam, sx, dv))
    _exchange(plans, [i[0] for i in ins], [i[3] for i in ins])
    outs = []
    for h, (x, lam, sx, dv) in zip(hs, ins):
        h.set_sweep_schedule(*schedule)
        out = h.new_outputs()
        for v in out.values():
            v.fill_(float("nan"))
        h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=out)
        outs.append(out)
    torch.cuda.synchronize()
    return plans, hs, outs


@pytest.mark.parametrize("name", sorted(CASES))
def test_shards_stitch_to_the_unsharded_sweep(name):
    from paper_2405_14032_b300 import mpopf
    inst, parts_list = CASES[name]
    pt = synth.make_point(7, inst)
    h = mpopf.Handle(inst)
    ref = h.sweep(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    pat = {k: v.cpu().numpy() for k, v in h.pattern().items()}
    torch.cuda.synchronize()
    for parts in parts_list:
        # period chunks for two shards, the bus-end products' own launch (with the
        # programmatic dependencies) for three, the plain launches otherwise
        plans, hs, outs = run_shards(inst, pt, parts, schedule=(2, 0) if parts == 2 else (0, 20) if parts == 3
                                     else (0, 0))
        for key, what in KEYS:
            whole = torch.full_like(ref[key], float("nan"))
            for p, out in zip(plans, outs):
                shard.gather(p, what, out[key], whole)
            assert torch.equal(whole, ref[key]), (name, parts, key)
        f = sum(float(out["f"][0]) for out in outs)
        fr = float(ref["f"][0])
        assert abs(f - fr) <= 1e-12 * abs(fr) + 1e-14, (name, parts, f, fr)
        # local patterns, mapped to whole-model indices, are the whole pattern's owned entries
        for p, hs_ in zip(plans, hs):
            lp = {k: v.cpu().numpy() for k, v in hs_.pattern().items()}
            for l0, g0, n in p["ranges"]["jac"]:
                assert np.array_equal(shard.map_rows(p, lp["jac_row"][l0:l0 + n]), pat["jac_row"][g0:g0 + n])
                assert np.array_equal(shard.map_columns(p, lp["jac_col"][l0:l0 + n]), pat["jac_col"][g0:g0 + n])
            for l0, g0, n in p["ranges"]["hess"]:
                assert np.array_equal(shard.map_columns(p, lp["hess_row"][l0:l0 + n]), pat["hess_row"][g0:g0 + n])
                assert np.array_equal(shard.map_columns(p, lp["hess_col"][l0:l0 + n]), pat["hess_col"][g0:g0 + n])
            for l0, g0, n in p["ranges"]["kkt"]:
                assert np.array_equal(shard.map_columns(p, lp["kkt_col"][l0:l0 + n]), pat["kkt_col"][g0:g0 + n])
            for l0, g0, n in p["ranges"]["x"]:
                assert np.array_equal(np.diff(lp["kkt_rowptr"][l0:l0 + n + 1]), np.diff(pat["kkt_rowptr"][g0:g0 + n + 1]))
                for k in ("xl", "xu"):
                    assert np.array_equal(lp[k][l0:l0 + n], pat[k][g0:g0 + n])
            for l0, g0, n in p["ranges"]["rows"]:
                for k in ("gl", "gu"):
                    assert np.array_equal(lp[k][l0:l0 + n], pat[k][g0:g0 + n])
        for hs_ in hs:
            hs_.close()
    h.close()


def test_shard_handles_refuse_other_entry_points():
    from paper_2405_14032_b300 import mpopf
    inst = synth.config_instance("cfg1")
    pt = synth.make_point(1, inst)
    hsh = mpopf.Handle(inst, shard=(1, 3))
    p = mpopf.shard_plan(inst.net, inst.T, 1, 3)
    assert (hsh.n, hsh.m, hsh.nnz_kkt) == (p["n"], p["m"], p["nnz_kkt"])
    x = torch.zeros(hsh.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(hsh.m, dtype=torch.float64, device="cuda")
    for call in (lambda: hsh.vjp(x, y), lambda: hsh.jvp(x, x), lambda: hsh.hvp(x, y, 1.0, x),
                 lambda: hsh.csc_pattern(mpopf.CSC_JAC),
                 lambda: hsh.assemble_kkt_noalloc(x, y, 1.0, x, y, 0.0, torch.zeros(hsh.nnz_kkt, dtype=torch.float64,
                                                                                      device="cuda")),
                 lambda: mpopf.Batch([hsh])):
        with pytest.raises(mpopf.MpopfError, match="period shard"):
            call()
    with pytest.raises(mpopf.MpopfError, match="t0 < t1"):
        mpopf.Handle(inst, shard=(2, 2))
    with pytest.raises(mpopf.MpopfError, match="t0 < t1"):
        mpopf.Handle(inst, shard=(0, 5))
    hsh.close()


def test_benchmark_workload_in_three_shards():
    """The 10k-bus, 168-period workload as bench.py's sharded mode splits it
    for three GPUs (periods 0-55, 56-111, 112-167): stitched outputs equal the
    unsharded sweep bit for bit."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(3, 10000, 16000, 2000, 6000, 168)
    pt = synth.make_point(3, inst)
    plans, hs, outs = run_shards(inst, pt, 3)
    h = mpopf.Handle(inst)
    ref = h.sweep(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    torch.cuda.synchronize()
    for key, what in KEYS:
        w = torch.full_like(ref[key], float("nan"))
        for p, out in zip(plans, outs):
            shard.gather(p, what, out[key], w)
        assert torch.equal(w, ref[key]), key
        del w
    f = sum(float(out["f"][0]) for out in outs)
    assert abs(f - float(ref["f"][0])) <= 1e-12 * abs(float(ref["f"][0]))
    for x in hs + [h]:
        x.close()


def test_halo_exchange_on_another_stream_is_waited_for():
    """The halo copies run on a stream of their own, held back by a delay on
    that stream, while the shards are evaluated at once; the generator work
    waits for the exchange through the handle's dependency event
    (mpopf_set_gen_dependency), so the stitched outputs are still exact (a
    generator kernel that ran early would read the NaN halo slots)."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.with_reactive_ramp(synth.make_instance(64, 300, 480, 60, 180, 9))
    pt = synth.make_point(9, inst)
    h = mpopf.Handle(inst)
    ref = h.sweep(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    torch.cuda.synchronize()
    spans = shard.split(inst.T, 3)
    plans = [mpopf.shard_plan(inst.net, inst.T, t0, t1) for t0, t1 in spans]
    hs = [mpopf.Handle(inst, shard=sp) for sp in spans]
    ins = []
    for p in plans:
        nan = lambda k: torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        x, sx, lam, dv = nan(p["n"]), nan(p["n"]), nan(p["m"]), nan(p["m"])
        shard.scatter(p, "x", _dev(pt.x), x)
        shard.scatter(p, "x", _dev(pt.sigma_x), sx)
        shard.scatter(p, "rows", _dev(pt.lam), lam)
        shard.scatter(p, "rows", _dev(pt.dvec), dv)
        ins.append((x, lam, sx, dv))
    halo = torch.cuda.Stream()
    ev = torch.cuda.Event()
    halo.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(halo):
        torch.cuda._sleep(50_000_000)  # holds the copies back (a bounded busy loop on this stream)
        _exchange(plans, [i[0] for i in ins], [i[3] for i in ins])
        ev.record(halo)
    outs = []
    for hs_, (x, lam, sx, dv) in zip(hs, ins):
        hs_.set_gen_dependency(ev)
        outs.append(hs_.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w))
    torch.cuda.synchronize()
    for key, what in KEYS:
        whole = torch.full_like(ref[key], float("nan"))
        for p, out in zip(plans, outs):
            shard.gather(p, what, out[key], whole)
        assert torch.equal(whole, ref[key]), key
    for hs_ in hs:
        hs_.set_gen_dependency(None)
        hs_.close()
    h.close()
