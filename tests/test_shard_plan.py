"""Period shards on the host (no GPU): the layout of mpopf_shard_plan, the
halo-exchange protocol and the stitching of owned outputs.

The oracle stands in for the GPU here: each shard's local model (its owned
periods plus a halo period on each side that has a neighbour) is evaluated by
the CPU oracle on the owned periods only, after a halo exchange that copies
values from the neighbouring shards' local arrays (never from the whole
model).  The owned outputs, placed by the plan's ranges, must equal the
whole-horizon oracle's outputs bit for bit (f, a sum over the shards, within
1e-12), which pins the plan's offsets and the exchange to the model of Eq. 1:
only the ramp rows (Eq. 1k) couple periods.
"""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import mpopf, shard, synth
from tests import helpers as H


def _cases():
    yield "cfg1", synth.config_instance("cfg1")
    yield "ragged_T7", synth.make_instance(61, 50, 80, 11, 30, 7)
    yield "qramp_T6", synth.with_reactive_ramp(synth.make_instance(62, 40, 66, 9, 20, 6))
    yield "no_gens_T5", H.instance(H.network(5, [0, 1, 2, 3], [1, 2, 3, 4], [0.01] * 4, [0.1] * 4, [0.02] * 4,
                                             ref=2), 5, pd=np.zeros(0), qd=np.zeros(0))


CASES = dict(_cases())


def test_split():
    assert shard.split(168, 8) == [(21 * k, 21 * (k + 1)) for k in range(8)]
    assert shard.split(7, 3) == [(0, 3), (3, 5), (5, 7)]
    assert shard.split(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    with pytest.raises(ValueError):
        shard.split(3, 4)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("parts", [1, 2, 3])
def test_owned_ranges_partition_every_array(name, parts):
    """The owned ranges of the shards cover every entry of every whole-horizon
    array exactly once, and every local range lies inside the local model's
    arrays, whose sizes are those of a T_loc-period model."""
    inst = CASES[name]
    o = oracle.Oracle(inst)
    rp = o.jac_rowptr()
    sizes = dict(x=o.n, rows=o.m, jac=o.nnz_jac, hess=o.nnz_hess, kkt=None)
    hits = {k: np.zeros(v, np.int32) for k, v in sizes.items() if v is not None}
    kkt_total = 0
    for t0, t1 in shard.split(inst.T, parts):
        p = mpopf.shard_plan(inst.net, inst.T, t0, t1)
        h0, h1 = int(t0 > 0), int(t1 < inst.T)
        assert (p["own0"], p["own1"], p["local_periods"]) == (h0, h0 + t1 - t0, t1 - t0 + h0 + h1)
        lo = oracle.Oracle(synth.Instance(net=inst.net, T=p["local_periods"], pd=inst.pd[t0 - h0:t1 + h1],
                                          qd=inst.qd[t0 - h0:t1 + h1]))
        assert (p["n"], p["m"], p["nnz_jac"], p["nnz_hess"]) == (lo.n, lo.m, lo.nnz_jac, lo.nnz_hess)
        local_size = dict(x=p["n"], xall=p["n"], rows=p["m"], jac=p["nnz_jac"], hess=p["nnz_hess"], kkt=p["nnz_kkt"])
        for what, rs in p["ranges"].items():
            for l0, g0, n in rs:
                assert 0 <= l0 and l0 + n <= local_size[what], (what, l0, n)
                if what in hits:
                    hits[what][g0:g0 + n] += 1
                if what == "kkt":
                    kkt_total += n
        # the J entries of the owned rows are the owned J ranges
        rows = np.concatenate([np.arange(g0, g0 + n) for _, g0, n in p["ranges"]["rows"]] or [np.zeros(0, int)])
        njac = sum(int(rp[r + 1] - rp[r]) for r in rows)
        assert njac == sum(n for _, _, n in p["ranges"]["jac"])
    for what, h in hits.items():
        assert np.all(h == 1), (what, np.nonzero(h != 1)[0][:5])
    pt = synth.make_point(1, inst)
    _, cols, _ = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    assert kkt_total == cols.size


def _pair_exchange(plans, xs, dvs):
    """Every rank's halo receives, filled from the matching sends of its
    neighbours (the k-th receive of rank r from peer p gets the k-th send of
    p to r, the order in which both post them): the protocol of
    shard.exchange_halos, carried out by plain copies."""
    world = len(plans)
    ops = [shard.halo_ops(plans[r], xs[r], dvs[r], r, world) for r in range(world)]
    for r in range(world):
        for peer in {p for _, p, _ in ops[r]}:
            recvs = [t for kind, p, t in ops[r] if kind == "recv" and p == peer]
            sends = [t for kind, p, t in ops[peer] if kind == "send" and p == r]
            assert len(recvs) == len(sends)
            for dst, src in zip(recvs, sends):
                dst[:] = src


def local_inputs(plan, inst, pt):
    """The shard's local inputs: owned entries from the whole-horizon point,
    every halo entry NaN (the exchange must supply the ones that are read)."""
    x = np.full(plan["n"], np.nan)
    sx = np.full(plan["n"], np.nan)
    lam = np.full(plan["m"], np.nan)
    dv = np.full(plan["m"], np.nan)
    shard.scatter(plan, "x", pt.x, x)
    shard.scatter(plan, "x", pt.sigma_x, sx)
    shard.scatter(plan, "rows", pt.lam, lam)
    shard.scatter(plan, "rows", pt.dvec, dv)
    return x, lam, sx, dv


def local_oracle(plan, inst):
    T0 = plan["t0"] - plan["own0"]
    T1 = T0 + plan["local_periods"]
    return oracle.Oracle(synth.Instance(net=inst.net, T=plan["local_periods"], pd=inst.pd[T0:T1], qd=inst.qd[T0:T1]))


def stitch_with_oracle(inst, pt, parts):
    """Whole-horizon outputs assembled from the shards' oracle evaluations."""
    o = oracle.Oracle(inst)
    plans = [mpopf.shard_plan(inst.net, inst.T, t0, t1) for t0, t1 in shard.split(inst.T, parts)]
    ins = [local_inputs(p, inst, pt) for p in plans]
    _pair_exchange(plans, [i[0] for i in ins], [i[3] for i in ins])
    out = dict(g=np.full(o.n, np.nan), c=np.full(o.m, np.nan), jv=np.full(o.nnz_jac, np.nan),
               hv=np.full(o.nnz_hess, np.nan))
    rows_all, cols_all, vals_all, f = [], [], [], 0.0
    for p, (x, lam, sx, dv) in zip(plans, ins):
        lo = local_oracle(p, inst)
        r = lo.eval(x, lam, pt.sigma, t0=p["own0"], t1=p["own1"])
        for key, what in (("g", "x"), ("c", "rows"), ("jv", "jac"), ("hv", "hess")):
            shard.gather(p, what, r[key], out[key])
        f += r["f"]
        rows, rowlen, cols, vals = lo.kkt(x, lam, pt.sigma, sx, dv, pt.delta_w, t0=p["own0"], t1=p["own1"])
        grow = shard.map_columns(p, rows)
        rows_all.append(np.repeat(grow, rowlen))
        cols_all.append(shard.map_columns(p, cols))
        vals_all.append(vals)
    return o, out, f, np.concatenate(rows_all), np.concatenate(cols_all), np.concatenate(vals_all)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("parts", [2, 3])
def test_shards_stitch_to_the_whole_model(name, parts):
    inst = CASES[name]
    if parts > inst.T:
        pytest.skip("more shards than periods")
    pt = synth.make_point(3, inst)
    o, out, f, rows, cols, vals = stitch_with_oracle(inst, pt, parts)
    ref = o.eval(pt.x, pt.lam, pt.sigma)
    for key in ("g", "c", "jv", "hv"):
        assert np.array_equal(out[key], ref[key]), key
    assert abs(f - ref["f"]) <= 1e-12 * abs(ref["f"]) + 1e-14
    rp, rc, rv = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    order = np.lexsort((cols, rows))
    assert np.array_equal(rows[order], np.repeat(np.arange(o.n), np.diff(rp)))
    assert np.array_equal(cols[order], rc)
    assert np.array_equal(vals[order], rv)


def test_exchange_fills_exactly_the_halo_values_read():
    """After the exchange the halo slots hold pg (qg) of period t0 - 1 and D of
    the ramp rows at t1 from the whole model; with a halo slot left NaN the
    stitched outputs differ (so the exchanged values are really read)."""
    inst = CASES["qramp_T6"]
    pt = synth.make_point(4, inst)
    plans = [mpopf.shard_plan(inst.net, inst.T, t0, t1) for t0, t1 in shard.split(inst.T, 3)]
    ins = [local_inputs(p, inst, pt) for p in plans]
    _pair_exchange(plans, [i[0] for i in ins], [i[3] for i in ins])
    G = inst.net.n_gen
    sl = H.var_slices(inst.net, inst.T)
    ro = H.row_offsets(inst.net, inst.T)
    for p, (x, lam, sx, dv) in zip(plans, ins):
        t0, t1 = p["t0"], p["t1"]
        assert p["halo_blocks"] == 2
        for b, (kind, rstart) in enumerate((("pg", ro[10]), ("qg", ro[11]))):
            if t0 > 0:
                want = pt.x[sl[kind]][(t0 - 1) * G:t0 * G]
                assert np.array_equal(x[p["x_recv"][b]:p["x_recv"][b] + G], want)
            else:
                assert p["x_recv"][b] == -1 and p["d_send"][b] == -1
            if t1 < inst.T:
                want = pt.dvec[rstart + (t1 - 1) * G:rstart + t1 * G]
                assert np.array_equal(dv[p["d_recv"][b]:p["d_recv"][b] + G], want)
            else:
                assert p["d_recv"][b] == -1 and p["x_send"][b] == -1
    # a missing halo value shows up in the outputs
    p, (x, lam, sx, dv) = plans[1], ins[1]
    x[p["x_recv"][0]] = np.nan
    r = local_oracle(p, inst).eval(x, lam, pt.sigma, t0=p["own0"], t1=p["own1"])
    assert np.isnan(r["c"]).any()
