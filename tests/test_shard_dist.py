"""The halo exchange of period shards over torch.distributed (gloo, on the
host, world sizes 2 and 3): each rank holds only its shard's local arrays,
with every halo entry NaN; after shard.exchange_halos the halo slots hold the
neighbours' values, each rank evaluates its owned periods with the CPU oracle
(standing in for the GPU), the partial objectives are summed by
shard.reduce_objective, and the stitched outputs equal the whole-horizon
oracle's bit for bit (f within 1e-12)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instance():
    from paper_2405_14032_b300 import synth
    return synth.with_reactive_ramp(synth.make_instance(63, 60, 96, 13, 36, 7))


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2405_14032_b300 import mpopf, shard, synth
        from tests import test_shard_plan as S
        inst = _instance()
        pt = synth.make_point(5, inst)
        t0, t1 = shard.split(inst.T, world)[rank]
        plan = mpopf.shard_plan(inst.net, inst.T, t0, t1)
        x, lam, sx, dv = (torch.from_numpy(a) for a in S.local_inputs(plan, inst, pt))
        shard.exchange_halos(plan, x, dv, rank, world)
        halo_ok = all(
            (o < 0 or not torch.isnan(t[o:o + plan["halo_len"]]).any())
            for t, offs in ((x, plan["x_recv"]), (dv, plan["d_recv"])) for o in offs)
        lo = S.local_oracle(plan, inst)
        x, lam, sx, dv = (a.numpy() for a in (x, lam, sx, dv))
        r = lo.eval(x, lam, pt.sigma, t0=plan["own0"], t1=plan["own1"])
        f = torch.tensor([r["f"]], dtype=torch.float64)
        shard.reduce_objective(f)
        rows, rowlen, cols, vals = lo.kkt(x, lam, pt.sigma, sx, dv, pt.delta_w, t0=plan["own0"], t1=plan["own1"])
        kkt = (np.repeat(shard.map_columns(plan, rows), rowlen), shard.map_columns(plan, cols), vals)
        parts = {}
        for key, what in (("g", "x"), ("c", "rows"), ("jv", "jac"), ("hv", "hess")):
            parts[key] = [(g0, r[key][l0:l0 + n].copy()) for l0, g0, n in plan["ranges"][what]]
        q.put((rank, halo_ok, float(f[0]), parts, kkt))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_gloo(world):
    import oracle
    from paper_2405_14032_b300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    inst = _instance()
    pt = synth.make_point(5, inst)
    o = oracle.Oracle(inst)
    ref = o.eval(pt.x, pt.lam, pt.sigma)
    out = {k: np.full(ref[k].size, np.nan) for k in ("g", "c", "jv", "hv")}
    rows, cols, vals = [], [], []
    for rank, halo_ok, f, parts, kkt in res:
        assert halo_ok, rank
        assert abs(f - ref["f"]) <= 1e-12 * abs(ref["f"]), (rank, f, ref["f"])
        for key, pieces in parts.items():
            for g0, a in pieces:
                out[key][g0:g0 + a.size] = a
        rows.append(kkt[0]); cols.append(kkt[1]); vals.append(kkt[2])
    for key in out:
        assert np.array_equal(out[key], ref[key]), key
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    rp, rc, rv = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    order = np.lexsort((cols, rows))
    assert np.array_equal(rows[order], np.repeat(np.arange(o.n), np.diff(rp)))
    assert np.array_equal(cols[order], rc) and np.array_equal(vals[order], rv)


def _lost_peer_worker(rank, world, port, q):
    import datetime
    import time

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    from paper_2405_14032_b300 import mpopf, shard
    inst = _instance()
    t0, t1 = shard.split(inst.T, world)[rank]
    plan = mpopf.shard_plan(inst.net, inst.T, t0, t1)
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()  # the message is sent before the process goes
        os._exit(0)  # leaves before its first exchange, without a goodbye
    x = torch.zeros(plan["n"], dtype=torch.float64)
    dv = torch.zeros(plan["m"], dtype=torch.float64)
    start = time.perf_counter()
    try:
        shard.exchange_halos(plan, x, dv, rank, world)
        q.put((rank, "no error"))
    except Exception as exc:  # the lost peer surfaces as an error, not a hang
        q.put((rank, f"error after {time.perf_counter() - start:.1f}s: {type(exc).__name__}"))


def test_lost_peer_is_an_error_not_a_hang():
    """A rank that leaves before a halo exchange: its neighbour's exchange
    ends with an error (the closed connection, or the process group's
    10-second timeout) instead of waiting forever."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lost_peer_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "left"
    assert res[0].startswith("error after"), res[0]
    assert float(res[0].split()[2].rstrip("s:")) < 60.0
