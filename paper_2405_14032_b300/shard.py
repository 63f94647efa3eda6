"""Period shards across GPUs: the split of the horizon, the halo exchange and
the local <-> whole-horizon index ranges (``mpopf_shard_plan`` /
``mpopf_shard_setup`` in ``include/mpopf.h``).

Only the ramp rows (Eq. 1k) couple periods, so each rank owns a contiguous
block of periods.  Before an evaluation a rank receives two G-vectors (per
ramp block: P, and Q with the reactive ramp): pg[t0 - 1] from the previous
rank, which its ramp rows at t0 read, and D of the ramp rows at t1 from the
next rank, the last term of its pg diagonals of M at t1 - 1.  The objective is
the sum of the ranks' partial objectives.  This module moves those values with
torch.distributed point-to-point calls (NCCL between GPUs, gloo on the host);
it computes nothing of the method itself.
"""
from __future__ import annotations


def split(T: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous blocks [t0, t1) covering [0, T), sizes differing by at most
    one (the first T mod parts blocks one longer)."""
    if not 1 <= parts <= T:
        raise ValueError(f"cannot split {T} periods into {parts} shards")
    q, r = divmod(T, parts)
    out, t = [], 0
    for k in range(parts):
        n = q + (1 if k < r else 0)
        out.append((t, t + n))
        t += n
    return out


def scatter(plan: dict, what: str, whole, local):
    """Copy the whole-horizon entries of range kind `what` ("x", "xall",
    "rows", "jac", "hess", "kkt") into the shard's local array."""
    for lo, gl, n in plan["ranges"][what]:
        local[lo:lo + n] = whole[gl:gl + n]
    return local


def gather(plan: dict, what: str, local, whole):
    """Copy the shard's owned entries of range kind `what` into the
    whole-horizon array."""
    for lo, gl, n in plan["ranges"][what]:
        whole[gl:gl + n] = local[lo:lo + n]
    return whole


def map_columns(plan: dict, local_cols):
    """Whole-horizon variable index of each local variable index (numpy)."""
    import numpy as np
    cols = np.asarray(local_cols, dtype=np.int64)
    out = np.full(cols.shape, -1, dtype=np.int64)
    for lo, gl, n in plan["ranges"]["xall"]:
        sel = (cols >= lo) & (cols < lo + n)
        out[sel] = cols[sel] - lo + gl
    return out


def map_rows(plan: dict, local_rows):
    """Whole-horizon row index of each owned local row index (numpy; -1 for a
    row that is not owned)."""
    import numpy as np
    rows = np.asarray(local_rows, dtype=np.int64)
    out = np.full(rows.shape, -1, dtype=np.int64)
    for lo, gl, n in plan["ranges"]["rows"]:
        sel = (rows >= lo) & (rows < lo + n)
        out[sel] = rows[sel] - lo + gl
    return out


def halo_ops(plan: dict, x, dvec, rank: int, world: int):
    """The point-to-point operations of one halo exchange of this rank, as
    (kind, peer, tensor view) triples, kind "send" or "recv", in the order in
    which they are posted.  The next rank receives x[x_send] into its
    x[x_recv]; the previous rank receives dvec[d_send] into its dvec[d_recv]."""
    G = plan["halo_len"]
    ops = []
    if G == 0:
        return ops
    for b in range(plan["halo_blocks"]):
        if rank + 1 < world:
            o = plan["x_send"][b]
            ops.append(("send", rank + 1, x[o:o + G]))
            o = plan["d_recv"][b]
            ops.append(("recv", rank + 1, dvec[o:o + G]))
        if rank > 0:
            o = plan["x_recv"][b]
            ops.append(("recv", rank - 1, x[o:o + G]))
            o = plan["d_send"][b]
            ops.append(("send", rank - 1, dvec[o:o + G]))
    return ops


def exchange_halos(plan: dict, x, dvec, rank: int, world: int, group=None):
    """One halo exchange (all sends and receives posted together, then
    waited for): x and dvec are this rank's local arrays (torch tensors).
    With NCCL the device tensors move directly; with gloo, device tensors are
    staged through host memory."""
    import torch.distributed as dist
    triples = halo_ops(plan, x, dvec, rank, world)
    if not triples:
        return
    staged = dist.get_backend(group) == "gloo" and x.is_cuda
    bufs = [t.cpu() if staged else t for _, _, t in triples]
    ops = [dist.P2POp(dist.isend if kind == "send" else dist.irecv, b, peer, group)
           for (kind, peer, _), b in zip(triples, bufs)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    if staged:
        for (kind, _, t), b in zip(triples, bufs):
            if kind == "recv":
                t.copy_(b)


def exchange_halos_async(plan: dict, x, dvec, rank: int, world: int, stream, event, group=None):
    """The halo exchange on its own CUDA `stream` (ordered after the work
    enqueued on the current stream so far), with `event` recorded on that
    stream after it.  A shard handle whose generator work waits for `event`
    (Handle.set_gen_dependency) can be evaluated right away: its branch and
    bus kernels, which read no halo value, overlap the exchange."""
    import torch
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        exchange_halos(plan, x, dvec, rank, world, group)
        event.record(stream)


def reduce_objective_async(f, buf, stream, group=None):
    """The whole objective into `buf` (a one-element tensor on f's device):
    f is copied into buf and buf summed over the ranks on `stream`, ordered
    after the work enqueued on the current stream so far; later work on
    `stream` is ordered after the sum, while the current stream goes on (the
    next evaluation, which rewrites f, does not wait for it).  Under gloo the
    sum is taken synchronously (host-staged)."""
    import torch
    import torch.distributed as dist
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        buf.copy_(f)
        if dist.get_backend(group) == "gloo":
            reduce_objective(buf, group)
        else:
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group, async_op=True).wait()
    return buf


def reduce_objective(f, group=None):
    """The whole objective from the ranks' partial objectives (sum, in place;
    staged through host memory for a device tensor under gloo)."""
    import torch.distributed as dist
    if dist.get_backend(group) == "gloo" and f.is_cuda:
        h = f.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        f.copy_(h)
    else:
        dist.all_reduce(f, op=dist.ReduceOp.SUM, group=group)
    return f
