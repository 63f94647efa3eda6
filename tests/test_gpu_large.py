"""Beyond 2^31 value entries.  The 100,000-bus network (L = 160,000, G =
20,000, D = 60,000) with T = 440 periods has n = 387M variables and m = 590M
rows (indices below 2^31, as the ABI requires) but 2.2e9 Jacobian entries and
2.5e9 entries of M, so every kernel offset into J, W and M past 2^31 is
exercised.  Periods are coupled only by the ramp rows, so every output of the
last period must equal, bit for bit, period 1 of the same network evaluated
with T = 2 on the big instance's last two periods of inputs and loads.  The
comparison runs on the device.  Needs about 140 GB of device memory: skipped
when less than 180 GB is free on the device, or with MPOPF_LARGE=0."""
import os

import numpy as np
import pytest

from paper_2405_14032_b300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("MPOPF_LARGE") == "0", reason="MPOPF_LARGE=0 (~140 GB test)")]

torch = pytest.importorskip("torch")

NEED_BYTES = 180 * 2**30

N, L, G, D, T = 100_000, 160_000, 20_000, 60_000, 440


class Layout:
    """Offsets of the variable, row, J and W layouts (include/mpopf.h)."""

    def __init__(self, T, jk8_per):
        self.T, self.jk8 = T, jk8_per
        TN, TG, TL = T * N, T * G, T * L
        self.var_start = [0, TN, 2 * TN, 2 * TN + TG, 2 * TN + 2 * TG, 2 * TN + 2 * TG + 2 * TL]
        self.var_per = [N, N, G, G, 2 * L, 2 * L]
        self.n = 2 * TN + 2 * TG + 4 * TL

    def vars_of(self, kind, t):
        s = self.var_start[kind] + t * self.var_per[kind]
        return s, s + self.var_per[kind]

    def row_blocks(self, t):  # (first, count) of every row kind at period t (t >= 1)
        T, TL, TN = self.T, self.T * L, self.T * N
        out = [(t, 1)] + [(T + (k - 1) * TL + t * L, L) for k in range(1, 8)]
        out += [(T + 7 * TL + t * N, N), (T + 7 * TL + TN + t * N, N)]
        out += [(T + 7 * TL + 2 * TN + (t - 1) * G, G)]
        return out

    def jac_blocks(self, t):
        T, TL = self.T, self.T * L
        j5, j8 = T + 20 * TL, T + 26 * TL
        out = [(t, 1)] + [(T + 5 * (k - 1) * TL + 5 * t * L, 5 * L) for k in range(1, 5)]
        out += [(j5 + (k - 5) * 2 * TL + 2 * t * L, 2 * L) for k in range(5, 8)]
        out += [(j8 + t * self.jk8, self.jk8), (j8 + T * self.jk8 + t * self.jk8, self.jk8)]
        out += [(j8 + 2 * T * self.jk8 + 2 * (t - 1) * G, 2 * G)]
        return out

    def hess_blocks(self, t):
        TG, TL = self.T * G, self.T * L
        return [(t * G, G), (TG + 10 * t * L, 10 * L), (TG + 10 * TL + 4 * t * L, 4 * L),
                (TG + 14 * TL + 2 * t * N, 2 * N)]


def _slice(a, first, count):
    return a[first:first + count]


def test_last_period_of_a_beyond_2e31_instance():
    from paper_2405_14032_b300 import mpopf
    free, _ = torch.cuda.mem_get_info()
    if free < NEED_BYTES:
        pytest.skip(f"{free / 2**30:.0f} GiB free on the device, the test needs about 140 GB")
    big = synth.make_instance(11, N, L, G, D, T)
    hb = mpopf.Handle(big)
    assert hb.nnz_jac > 2**31 and hb.nnz_kkt > 2**31 and hb.n < 2**31 and hb.m < 2**31
    gen = torch.Generator(device="cuda").manual_seed(11)
    u = lambda k, lo, hi: lo + (hi - lo) * torch.rand(k, generator=gen, device="cuda", dtype=torch.float64)
    xb = u(hb.n, 0.9, 1.1)
    lb, sb, db = u(hb.m, -1.0, 1.0), u(hb.n, 0.1, 10.0), u(hb.m, 0.1, 10.0)
    ob = hb.sweep(xb, lb, 1.0, sb, db, 1e-8)

    small = synth.Instance(net=big.net, T=2, pd=big.pd[T - 2:], qd=big.qd[T - 2:])
    hs = mpopf.Handle(small)
    jk8 = N + G + 2 * L
    lay_b, lay_s = Layout(T, jk8), Layout(2, jk8)
    # inputs of periods T-2, T-1 in the small instance's layout
    two = lambda v, k: torch.cat([v[slice(*lay_b.vars_of(k, T - 2))], v[slice(*lay_b.vars_of(k, T - 1))]])
    xs = torch.cat([two(xb, k) for k in range(6)])
    ss = torch.cat([two(sb, k) for k in range(6)])
    TL, TN = T * L, T * N

    def rows_small(v):  # rows of periods T-2, T-1 (the ramp rows of period T-1 only)
        parts = [v[T - 2:T]]
        parts += [_slice(v, T + (k - 1) * TL + (T - 2) * L, 2 * L) for k in range(1, 8)]
        parts += [_slice(v, T + 7 * TL + (T - 2) * N, 2 * N), _slice(v, T + 7 * TL + TN + (T - 2) * N, 2 * N)]
        parts += [_slice(v, T + 7 * TL + 2 * TN + (T - 2) * G, G)]
        return torch.cat(parts)

    ls, ds = rows_small(lb), rows_small(db)
    assert xs.numel() == hs.n and ls.numel() == hs.m
    os_ = hs.sweep(xs, ls, 1.0, ss, ds, 1e-8)
    torch.cuda.synchronize()

    # every output of big period T-1 equals small period 1
    for (fb, cb), (fs, cs) in zip(lay_b.row_blocks(T - 1), lay_s.row_blocks(1)):
        assert cb == cs and torch.equal(_slice(ob["c"], fb, cb), _slice(os_["c"], fs, cs)), ("c", fb)
    for k in range(6):
        assert torch.equal(ob["grad"][slice(*lay_b.vars_of(k, T - 1))], os_["grad"][slice(*lay_s.vars_of(k, 1))])
    for (fb, cb), (fs, cs) in zip(lay_b.jac_blocks(T - 1), lay_s.jac_blocks(1)):
        assert cb == cs and torch.equal(_slice(ob["jv"], fb, cb), _slice(os_["jv"], fs, cs)), ("jv", fb)
    for (fb, cb), (fs, cs) in zip(lay_b.hess_blocks(T - 1), lay_s.hess_blocks(1)):
        assert torch.equal(_slice(ob["hv"], fb, cb), _slice(os_["hv"], fs, cs)), ("hv", fb)
    assert max(f + c for f, c in lay_b.jac_blocks(T - 1)) > 2**31  # its last J blocks lie beyond 2^31

    # rows of M of the last period's variables: values equal; columns map
    # period T-2 -> 0 and T-1 -> 1 within each variable kind
    pb, ps = hb.pattern(), hs.pattern()
    vs = torch.tensor(lay_b.var_start + [lay_b.n], device="cuda")
    per_b = torch.tensor(lay_b.var_per, device="cuda")
    start_s = torch.tensor(lay_s.var_start, device="cuda")
    for k in range(6):
        rb0, rb1 = lay_b.vars_of(k, T - 1)
        rs0, rs1 = lay_s.vars_of(k, 1)
        a0, a1 = int(pb["kkt_rowptr"][rb0]), int(pb["kkt_rowptr"][rb1])
        b0, b1 = int(ps["kkt_rowptr"][rs0]), int(ps["kkt_rowptr"][rs1])
        assert a1 - a0 == b1 - b0 and a1 > a0
        assert torch.equal(ob["kv"][a0:a1], os_["kv"][b0:b1]), ("kv", k)
        cb = pb["kkt_col"][a0:a1].long()
        kind = torch.searchsorted(vs, cb, right=True) - 1
        local = cb - vs[kind]
        t = torch.div(local, per_b[kind], rounding_mode="floor")
        mapped = start_s[kind] + (t - (T - 2)) * per_b[kind] + (local - t * per_b[kind])
        assert torch.equal(mapped, ps["kkt_col"][b0:b1].long()), ("kkt_col", k)
    assert int(pb["kkt_rowptr"][lay_b.vars_of(5, T - 1)[0]]) > 2**31  # M entries beyond 2^31
    hs.close()
    hb.close()
