"""Run one workload of the library a few times, for an external profiler.

    python -m paper_2405_14032_b300.profile_run sweep|ipm|adjoint|csc|batch|points \
        [--buses 10000] [--periods 24] [--reps 3]

The network is the seeded synthetic one (L = 1.6 N, G = 0.2 N, D = 0.6 N,
seed 3); every call goes through the C ABI exactly as an application would
call it, with inputs resident on the device.  Nothing is timed or checked
here: the profiler measures.
"""
from __future__ import annotations

import argparse

import torch

from . import mpopf, synth


def _instance(buses: int, periods: int, seed: int = 3):
    return synth.make_instance(seed, buses, round(1.6 * buses), round(0.2 * buses), round(0.6 * buses), periods)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", choices=["sweep", "ipm", "adjoint", "csc", "batch", "points"])
    ap.add_argument("--buses", type=int, default=10000)
    ap.add_argument("--periods", type=int, default=24)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--launches", type=int, default=1, choices=[0, 1, 2],
                    help="batch: one persistent launch or two (generator/branch, then bus/objective), or 0: "
                         "the plain sweeps on --streams parallel graph branches")
    ap.add_argument("--streams", type=int, default=32, help="batch --launches 0: parallel graph branches")
    ap.add_argument("--points", type=int, default=16, help="points: points per mpopf_sweep_points call")
    ap.add_argument("--instances", type=int, default=64,
                    help="batch: the first INSTANCES of the 64 benchmark instances (a smaller capture)")
    a = ap.parse_args(argv)
    dev = lambda v: torch.as_tensor(v, dtype=torch.float64, device="cuda")

    if a.workload == "batch":
        shapes = synth.batch_shapes(64)[:max(1, min(64, a.instances))]
        hs, ios = [], []
        for s in shapes:
            inst = synth.make_instance(s["seed"], s["n_bus"], s["n_branch"], s["n_gen"], s["n_load"], s["T"])
            pt = synth.make_point(s["seed"], inst)
            h = mpopf.Handle(inst)
            io = dict(x=dev(pt.x), lam=dev(pt.lam), sigma=pt.sigma, sigma_x=dev(pt.sigma_x), dvec=dev(pt.dvec),
                      delta_w=pt.delta_w)
            io.update(h.new_outputs())
            hs.append(h)
            ios.append(io)
        b = mpopf.Batch(hs)
        b.set_io(ios)
        if a.launches == 2:
            b.set_schedule(0, 1, 3, 0, 2)
        elif a.launches == 0:
            b.set_schedule(1, 1, a.streams, 0, 0)
        for _ in range(a.reps):
            b.sweep()
        b.status()
        torch.cuda.synchronize()
        print(f"batch: {a.reps} batched sweeps of {len(shapes)} instances")
        return 0

    inst = _instance(a.buses, a.periods)
    pt = synth.make_point(3, inst)
    h = mpopf.Handle(inst)
    x, lam, sx, dv = dev(pt.x), dev(pt.lam), dev(pt.sigma_x), dev(pt.dvec)
    out = h.new_outputs()
    if a.workload == "sweep":
        for _ in range(a.reps):
            h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=out)
    elif a.workload == "points":
        k = max(1, a.points)
        X = dev(pt.x).unsqueeze(0) + 1e-3 * torch.randn(k, h.n, dtype=torch.float64, device="cuda",
                                                        generator=torch.Generator(device="cuda").manual_seed(3))
        rep = lambda t: t.unsqueeze(0).repeat(k, 1).contiguous()
        LAM, SX, DV = rep(lam), rep(sx), rep(dv)
        outs = h.new_point_outputs(k)
        for _ in range(a.reps):
            h.sweep_points(X, LAM, pt.sigma, SX, DV, pt.delta_w, out=outs)
    elif a.workload == "adjoint":
        y = dev(synth.uniform(3, 5000, h.m, -1.0, 1.0))
        v = dev(synth.normal(3, 9000, h.n))
        for _ in range(a.reps):
            h.vjp(x, y)
            h.jvp(x, v)
            h.hvp(x, lam, pt.sigma, v)
    elif a.workload == "csc":
        h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=out)
        for which, key in ((mpopf.CSC_JAC, "jv"), (mpopf.CSC_HESS, "hv")):
            h.csc_pattern(which)
            for _ in range(a.reps):
                h.coo_to_csc(which, out[key])
    else:  # ipm: an interior point from the pattern's bounds (midpoints, unit duals)
        pat = h.pattern()
        eps = 1e-2
        xl, xu, gl, gu = (pat[k] for k in ("xl", "xu", "gl", "gu"))

        def interior(lo, hi, other):
            fl, fu = torch.isfinite(lo), torch.isfinite(hi)
            w = torch.where(fl & fu, 0.5 * (lo + hi), other)
            w = torch.where(fl & ~fu, lo + 0.5, w)
            return torch.where(~fl & fu, hi - 0.5, w)

        eq = gl == gu
        sl, su = torch.where(eq, gl - eps, gl), torch.where(eq, gu + eps, gu)
        xi = interior(xl, xu, torch.zeros_like(xl))
        s = interior(sl, su, torch.zeros_like(sl))
        one = lambda b: torch.where(torch.isfinite(b), 1.0, 0.0).double()
        zlx, zux, zls, zus = one(xl), one(xu), one(sl), one(su)
        y = torch.full_like(s, 0.25)
        ev = h.eval(mpopf.OUT_GRAD | mpopf.OUT_CONS, xi)
        for _ in range(a.reps):
            sigx, dvec, cvec, recip = h.ipm_prepare(xi, s, zlx, zux, zls, zus, 1e-3, 1e-4, eps)
            rhs = h.ipm_rhs(xi, s, y, ev["grad"], ev["c"], recip, dvec, cvec, 0.05)
            h.ipm_recover(xi, s, y, zlx, zux, zls, zus, ev["c"], recip, cvec, rhs, 0.05, 1e-3, 1e-4)
    torch.cuda.synchronize()
    h.close()
    print(f"{a.workload}: {a.reps} reps, {a.buses} buses x {a.periods} periods")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
