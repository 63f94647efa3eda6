"""Shared test helpers: small hand-built networks and dense reconstructions."""
from __future__ import annotations

import numpy as np

from paper_2405_14032_b300 import synth


def network(N, f, t, r, x, b, gen_bus=(), load_bus=(), ref=0, tap=None, shift=None, gs=None, bs=None,
            c2=None, c1=None):
    f = np.asarray(f, np.int32)
    t = np.asarray(t, np.int32)
    L = f.size
    G = len(gen_bus)
    D = len(load_bus)
    pmax = np.full(G, 3.0)
    return synth.Network(
        n_bus=N, n_branch=L, n_gen=G, n_load=D, ref_bus=ref,
        bus_gs=np.zeros(N) if gs is None else np.asarray(gs, float),
        bus_bs=np.zeros(N) if bs is None else np.asarray(bs, float),
        bus_vmin=np.full(N, 0.9), bus_vmax=np.full(N, 1.1),
        br_f=f, br_t=t, br_r=np.asarray(r, float), br_x=np.asarray(x, float), br_b=np.asarray(b, float),
        br_tap=np.ones(L) if tap is None else np.asarray(tap, float),
        br_shift=np.zeros(L) if shift is None else np.asarray(shift, float),
        br_smax=np.full(L, 1.5), br_angmin=np.full(L, -0.5), br_angmax=np.full(L, 0.5),
        gen_bus=np.asarray(gen_bus, np.int32),
        gen_c2=np.full(G, 0.05) if c2 is None else np.asarray(c2, float),
        gen_c1=np.full(G, 20.0) if c1 is None else np.asarray(c1, float),
        gen_c0=np.zeros(G), gen_pmin=np.zeros(G), gen_pmax=pmax, gen_qmin=-0.5 * pmax, gen_qmax=0.5 * pmax,
        gen_ramp=0.2 * pmax, load_bus=np.asarray(load_bus, np.int32))


def instance(net, T, pd=None, qd=None, seed=7):
    if pd is None:
        pd, qd = synth.make_loads(seed, net, T)
    return synth.Instance(net=net, T=T, pd=np.asarray(pd, float).reshape(T, net.n_load),
                          qd=np.asarray(qd, float).reshape(T, net.n_load))


def var_slices(net, T):
    N, L, G = net.n_bus, net.n_branch, net.n_gen
    o = np.cumsum([0, T * N, T * N, T * G, T * G, T * 2 * L, T * 2 * L])
    names = ["va", "vm", "pg", "qg", "p", "q"]
    return {k: slice(o[i], o[i + 1]) for i, k in enumerate(names)}


def row_offsets(net, T):
    """Start of each constraint kind K0..K10 (and the end)."""
    N, L, G = net.n_bus, net.n_branch, net.n_gen
    sizes = [T] + [T * L] * 7 + [T * N] * 2 + [G * (T - 1)]
    return np.concatenate([[0], np.cumsum(sizes)])


def dense_jac(rows, cols, vals, m, n):
    J = np.zeros((m, n))
    np.add.at(J, (rows, cols), vals)
    return J


def dense_sym(rows, cols, vals, n):
    W = np.zeros((n, n))
    np.add.at(W, (rows, cols), vals)
    off = rows != cols
    np.add.at(W, (cols[off], rows[off]), vals[off])
    return W


def csr_to_dense_sym(rowptr, cols, vals, n):
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return dense_sym(rows, cols.astype(np.int64), vals, n)


def ulp(x):
    return np.spacing(np.abs(x))


def ipm_point(inst, o, seed, eps):
    """A strictly interior point for the interior-point algebra: x inside its
    bounds, slacks inside [gl, gu] (equality rows widened to [g - eps, g + eps]),
    positive duals on finite bounds and 0 on infinite ones, y uniform in
    [-1, 1].  o provides n, m and bounds() (the oracle or a handle's pattern)."""
    rng = np.random.default_rng(seed)
    xl, xu, gl, gu = o.bounds()
    pt = synth.make_point(seed, inst)
    x = pt.x.copy()
    fin = np.isfinite(xl) & np.isfinite(xu)
    x[fin] = xl[fin] + (0.1 + 0.8 * rng.uniform(size=fin.sum())) * (xu[fin] - xl[fin])
    sl = np.where(gl == gu, gl - eps, gl)
    su = np.where(gl == gu, gu + eps, gu)
    both = np.isfinite(sl) & np.isfinite(su)
    s = np.where(np.isfinite(su), su - rng.uniform(0.1, 1.0, o.m), sl + rng.uniform(0.1, 1.0, o.m))
    s[both] = sl[both] + (0.1 + 0.8 * rng.uniform(size=both.sum())) * (su[both] - sl[both])
    zlx = np.where(np.isfinite(xl), rng.uniform(0.1, 2.0, o.n), 0.0)
    zux = np.where(np.isfinite(xu), rng.uniform(0.1, 2.0, o.n), 0.0)
    zls = np.where(np.isfinite(sl), rng.uniform(0.1, 2.0, o.m), 0.0)
    zus = np.where(np.isfinite(su), rng.uniform(0.1, 2.0, o.m), 0.0)
    y = rng.uniform(-1, 1, o.m)
    return x, s, y, zlx, zux, zls, zus, xl, xu, sl, su


def lifted_system(W, A, x, s, y, zlx, zux, zls, zus, xl, xu, sl, su, grad, c, mu, dw, dc):
    """The full block system of Eq. (5) (unknowns dx, ds, dy and the bound-dual
    steps of the finite bounds only), assembled densely, with its right-hand
    side as printed.  Returns (K, p, slices of the seven blocks)."""
    n, m = x.size, s.size
    il, iu = np.nonzero(np.isfinite(xl))[0], np.nonzero(np.isfinite(xu))[0]
    jl, ju = np.nonzero(np.isfinite(sl))[0], np.nonzero(np.isfinite(su))[0]
    sizes = [n, m, m, il.size, iu.size, jl.size, ju.size]
    off = np.concatenate([[0], np.cumsum(sizes)])
    K = np.zeros((off[-1], off[-1]))
    X, S_, Y, ZLX, ZUX, ZLS, ZUS = (slice(off[k], off[k + 1]) for k in range(7))
    K[X, X] = W + dw * np.eye(n)
    K[X, Y] = A.T
    K[X, ZLX][il, np.arange(il.size)] = -1.0
    K[X, ZUX][iu, np.arange(iu.size)] = 1.0
    K[S_, S_] = dw * np.eye(m)
    K[S_, Y] = -np.eye(m)
    K[S_, ZLS][jl, np.arange(jl.size)] = -1.0
    K[S_, ZUS][ju, np.arange(ju.size)] = 1.0
    K[Y, X] = A
    K[Y, S_] = -np.eye(m)
    K[Y, Y] = -dc * np.eye(m)
    K[ZLX, X][np.arange(il.size), il] = zlx[il]
    K[ZLX, ZLX] = np.diag(x[il] - xl[il])
    K[ZUX, X][np.arange(iu.size), iu] = -zux[iu]
    K[ZUX, ZUX] = np.diag(xu[iu] - x[iu])
    K[ZLS, S_][np.arange(jl.size), jl] = zls[jl]
    K[ZLS, ZLS] = np.diag(s[jl] - sl[jl])
    K[ZUS, S_][np.arange(ju.size), ju] = -zus[ju]
    K[ZUS, ZUS] = np.diag(su[ju] - s[ju])
    p = np.concatenate([grad - A.T @ y - zlx + zux, -zls + zus + y, c - s,
                        zlx[il] * (x[il] - xl[il]) - mu, zux[iu] * (xu[iu] - x[iu]) - mu,
                        zls[jl] * (s[jl] - sl[jl]) - mu, zus[ju] * (su[ju] - s[ju]) - mu])
    return K, p, (X, S_, Y, ZLX, ZUX, ZLS, ZUS)
