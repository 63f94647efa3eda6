"""Seeded synthetic multi-period AC OPF instances (inputs only).

This module draws inputs and nothing else: network topology and parameters,
per-period load profiles and evaluation points (x, lambda, Sigma_x, D).  It
holds none of the method's arithmetic (no admittances, flows, derivatives or
assembly), so both the CPU oracle and the CUDA path can be fed from it.

Recipe (the paper's workloads are IEEE/PEGASE cases with sinusoid-perturbed
loads, Sec. IV and Table II; those files are not available, so these seeded
networks stand in with the same shape):

* topology: random recursive spanning tree (bus i attaches to a uniform bus
  in 0..i-1), then random chords (no self-loops, parallel lines allowed),
  random orientation of every branch, random branch order, random bus
  relabelling; the reference bus is the relabelled root;
* branches: r ~ U[0.005, 0.05], x ~ U[0.02, 0.2], b ~ U[0, 0.05],
  smax ~ U[0.5, 2], tap 1, shift 0, angle limits +-pi/6;
* buses: v in [0.9, 1.1]; 10% of buses carry a shunt gs ~ U[0, 0.05],
  bs ~ U[0, 0.3];
* generators at uniform buses (with replacement): c2 ~ U[0.01, 0.1],
  c1 ~ U[10, 40], c0 = 0, Pmin = 0, Pmax ~ U[1, 5], Qmax = -Qmin = Pmax/2,
  ramp = Pmax/5;
* loads at uniform buses: Pd0 ~ U[0.2, 1], Qd0 = Pd0 U[0.1, 0.3];
  Pd[t] = Pd0 (1 + 0.2 sin(2 pi t / 24)) (1 + 0.05 eps), eps ~ N(0, 1)
  per (t, d), and likewise for Qd with an independent eps (Sec. IV:
  random perturbation of a scaled periodic function);
* evaluation point: vm ~ U[0.95, 1.05], va ~ U[-0.3, 0.3],
  pg ~ U[Pmin, Pmax], qg ~ U[Qmin, Qmax], arc p, q ~ U[-2, 2];
  lambda ~ U[-1, 1], sigma = 1, Sigma_x, D ~ logU[1e-6, 1e6], delta_w = 1e-8.

Random numbers: a counter-based splitmix64 generator.  Stream s of seed k
yields mix(key + (i + 1) * 0x9E3779B97F4A7C15) for i = 0, 1, ..., with
key = mix(k * 0x9E3779B97F4A7C15 + s) and mix the splitmix64 finaliser
(Steele, Lea and Flood, OOPSLA 2014).  Uniforms take the top 53 bits.
Each quantity has its own stream id, so adding draws never shifts others.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _bits(seed: int, stream: int, count: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed], dtype=np.uint64) * _GOLDEN + np.uint64(stream))[0]
        ctr = np.arange(1, count + 1, dtype=np.uint64) * _GOLDEN + key
        return _mix(ctr)


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    u = (_bits(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Box-Muller on two uniform streams (stream, stream + 1)."""
    u1 = 1.0 - uniform(seed, stream, count)          # (0, 1]
    u2 = uniform(seed, stream + 1, count)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def log_uniform(seed: int, stream: int, count: int, lo: float, hi: float) -> np.ndarray:
    return 10.0 ** uniform(seed, stream, count, math.log10(lo), math.log10(hi))


def randint(seed: int, stream: int, count: int, upper) -> np.ndarray:
    """floor(u * upper) for a scalar or per-draw upper bound (exclusive)."""
    u = uniform(seed, stream, count)
    return np.minimum(np.floor(u * upper), np.asarray(upper) - 1).astype(np.int64)


@dataclasses.dataclass
class Network:
    """Host arrays of one network (0-based int32 indices, FP64 values)."""
    n_bus: int
    n_branch: int
    n_gen: int
    n_load: int
    ref_bus: int
    bus_gs: np.ndarray
    bus_bs: np.ndarray
    bus_vmin: np.ndarray
    bus_vmax: np.ndarray
    br_f: np.ndarray
    br_t: np.ndarray
    br_r: np.ndarray
    br_x: np.ndarray
    br_b: np.ndarray
    br_tap: np.ndarray
    br_shift: np.ndarray
    br_smax: np.ndarray
    br_angmin: np.ndarray
    br_angmax: np.ndarray
    gen_bus: np.ndarray
    gen_c2: np.ndarray
    gen_c1: np.ndarray
    gen_c0: np.ndarray
    gen_pmin: np.ndarray
    gen_pmax: np.ndarray
    gen_qmin: np.ndarray
    gen_qmax: np.ndarray
    gen_ramp: np.ndarray
    load_bus: np.ndarray
    gen_qramp: np.ndarray | None = None  # reactive ramp limits [G]; None: no reactive ramp rows


@dataclasses.dataclass
class Instance:
    net: Network
    T: int
    pd: np.ndarray  # [T][D]
    qd: np.ndarray  # [T][D]


# Stream ids (one per drawn quantity).
_S_PARENT, _S_CHORD_A, _S_CHORD_B, _S_ORIENT, _S_BR_PERM, _S_BUS_PERM = 1, 2, 3, 4, 5, 6
_S_R, _S_X, _S_B, _S_SMAX = 10, 11, 12, 13
_S_SHUNT, _S_GS, _S_BS = 20, 21, 22
_S_GBUS, _S_C2, _S_C1, _S_PMAX = 30, 31, 32, 33
_S_LBUS, _S_PD0, _S_QFRAC, _S_EPS_P, _S_EPS_Q = 40, 41, 42, 44, 46
_S_VA, _S_VM, _S_PG, _S_QG, _S_P, _S_Q = 60, 61, 62, 63, 64, 65
_S_LAM, _S_SIGX, _S_D = 70, 71, 72
_S_PERTURB = 1000


def make_network(seed: int, n_bus: int, n_branch: int, n_gen: int, n_load: int) -> Network:
    N, L, G, D = int(n_bus), int(n_branch), int(n_gen), int(n_load)
    if N < 1 or L < N - 1:
        raise ValueError("need N >= 1 and L >= N - 1 for a spanning tree")
    # Spanning tree: bus i (1..N-1) attaches to a uniform earlier bus.
    child = np.arange(1, N, dtype=np.int64)
    parent = randint(seed, _S_PARENT, N - 1, child) if N > 1 else np.zeros(0, np.int64)
    nc = L - (N - 1)
    ca = randint(seed, _S_CHORD_A, nc, N) if nc else np.zeros(0, np.int64)
    cb = randint(seed, _S_CHORD_B, nc, max(N - 1, 1)) if nc else np.zeros(0, np.int64)
    cb = np.where(cb >= ca, cb + 1, cb)          # cb != ca
    if nc and N < 2:
        raise ValueError("chords need at least two buses")
    ends_a = np.concatenate([parent, ca])
    ends_b = np.concatenate([child, cb])
    flip = uniform(seed, _S_ORIENT, L) < 0.5
    f_old = np.where(flip, ends_b, ends_a)
    t_old = np.where(flip, ends_a, ends_b)
    border = np.argsort(_bits(seed, _S_BR_PERM, L), kind="stable")
    f_old, t_old = f_old[border], t_old[border]
    # Bus relabelling: new label of old bus i is the rank of its key.
    relabel = np.empty(N, np.int64)
    relabel[np.argsort(_bits(seed, _S_BUS_PERM, N), kind="stable")] = np.arange(N)
    br_f = relabel[f_old].astype(np.int32)
    br_t = relabel[t_old].astype(np.int32)
    ref = int(relabel[0])

    shunt = uniform(seed, _S_SHUNT, N) < 0.1
    gs = np.where(shunt, uniform(seed, _S_GS, N, 0.0, 0.05), 0.0)
    bs = np.where(shunt, uniform(seed, _S_BS, N, 0.0, 0.3), 0.0)

    pmax = uniform(seed, _S_PMAX, G, 1.0, 5.0)
    qmax = 0.5 * pmax
    return Network(
        n_bus=N, n_branch=L, n_gen=G, n_load=D, ref_bus=ref,
        bus_gs=gs, bus_bs=bs, bus_vmin=np.full(N, 0.9), bus_vmax=np.full(N, 1.1),
        br_f=br_f, br_t=br_t,
        br_r=uniform(seed, _S_R, L, 0.005, 0.05), br_x=uniform(seed, _S_X, L, 0.02, 0.2),
        br_b=uniform(seed, _S_B, L, 0.0, 0.05), br_tap=np.ones(L), br_shift=np.zeros(L),
        br_smax=uniform(seed, _S_SMAX, L, 0.5, 2.0),
        br_angmin=np.full(L, -math.pi / 6), br_angmax=np.full(L, math.pi / 6),
        gen_bus=randint(seed, _S_GBUS, G, N).astype(np.int32),
        gen_c2=uniform(seed, _S_C2, G, 0.01, 0.1), gen_c1=uniform(seed, _S_C1, G, 10.0, 40.0),
        gen_c0=np.zeros(G), gen_pmin=np.zeros(G), gen_pmax=pmax,
        gen_qmin=-qmax, gen_qmax=qmax, gen_ramp=0.2 * pmax,
        load_bus=randint(seed, _S_LBUS, D, N).astype(np.int32),
    )


def make_loads(seed: int, net: Network, T: int) -> tuple[np.ndarray, np.ndarray]:
    D = net.n_load
    pd0 = uniform(seed, _S_PD0, D, 0.2, 1.0)
    qd0 = pd0 * uniform(seed, _S_QFRAC, D, 0.1, 0.3)
    t = np.arange(T, dtype=np.float64)[:, None]
    shape = 1.0 + 0.2 * np.sin(2.0 * math.pi * t / 24.0)
    eps_p = normal(seed, _S_EPS_P, T * D).reshape(T, D)
    eps_q = normal(seed, _S_EPS_Q, T * D).reshape(T, D)
    pd = pd0[None, :] * shape * (1.0 + 0.05 * eps_p)
    qd = qd0[None, :] * shape * (1.0 + 0.05 * eps_q)
    return np.ascontiguousarray(pd), np.ascontiguousarray(qd)


def make_instance(seed: int, n_bus: int, n_branch: int, n_gen: int, n_load: int, T: int) -> Instance:
    net = make_network(seed, n_bus, n_branch, n_gen, n_load)
    pd, qd = make_loads(seed, net, T)
    return Instance(net=net, T=int(T), pd=pd, qd=qd)


def with_reactive_ramp(inst: Instance, frac: float = 0.2) -> Instance:
    """The same instance with reactive ramp limits Q_ramp = frac * Qmax (the
    counterpart of the real ramp limits 0.2 * Pmax)."""
    net = dataclasses.replace(inst.net, gen_qramp=frac * np.asarray(inst.net.gen_qmax, np.float64))
    return Instance(net=net, T=inst.T, pd=inst.pd, qd=inst.qd)


def sizes(net: Network, T: int) -> tuple[int, int]:
    """(n, m): variables T(2N + 2G + 4L) and constraints T(1 + 7L + 2N) + G(T - 1),
    plus G(T - 1) reactive ramp rows when the network has them.

    Interface sizes only (the variable and row counts of the model, Table II),
    so that evaluation vectors of the right length can be drawn.
    """
    N, L, G = net.n_bus, net.n_branch, net.n_gen
    ramps = 2 if net.gen_qramp is not None else 1
    return T * (2 * N + 2 * G + 4 * L), T * (1 + 7 * L + 2 * N) + ramps * G * (T - 1)


@dataclasses.dataclass
class Point:
    x: np.ndarray        # [n] in the variable order va, vm, pg, qg, p, q (kind, period, component)
    lam: np.ndarray      # [m]
    sigma: float
    sigma_x: np.ndarray  # [n]
    dvec: np.ndarray     # [m]
    delta_w: float


def make_point(seed: int, inst: Instance, stream_offset: int = 0) -> Point:
    net, T = inst.net, inst.T
    N, L, G = net.n_bus, net.n_branch, net.n_gen
    n, m = sizes(net, T)
    s = stream_offset
    va = uniform(seed, s + _S_VA, T * N, -0.3, 0.3)
    vm = uniform(seed, s + _S_VM, T * N, 0.95, 1.05)
    ug = uniform(seed, s + _S_PG, T * G).reshape(T, G)
    pg = (net.gen_pmin[None, :] + (net.gen_pmax - net.gen_pmin)[None, :] * ug).ravel()
    uq = uniform(seed, s + _S_QG, T * G).reshape(T, G)
    qg = (net.gen_qmin[None, :] + (net.gen_qmax - net.gen_qmin)[None, :] * uq).ravel()
    p = uniform(seed, s + _S_P, T * 2 * L, -2.0, 2.0)
    q = uniform(seed, s + _S_Q, T * 2 * L, -2.0, 2.0)
    x = np.concatenate([va, vm, pg, qg, p, q])
    assert x.shape[0] == n
    return Point(
        x=x,
        lam=uniform(seed, s + _S_LAM, m, -1.0, 1.0),
        sigma=1.0,
        sigma_x=log_uniform(seed, s + _S_SIGX, n, 1e-6, 1e6),
        dvec=log_uniform(seed, s + _S_D, m, 1e-6, 1e6),
        delta_w=1e-8,
    )


def perturb(seed: int, x: np.ndarray, k: int, scale: float = 1e-3) -> np.ndarray:
    """Iterate k of a sweep sequence: x + scale N(0, 1)."""
    return x + scale * normal(seed, _S_PERTURB + 2 * k, x.shape[0])


# The five workloads (N, L, G, D, T, seed).
CONFIGS = {
    "cfg1": dict(n_bus=30, n_branch=41, n_gen=6, n_load=20, T=4, seed=1),
    "cfg2": dict(n_bus=2000, n_branch=3200, n_gen=400, n_load=1200, T=24, seed=2),
    "cfg3": dict(n_bus=10000, n_branch=16000, n_gen=2000, n_load=6000, T=168, seed=3),
}


def config_instance(name: str) -> Instance:
    c = CONFIGS[name]
    return make_instance(c["seed"], c["n_bus"], c["n_branch"], c["n_gen"], c["n_load"], c["T"])


def batch_shapes(count: int = 64, seed: int = 1000) -> list[dict]:
    """Uneven instances: N log-uniform in [500, 5000], L = round(1.6 N),
    G = round(0.2 N), D = round(0.6 N), T uniform in {12, 24, 48, 96}.
    Instance k uses seed 1000 + k for its own network."""
    nb = np.round(log_uniform(seed, 1, count, 500.0, 5000.0)).astype(np.int64)
    tt = np.array([12, 24, 48, 96])[randint(seed, 2, count, 4)]
    out = []
    for k in range(count):
        N = int(nb[k])
        out.append(dict(n_bus=N, n_branch=int(round(1.6 * N)), n_gen=int(round(0.2 * N)),
                        n_load=int(round(0.6 * N)), T=int(tt[k]), seed=seed + k))
    return out
