"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test pins one part of the oracle to something other than itself: values
printed in Table II, textbook complex-power flows, closed forms at flat start,
the series-loss identity, invariances of the flow equations, complex-step and
finite-difference derivatives of an independently written textbook c(x), dense
brute force for the condensed matrix, and the C library and exact rational
and high-precision arithmetic for sin/cos.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", params=["cfg1", "cfg1_reactive_ramp"])
def cfg1(request):
    inst = synth.config_instance("cfg1")
    if request.param == "cfg1_reactive_ramp":
        inst = synth.with_reactive_ramp(inst)
    pt = synth.make_point(1, inst)
    o = oracle.Oracle(inst)
    return inst, pt, o


def _parse_rounded(s):
    return float(s[:-1]) * (1e3 if s.endswith("k") else 1e6)


# ---------------------------------------------------------------------------
# Layout counts (Table II)
# ---------------------------------------------------------------------------
def test_table2_counts_match_paper():
    """nvars and ncons of Table II (rounded as printed) come out of the oracle's
    layout for networks of those sizes; the reference row must be counted
    (case118 x 168 gives 268k only with it)."""
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "table2_counts.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for case, N, L, G, T, nv, nc in rows:
        N, L, G, T = int(N), int(L), int(G), int(T)
        net = H.network(N, np.zeros(L, np.int32), np.ones(L, np.int32), np.full(L, 0.01), np.full(L, 0.1),
                        np.zeros(L), gen_bus=np.zeros(G, np.int32), load_bus=[0])
        o = oracle.Oracle(H.instance(net, T, pd=np.zeros(T), qd=np.zeros(T)))
        unit = 1e3 if nv.endswith("k") else 1e6
        assert round(o.n / unit) == _parse_rounded(nv) / unit, (case, T, o.n)
        unit = 1e3 if nc.endswith("k") else 1e6
        assert round(o.m / unit) == _parse_rounded(nc) / unit, (case, T, o.m)
        if case == "case118" and T == 168:
            assert round((o.m - T) / 1e3) != 268  # without the reference row it would read 267k


def test_cfg_sizes():
    o = oracle.Oracle(synth.config_instance("cfg1"))
    assert (o.n, o.m, o.nnz_jac, o.nnz_hess) == (944, 1410, 5248, 2560)


# ---------------------------------------------------------------------------
# Flows
# ---------------------------------------------------------------------------
def _two_bus(tap=1.0, shift=0.0, r=0.02, x=0.08, b=0.03):
    net = H.network(2, [0], [1], [r], [x], [b], gen_bus=[0], load_bus=[1], tap=[tap], shift=[shift])
    return H.instance(net, 1, pd=[0.0], qd=[0.0])


def _flows_from_complex_power(r, x, b, tap, shift, vf, vt, thf, tht):
    """Textbook branch flows from complex power S = V conj(I)."""
    y = 1.0 / complex(r, x)
    Vf = vf * np.exp(1j * thf)
    Vt = vt * np.exp(1j * tht)
    a = tap * np.exp(1j * shift)
    If = (y + 1j * b / 2) / abs(a) ** 2 * Vf - y / np.conj(a) * Vt
    It = -y / a * Vf + (y + 1j * b / 2) * Vt
    Sf = Vf * np.conj(If)
    St = Vt * np.conj(It)
    return Sf.real, Sf.imag, St.real, St.imag


@pytest.mark.parametrize("tap,shift", [(1.0, 0.0), (1.05, 0.0), (0.97, 0.1), (1.0, -0.2)])
def test_two_bus_closed_form(tap, shift):
    inst = _two_bus(tap, shift)
    o = oracle.Oracle(inst)
    sl = H.var_slices(inst.net, 1)
    x = np.zeros(o.n)
    vf, vt, thf, tht = 1.03, 0.98, 0.12, -0.07
    x[sl["va"]] = [thf, tht]
    x[sl["vm"]] = [vf, vt]
    c = o.eval(x, np.zeros(o.m), 1.0)["c"]
    ro = H.row_offsets(inst.net, 1)
    Pf, Qf, Pt, Qt = (-c[ro[k]] for k in (1, 2, 3, 4))  # arc variables are 0
    ePf, eQf, ePt, eQt = _flows_from_complex_power(0.02, 0.08, 0.03, tap, shift, vf, vt, thf, tht)
    for got, exp in ((Pf, ePf), (Qf, eQf), (Pt, ePt), (Qt, eQt)):
        assert abs(got - exp) <= 1e-13 * (1 + abs(exp)), (got, exp)


def test_flat_start(cfg1):
    """vm = 1, va = 0, tau = 1, phi = 0: P_fr = gff + gft = 0 and
    Q_fr = -bff - bft = -b/2 (charging only)."""
    inst, pt, o = cfg1
    net = inst.net
    sl = H.var_slices(net, inst.T)
    x = np.zeros(o.n)
    x[sl["vm"]] = 1.0
    c = o.eval(x, pt.lam, 1.0)["c"]
    ro = H.row_offsets(net, inst.T)
    L = net.n_branch
    for k, expect in ((1, 0.0), (2, net.br_b / 2), (3, 0.0), (4, net.br_b / 2)):
        got = c[ro[k]:ro[k + 1]].reshape(inst.T, L)  # p - P = 0 - P
        np.testing.assert_allclose(got, np.broadcast_to(expect, got.shape), rtol=0, atol=1e-13)


def test_series_loss_identity(cfg1):
    """tau = 1: P_fr + P_to = g |V_f - V_t|^2 and
    Q_fr + Q_to = -b |V_f - V_t|^2 - (b_c/2)(vf^2 + vt^2), y = g + jb."""
    inst, pt, o = cfg1
    net, T, L = inst.net, inst.T, inst.net.n_branch
    sl = H.var_slices(net, T)
    x = pt.x.copy()
    x[sl["p"]] = 0.0
    x[sl["q"]] = 0.0
    c = o.eval(x, pt.lam, 1.0)["c"]
    ro = H.row_offsets(net, T)
    Pf, Qf, Pt, Qt = (-c[ro[k]:ro[k + 1]].reshape(T, L) for k in (1, 2, 3, 4))
    va = x[sl["va"]].reshape(T, -1)
    vm = x[sl["vm"]].reshape(T, -1)
    f, t = net.br_f, net.br_t
    y = 1.0 / (net.br_r + 1j * net.br_x)
    dV2 = np.abs(vm[:, f] * np.exp(1j * va[:, f]) - vm[:, t] * np.exp(1j * va[:, t])) ** 2
    np.testing.assert_allclose(Pf + Pt, y.real * dV2, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(Qf + Qt, -y.imag * dV2 - net.br_b / 2 * (vm[:, f] ** 2 + vm[:, t] ** 2),
                               rtol=1e-11, atol=1e-13)


def test_paper_mutual_term_form(cfg1):
    """Without its self term, the to-end flow is the form printed in Eq. (1d, 1e):
    v_m v_n [G cos(th_n - th_m) + B sin(th_n - th_m)] and
    v_m v_n [G sin(th_n - th_m) - B cos(th_n - th_m)] with G = gtf, B = btf."""
    inst, pt, o = cfg1
    net, T, L = inst.net, inst.T, inst.net.n_branch
    sl = H.var_slices(net, T)
    x = pt.x.copy()
    x[sl["p"]] = 0.0
    x[sl["q"]] = 0.0
    c = o.eval(x, pt.lam, 1.0)["c"]
    ro = H.row_offsets(net, T)
    Pt = -c[ro[3]:ro[4]].reshape(T, L)
    Qt = -c[ro[4]:ro[5]].reshape(T, L)
    gff, bff, gft, bft, gtf, btf, gtt, btt = o.branch_terms()
    va = x[sl["va"]].reshape(T, -1)
    vm = x[sl["vm"]].reshape(T, -1)
    f, t = net.br_f, net.br_t
    d = va[:, t] - va[:, f]
    u = vm[:, f] * vm[:, t]
    np.testing.assert_allclose(Pt - gtt * vm[:, t] ** 2, u * (gtf * np.cos(d) + btf * np.sin(d)), rtol=1e-12,
                               atol=1e-12)
    np.testing.assert_allclose(Qt + btt * vm[:, t] ** 2, u * (gtf * np.sin(d) - btf * np.cos(d)), rtol=1e-12,
                               atol=1e-12)


def test_pi_model_terms_textbook():
    """tau = 1, phi = 0: Y_ff = Y_tt = y + j b/2, Y_ft = Y_tf = -y (exactly)."""
    inst = synth.config_instance("cfg1")
    o = oracle.Oracle(inst)
    gff, bff, gft, bft, gtf, btf, gtt, btt = o.branch_terms()
    y = 1.0 / (inst.net.br_r + 1j * inst.net.br_x)
    np.testing.assert_allclose(gff + 1j * bff, y + 0.5j * inst.net.br_b, rtol=1e-15)
    np.testing.assert_array_equal(gff, gtt)
    np.testing.assert_array_equal(bff, btt)
    np.testing.assert_array_equal(gft, -gff)
    np.testing.assert_array_equal(gtf, gft)
    np.testing.assert_array_equal(bft, btf)


def test_rotation_invariance_and_homogeneity(cfg1):
    """Flows depend on angle differences only, so d/dth_f + d/dth_t = 0 on the
    flow rows and c is unchanged by a common angle shift; flows are degree-2
    homogeneous in (vf, vt): vf dE/dvf + vt dE/dvt = 2E."""
    inst, pt, o = cfg1
    net, T, L = inst.net, inst.T, inst.net.n_branch
    sl = H.var_slices(net, T)
    r = o.eval(pt.x, pt.lam, 1.0)
    jr, jc = o.jac_pattern()
    ro = H.row_offsets(net, T)
    rp = o.jac_rowptr()
    x2 = pt.x.copy()
    x2[sl["va"]] += 0.37
    c2 = o.eval(x2, pt.lam, 1.0)["c"]
    flow = slice(ro[1], ro[5])
    np.testing.assert_allclose(c2[flow], r["c"][flow], rtol=0, atol=5e-14 * 60)
    for k in (1, 2, 3, 4):
        for i in range(ro[k], ro[k + 1]):
            s = rp[i]
            jv = r["jv"][s:s + 5]
            assert jv[1] + jv[2] == 0.0
            tt, l = divmod(i - ro[k], L)
            vf = pt.x[sl["vm"]][tt * net.n_bus + net.br_f[l]]
            vt = pt.x[sl["vm"]][tt * net.n_bus + net.br_t[l]]
            arc = pt.x[jc[s]]
            E = arc - r["c"][i]
            # J = -dE/dv, so vf J_vf + vt J_vt = -2E
            assert abs(vf * jv[3] + vt * jv[4] + 2 * E) <= 1e-13 * (1 + abs(E) + abs(vf * jv[3]) + abs(vt * jv[4]))


def test_balance_constructed_feasible():
    """A point made feasible by hand (arc variables set to the textbook flows,
    one load per bus set to close the balance) has zero flow and balance
    residuals up to rounding."""
    net0 = synth.make_network(11, 40, 64, 9, 0)
    N, T = net0.n_bus, 3
    net = H.network(N, net0.br_f, net0.br_t, net0.br_r, net0.br_x, net0.br_b, gen_bus=net0.gen_bus,
                    load_bus=np.arange(N), gs=np.linspace(0, 0.05, N), bs=np.linspace(0.3, 0, N),
                    ref=net0.ref_bus)
    inst = H.instance(net, T, pd=np.zeros(T * N), qd=np.zeros(T * N))
    o = oracle.Oracle(inst)
    pt = synth.make_point(12, inst)
    x = pt.x.copy()
    sl = H.var_slices(net, T)
    ro = H.row_offsets(net, T)
    L = net.n_branch
    c0 = o.cons_textbook(x)
    # arc p, q := flows (c = arc - E  =>  E = arc - c)
    for k, (var, off) in enumerate((("p", 0), ("q", 0), ("p", L), ("q", L)), start=1):
        E = (x[sl[var]].reshape(T, 2 * L)[:, off:off + L] - c0[ro[k]:ro[k + 1]].reshape(T, L))
        blk = x[sl[var]].reshape(T, 2 * L)
        blk[:, off:off + L] = E
        x[sl[var]] = blk.ravel()
    va = x[sl["va"]].reshape(T, N)
    vm = x[sl["vm"]].reshape(T, N)
    p = x[sl["p"]].reshape(T, 2 * L)
    q = x[sl["q"]].reshape(T, 2 * L)
    pg = x[sl["pg"]].reshape(T, -1)
    qg = x[sl["qg"]].reshape(T, -1)
    arc_bus = np.concatenate([net.br_f, net.br_t])
    pd = np.zeros((T, N))
    qd = np.zeros((T, N))
    for n in range(N):
        gens = np.nonzero(net.gen_bus == n)[0]
        arcs = np.nonzero(arc_bus == n)[0]
        pd[:, n] = pg[:, gens].sum(1) - p[:, arcs].sum(1) - net.bus_gs[n] * vm[:, n] ** 2
        qd[:, n] = qg[:, gens].sum(1) - q[:, arcs].sum(1) + net.bus_bs[n] * vm[:, n] ** 2
    inst2 = H.instance(net, T, pd=pd, qd=qd)
    o2 = oracle.Oracle(inst2)
    c = o2.eval(x, pt.lam, 1.0)["c"]
    scale = 1 + np.abs(x).max() * 20
    assert np.abs(c[ro[1]:ro[5]]).max() <= 1e-14 * scale
    assert np.abs(c[ro[8]:ro[10]]).max() <= 1e-14 * scale
    assert np.array_equal(va, va)  # angles untouched


# ---------------------------------------------------------------------------
# Derivatives: complex step and finite differences of the textbook c(x)
# ---------------------------------------------------------------------------
def _dense_J(o, r):
    jr, jc = o.jac_pattern()
    return H.dense_jac(jr, jc, r["jv"], o.m, o.n), jr, jc


def test_jacobian_complex_step(cfg1):
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, 1.0)
    J, jr, jc = _dense_J(o, r)
    mask = np.zeros_like(J, dtype=bool)
    mask[jr, jc] = True
    worst = 0.0
    for j in range(o.n):
        e = np.zeros(o.n)
        e[j] = 1.0
        col = o.cons_cstep(pt.x, e)
        assert np.all(col[~mask[:, j]] == 0.0), j  # nothing outside the pattern
        err = np.abs(col - J[:, j]) / (1.0 + np.abs(J[:, j]))
        worst = max(worst, err.max())
    assert worst <= 2e-14, worst


def test_jacobian_finite_difference(cfg1):
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, 1.0)
    J, _, _ = _dense_J(o, r)
    h = 1e-6
    rng = np.random.default_rng(0)
    for j in rng.choice(o.n, 80, replace=False):
        xp, xm = pt.x.copy(), pt.x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (o.cons_textbook(xp) - o.cons_textbook(xm)) / (2 * h)
        np.testing.assert_allclose(fd, J[:, j], rtol=1e-7, atol=1e-7)


def test_constraints_match_textbook(cfg1):
    """The rounding-order evaluation equals the textbook expression (C-library
    sin/cos, no fma) to a few ulps of the terms."""
    inst, pt, o = cfg1
    c = o.eval(pt.x, pt.lam, 1.0)["c"]
    ct = o.cons_textbook(pt.x)
    assert np.abs(c - ct).max() <= 64 * np.spacing(60.0)


def test_objective_and_gradient(cfg1):
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, 1.0)
    assert abs(r["f"] - o.obj_textbook(pt.x)) <= 1e-13 * abs(r["f"])
    sl = H.var_slices(inst.net, inst.T)
    pg = pt.x[sl["pg"]].reshape(inst.T, -1)
    np.testing.assert_allclose(r["g"][sl["pg"]].reshape(inst.T, -1), 2 * inst.net.gen_c2 * pg + inst.net.gen_c1,
                               rtol=1e-15)
    g = r["g"].copy()
    g[sl["pg"]] = 0
    assert np.all(g == 0)


def test_hessian_complex_step_and_symmetry(cfg1):
    """Column j of W equals Im(grad L(x + i h e_j)) / h, and the complex-step
    matrix is symmetric (the J formulas are a true gradient)."""
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, pt.sigma)
    hr, hc = o.hess_pattern()
    assert np.all(hr >= hc)
    W = H.dense_sym(hr, hc, r["hv"], o.n)
    Wcs = np.empty((o.n, o.n))
    for j in range(o.n):
        e = np.zeros(o.n)
        e[j] = 1.0
        Wcs[:, j] = o.gradlag_cstep(pt.x, pt.lam, pt.sigma, e)
    scale = 1.0 + np.abs(W)
    assert (np.abs(Wcs - W) / scale).max() <= 2e-14
    assert (np.abs(Wcs - Wcs.T) / scale).max() <= 2e-14
    # outside the pattern, nothing
    mask = np.zeros((o.n, o.n), bool)
    mask[hr, hc] = True
    mask |= mask.T
    assert np.all(Wcs[~mask] == 0.0)


def test_hessian_finite_difference(cfg1):
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, pt.sigma)
    hr, hc = o.hess_pattern()
    W = H.dense_sym(hr, hc, r["hv"], o.n)
    h = 1e-6
    rng = np.random.default_rng(1)
    for j in rng.choice(o.n, 60, replace=False):
        xp, xm = pt.x.copy(), pt.x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (o.gradlag(xp, pt.lam, pt.sigma) - o.gradlag(xm, pt.lam, pt.sigma)) / (2 * h)
        np.testing.assert_allclose(fd, W[:, j], rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------------------
# Condensed matrix
# ---------------------------------------------------------------------------
def test_kkt_dense_brute_force(cfg1):
    """M = W + diag(Sigma_x + delta_w) + J^T D J (dense numpy) and its pattern
    is diag U pattern(W) U {pairs within a J row}."""
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, pt.sigma)
    J, jr, jc = _dense_J(o, r)
    hr, hc = o.hess_pattern()
    W = H.dense_sym(hr, hc, r["hv"], o.n)
    Md = W + np.diag(pt.sigma_x + pt.delta_w) + J.T @ (pt.dvec[:, None] * J)
    mag = np.abs(W) + np.diag(pt.sigma_x + pt.delta_w) + np.abs(J).T @ (pt.dvec[:, None] * np.abs(J))
    rowptr, cols, vals = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    rows = np.repeat(np.arange(o.n), np.diff(rowptr))
    assert np.all(cols <= rows)
    for i in range(o.n):  # sorted, unique, diagonal last
        seg = cols[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(seg) > 0) and seg[-1] == i
    # pattern from the definition
    pat = set(zip(range(o.n), range(o.n)))
    pat |= set(zip(hr.tolist(), hc.tolist()))
    rp = o.jac_rowptr()
    for i in range(o.m):
        cs = jc[rp[i]:rp[i + 1]]
        for a in cs:
            for b in cs:
                if a >= b:
                    pat.add((int(a), int(b)))
    assert pat == set(zip(rows.tolist(), cols.tolist()))
    err = np.abs(vals - Md[rows, cols])
    assert np.all(err <= 4e-16 * 8 * mag[rows, cols] + 1e-300)


def test_kkt_matrix_free_product(cfg1):
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, pt.sigma)
    J, _, _ = _dense_J(o, r)
    hr, hc = o.hess_pattern()
    rowptr, cols, vals = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    Ms = H.csr_to_dense_sym(rowptr, cols, vals, o.n)
    v = np.random.default_rng(2).standard_normal(o.n)
    Wv = o.hvp(pt.x, pt.lam, pt.sigma, v)
    mv = Wv + (pt.sigma_x + pt.delta_w) * v + o.vjp(pt.x, pt.dvec * o.jvp(pt.x, v))[0]
    mag = np.abs(Ms) @ np.abs(v)
    assert np.all(np.abs(Ms @ v - mv) <= 1e-13 * mag)


# ---------------------------------------------------------------------------
# Matrix-free products
# ---------------------------------------------------------------------------
def test_vjp_jvp_hvp(cfg1):
    inst, pt, o = cfg1
    r = o.eval(pt.x, pt.lam, pt.sigma)
    J, _, _ = _dense_J(o, r)
    hr, hc = o.hess_pattern()
    W = H.dense_sym(hr, hc, r["hv"], o.n)
    rng = np.random.default_rng(3)
    y = rng.standard_normal(o.m)
    v = rng.standard_normal(o.n)
    gx, gpd, gqd = o.vjp(pt.x, y)
    jv = o.jvp(pt.x, v)
    hv = o.hvp(pt.x, pt.lam, pt.sigma, v)
    assert np.all(np.abs(gx - J.T @ y) <= 1e-14 * (np.abs(J).T @ np.abs(y)) + 1e-300)
    assert np.all(np.abs(jv - J @ v) <= 1e-14 * (np.abs(J) @ np.abs(v)) + 1e-300)
    assert np.all(np.abs(hv - W @ v) <= 1e-14 * (np.abs(W) @ np.abs(v)) + 1e-300)
    # dot-product test <y, J v> = <J^T y, v>
    assert abs(y @ jv - gx @ v) <= 1e-13 * (np.abs(y) @ (np.abs(J) @ np.abs(v)))
    # load adjoint: dc/dPd = -1 at the P-balance row of the load's bus
    T, N, D = inst.T, inst.net.n_bus, inst.net.n_load
    ro = H.row_offsets(inst.net, T)
    for t in range(T):
        for d in range(D):
            assert gpd[t * D + d] == -y[ro[8] + t * N + inst.net.load_bus[d]]
            assert gqd[t * D + d] == -y[ro[9] + t * N + inst.net.load_bus[d]]


def test_load_adjoint_complex_step():
    """(dc/dPd)^T y by finite change of the loads through the textbook c."""
    inst = synth.make_instance(21, 12, 20, 3, 7, 2)
    o = oracle.Oracle(inst)
    pt = synth.make_point(21, inst)
    y = np.random.default_rng(4).standard_normal(o.m)
    _, gpd, _ = o.vjp(pt.x, y)
    base = o.cons_textbook(pt.x)
    pd = inst.pd.copy()
    pd[1, 3] += 0.5
    o2 = oracle.Oracle(synth.Instance(net=inst.net, T=2, pd=pd, qd=inst.qd))
    dc = (o2.cons_textbook(pt.x) - base) / 0.5
    assert abs(dc @ y - gpd[1 * 7 + 3]) <= 1e-12


def test_hvp_finite_difference(cfg1):
    inst, pt, o = cfg1
    v = np.random.default_rng(5).standard_normal(o.n)
    h = 1e-6
    fd = (o.gradlag(pt.x + h * v, pt.lam, pt.sigma) - o.gradlag(pt.x - h * v, pt.lam, pt.sigma)) / (2 * h)
    np.testing.assert_allclose(o.hvp(pt.x, pt.lam, pt.sigma, v), fd, rtol=1e-6, atol=1e-6)


def test_windowed_outputs_agree_with_full():
    inst = synth.make_instance(31, 25, 40, 5, 10, 6)
    o = oracle.Oracle(inst)
    pt = synth.make_point(31, inst)
    full = o.eval(pt.x, pt.lam, pt.sigma)
    rows, rowlen, cols, vals = o.kkt(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    rowptr = np.concatenate([[0], np.cumsum(rowlen)])
    covered = {k: np.zeros(full[k].size, np.int32) for k in ("g", "c", "jv", "hv")}
    for t0, t1 in ((0, 2), (2, 5), (5, 6)):
        w = o.eval(pt.x, pt.lam, pt.sigma, t0, t1)
        for k in ("g", "c", "jv", "hv"):
            ok = ~np.isnan(w[k])
            assert ok.any()
            assert np.array_equal(w[k][ok], full[k][ok])
            covered[k] += ok
        wr, wl, wc, wv = o.kkt(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w, t0, t1)
        pos = np.concatenate([np.arange(rowptr[r], rowptr[r + 1]) for r in wr])
        assert np.array_equal(cols[pos], wc) and np.array_equal(vals[pos], wv)
        gx, _, _ = o.vjp(pt.x, pt.lam, t0, t1)
        gxf, _, _ = o.vjp(pt.x, pt.lam)
        ok = ~np.isnan(gx)
        assert np.array_equal(gx[ok], gxf[ok])
    # the windows partition the horizon: every entry (the ramp rows of the
    # first period of each window included) is written by exactly one window
    for k, cnt in covered.items():
        assert np.all(cnt == 1), (k, np.nonzero(cnt != 1)[0][:5])


def test_objective_with_constant_cost():
    """f = sum over periods and generators of c2 pg^2 + c1 pg + c0 (Eq. 1a with
    the quadratic cost), written out, with every coefficient nonzero (the
    synthetic networks have c0 = 0)."""
    net = H.network(4, [0, 1, 2], [1, 2, 3], [0.01] * 3, [0.1] * 3, [0.0] * 3, gen_bus=[0, 2, 3], load_bus=[1],
                    c2=[0.02, 0.05, 0.08], c1=[11.0, 17.0, 23.0])
    net.gen_c0[:] = [3.5, -1.25, 7.0]
    T = 3
    o = oracle.Oracle(H.instance(net, T))
    sl = H.var_slices(net, T)
    x = np.zeros(o.n)
    x[sl["pg"]] = [0.5, 1.5, 2.5, 0.25, 1.0, 2.0, 0.75, 1.25, 1.75]
    f = o.eval(x, np.zeros(o.m), 1.0)["f"]
    want = 0.0
    for t in range(T):
        for g in range(3):
            pg = x[sl["pg"].start + t * 3 + g]
            want += net.gen_c2[g] * pg * pg + net.gen_c1[g] * pg + net.gen_c0[g]
    assert abs(f - want) <= 1e-13 * abs(want)


# ---------------------------------------------------------------------------
# sin / cos
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lo,hi", [(-math.pi / 4, math.pi / 4), (-3.0, 3.0), (-1e5, 1e5)])
def test_sincos_against_c_library(lo, hi):
    x = np.random.default_rng(6).uniform(lo, hi, 200000)
    s, c = oracle.sincos(x)
    es = np.abs(s - np.sin(x)) / np.spacing(np.abs(np.sin(x)) + 1e-300)
    ec = np.abs(c - np.cos(x)) / np.spacing(np.abs(np.cos(x)) + 1e-300)
    near_zero = (np.abs(np.sin(x)) < 1e-3) | (np.abs(np.cos(x)) < 1e-3)
    assert es[~near_zero].max() <= 2 and ec[~near_zero].max() <= 2
    assert np.all(np.abs(s - np.sin(x)) <= 4e-16) and np.all(np.abs(c - np.cos(x)) <= 4e-16)
    assert np.abs(s * s + c * c - 1).max() <= 5e-16


def test_sincos_special_values():
    s, c = oracle.sincos(np.array([0.0, -0.0, math.pi / 6, math.pi / 2, 1e-300]))
    # the sign of a zero result is not specified (values compare equal)
    assert s[0] == 0.0 and c[0] == 1.0 and s[1] == 0.0 and c[1] == 1.0
    assert abs(s[2] - 0.5) <= 2 * np.spacing(0.5)
    assert abs(c[3]) <= 1e-16 and s[3] == 1.0
    assert s[4] == 1e-300


# The polynomial coefficients, recomputed here from their definition: the
# Taylor series of (sin r - r)/r^3 through s^7 and of (cos r - 1)/r^2 through
# s^8 (s = r^2), economised with shifted Chebyshev polynomials on [0, 5/8] down
# to degrees 5 and 6, in exact rational arithmetic, then rounded to nearest.
def _economised(coef, degree, a):
    from fractions import Fraction as Fr

    def times(p, q):
        out = [Fr(0)] * (len(p) + len(q) - 1)
        for i, u in enumerate(p):
            for j, w in enumerate(q):
                out[i + j] += u * w
        return out

    y = [Fr(-1), Fr(2) / a]  # maps [0, a] onto [-1, 1]
    cheb = [[Fr(1)], y]
    for k in range(1, len(coef)):
        nxt = times([2 * u for u in y], cheb[k])
        for i, u in enumerate(cheb[k - 1]):
            nxt[i] -= u
        cheb.append(nxt)
    c = list(coef)
    while len(c) - 1 > degree:
        n = len(c) - 1
        f = c[n] / cheb[n][n]
        c = [c[i] - f * cheb[n][i] for i in range(n)]
    return c


def _sincos_polynomials():
    from fractions import Fraction as Fr
    a = Fr(5, 8)
    P = _economised([Fr((-1) ** (k + 1), math.factorial(2 * k + 3)) for k in range(8)], 5, a)
    Q = _economised([Fr((-1) ** (k + 1), math.factorial(2 * k + 2)) for k in range(9)], 6, a)
    return P, Q


def test_sincos_coefficients_are_the_economised_series():
    """Both sincos implementations (the oracle's and the CUDA path's, written
    separately) carry exactly the rounded economised coefficients, and the
    economised polynomials stay within 2e-17 of sin and 1e-18 of cos."""
    import re
    import mpmath as mp
    P, Q = _sincos_polynomials()
    want_p, want_q = [float(c) for c in P], [float(c) for c in Q]
    src = open(oracle._SRC).read()
    got_p = [float.fromhex(re.search(r"kP%d = (-?0x[0-9a-fp.+-]+)" % i, src).group(1)) for i in range(6)]
    got_q = [float.fromhex(re.search(r"kQ%d = (-?0x[0-9a-fp.+-]+)" % i, src).group(1)) for i in range(7)]
    assert got_p == want_p and got_q == want_q
    dev = open(os.path.join(HERE, "..", "paper_2405_14032_b300", "csrc", "mpopf_device.cuh")).read()
    body = dev[dev.index("void sincos_cw"):]
    body = body[:body.index("const double co")]
    lits = [float.fromhex(h) for h in re.findall(r"(-?0x[0-9a-f]\.[0-9a-f]+p[+-]\d+)", body)]
    # after the three Cody-Waite constants and 2/pi: P from the top down, then Q from the top down
    assert lits[4:] == want_p[::-1] + want_q[::-1]
    mp.mp.dps = 40
    es = ec = mp.mpf(0)
    for i in range(801):
        r = mp.mpf(5) / 8 * i / 800
        r = mp.sqrt(r)
        s2 = r * r
        ps = mp.mpf(0)
        for c in reversed(P):
            ps = ps * s2 + mp.mpf(c.numerator) / c.denominator
        qs = mp.mpf(0)
        for c in reversed(Q):
            qs = qs * s2 + mp.mpf(c.numerator) / c.denominator
        es = max(es, abs(r + r ** 3 * ps - mp.sin(r)))
        ec = max(ec, abs(1 + s2 * qs - mp.cos(r)))
    assert es < 2e-17 and ec < 1e-18, (es, ec)


def test_sincos_within_one_ulp_of_high_precision():
    """On the unreduced range (|x| <= pi/4, every angle difference of the
    benchmark inputs) the oracle's sin and cos are within one ulp of the
    correctly rounded values."""
    import mpmath as mp
    mp.mp.dps = 40
    x = np.random.default_rng(7).uniform(-math.pi / 4, math.pi / 4, 3000)
    x = np.concatenate([x, [math.pi / 4 * (1 - 2 ** -52), -0.6, 1e-9, 2.0 ** -30]])
    s, c = oracle.sincos(x)
    for xi, si, ci in zip(x, s, c):
        S, C = mp.sin(mp.mpf(float(xi))), mp.cos(mp.mpf(float(xi)))
        assert abs(mp.mpf(float(si)) - S) <= math.ulp(float(S)), xi
        assert abs(mp.mpf(float(ci)) - C) <= math.ulp(float(C)), xi


def test_jvp_load_tangent_finite_difference():
    """J v with load tangents equals the directional derivative of the
    textbook c(x, Pd, Qd) (linear in the loads: exact up to rounding)."""
    inst = synth.make_instance(22, 12, 20, 3, 7, 3)
    o = oracle.Oracle(inst)
    pt = synth.make_point(22, inst)
    rng = np.random.default_rng(7)
    dpd, dqd = rng.standard_normal(inst.pd.shape), rng.standard_normal(inst.qd.shape)
    zero = np.zeros(o.n)
    got = o.jvp(pt.x, zero, dpd=dpd, dqd=dqd)
    o2 = oracle.Oracle(synth.Instance(net=inst.net, T=inst.T, pd=inst.pd + dpd, qd=inst.qd + dqd))
    want = o2.cons_textbook(pt.x) - o.cons_textbook(pt.x)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    v = rng.standard_normal(o.n)
    both = o.jvp(pt.x, v, dpd=dpd, dqd=dqd)
    np.testing.assert_allclose(both, o.jvp(pt.x, v) + got, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# Interior-point algebra around M (Sec. III-B): pinned by a dense solve of the
# full lifted KKT system of Eq. (5)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dw,dc", [(1e-3, 1e-4), (0.0, 0.0), (0.3, 0.7)])
def test_ipm_condensation_solves_full_lifted_system(dw, dc):
    """Delta x from M_cond dx = q_x + A^T (C q_s + D q_y), with Delta s, Delta y
    and the Delta z recovered from it, solves the full 7-block system of
    Eq. (5) (assembled densely), so the condensation, the right-hand side and
    the recovery formulas are those of the printed block system."""
    inst = synth.make_instance(61, 5, 7, 2, 3, 2)
    o = oracle.Oracle(inst)
    n, m = o.n, o.m
    eps, mu = 1e-2, 0.05
    x, s, y, zlx, zux, zls, zus, xl, xu, sl, su = H.ipm_point(inst, o, 62, eps)
    lam = -y  # W = sigma grad^2 f + sum lam_i grad^2 c_i with the paper's p_x = grad f - J^T y
    r = o.eval(x, lam, 1.0)
    jr, jc = o.jac_pattern()
    A = H.dense_jac(jr, jc, r["jv"], m, n)
    hr, hc = o.hess_pattern()
    W = H.dense_sym(hr, hc, r["hv"], n)
    sigx, dvec, cvec, sigs, recip = o.ipm_prepare(x, s, zlx, zux, zls, zus, dw, dc, eps)
    rowptr, cols, kv = o.kkt_csr(x, lam, 1.0, sigx, dvec, dw)
    Mc = H.csr_to_dense_sym(rowptr, cols, kv, n)
    rhs, _ = o.ipm_rhs(x, s, y, zlx, zux, zls, zus, r["g"], r["c"], mu, dw, dc, eps)
    dx = np.linalg.solve(Mc, rhs)
    rec = o.ipm_recover(x, s, y, zlx, zux, zls, zus, r["c"], dx, mu, dw, dc, eps)
    # full system
    K, p, sl_ = H.lifted_system(W, A, x, s, y, zlx, zux, zls, zus, xl, xu, sl, su, r["g"], r["c"], mu, dw, dc)
    X, S_, Y, ZLX, ZUX, ZLS, ZUS = sl_
    fl, fu, gl_, gu_ = np.isfinite(xl), np.isfinite(xu), np.isfinite(sl), np.isfinite(su)
    il, iu, jl, ju = (np.nonzero(b)[0] for b in (fl, fu, gl_, gu_))
    full = np.linalg.solve(K, p)
    scale = np.abs(full).max()
    np.testing.assert_allclose(dx, full[X], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(rec["ds"], full[S_], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(rec["dy"], full[Y], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(rec["dzlx"][il], full[ZLX], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(rec["dzux"][iu], full[ZUX], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(rec["dzls"][jl], full[ZLS], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(rec["dzus"][ju], full[ZUS], rtol=0, atol=1e-9 * scale)
    assert np.all(rec["dzlx"][~fl] == 0) and np.all(rec["dzus"][~gu_] == 0)
    # The recovery as printed, C (dc q_s - (q_y + A dx)), does not solve Eq. (5);
    # C (A dx + dc q_s - q_y) (eliminating its rows 2 and 3) does (above).
    with np.errstate(invalid="ignore", divide="ignore"):
        qs = (zus - zls) + y + np.where(gl_, (zls * (s - sl) - mu) / (s - sl), 0.0) \
            - np.where(gu_, (zus * (su - s) - mu) / (su - s), 0.0)
    printed = cvec * (dc * qs - ((r["c"] - s) + A @ dx))
    assert np.abs(printed - full[S_]).max() > 1e-3 * scale
    # C and D are the paper's: C = (dc Sigma_s + (1 + dc dw) I)^-1, D = (Sigma_s + dw I) C
    np.testing.assert_allclose(cvec, 1.0 / (dc * sigs + 1.0 + dc * dw), rtol=1e-15)
    np.testing.assert_allclose(dvec, (sigs + dw) * cvec, rtol=1e-15)
    # Sigma = Z (V - VL)^-1 + Z (VU - V)^-1 over finite bounds; the reciprocals
    # are those distances' inverses and 0 for an infinite bound
    with np.errstate(invalid="ignore", divide="ignore"):
        for v, lo, hi, zl, zu, sig, rl, ru in ((x, xl, xu, zlx, zux, sigx, recip[:n], recip[n:2 * n]),
                                              (s, sl, su, zls, zus, sigs, recip[2 * n:2 * n + m],
                                               recip[2 * n + m:])):
            il_, iu_ = np.isfinite(lo), np.isfinite(hi)
            np.testing.assert_allclose(rl[il_], 1.0 / (v - lo)[il_], rtol=2e-16)
            np.testing.assert_allclose(ru[iu_], 1.0 / (hi - v)[iu_], rtol=2e-16)
            assert np.all(rl[~il_] == 0) and np.all(ru[~iu_] == 0)
            ref = np.where(il_, zl / (v - lo), 0.0) + np.where(iu_, zu / (hi - v), 0.0)
            np.testing.assert_allclose(sig, ref, rtol=1e-14)


# ---------------------------------------------------------------------------
# COO -> CSC compression (Sec. III-A): against scipy's conversion and a dense
# reconstruction with duplicates accumulated in COO order
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", [0, 1])
def test_csc_compression_matches_scipy_and_dense(which):
    import scipy.sparse as sp
    for inst in (synth.config_instance("cfg1"), synth.make_instance(63, 40, 70, 9, 20, 3)):
        o = oracle.Oracle(inst)
        r, c = o.jac_pattern() if which == 0 else o.hess_pattern()
        nrows = o.m if which == 0 else o.n
        vals = np.random.default_rng(64).standard_normal(r.size)
        colptr, rowidx, cv = o.csc(which, vals)
        ref = sp.coo_matrix((vals, (r.astype(np.int64), c.astype(np.int64))), shape=(nrows, o.n)).tocsc()
        ref.sum_duplicates()
        ref.sort_indices()
        assert np.array_equal(colptr, ref.indptr) and np.array_equal(rowidx, ref.indices)
        np.testing.assert_allclose(cv, ref.data, rtol=1e-15, atol=1e-15)
        # duplicates summed in COO order, exactly
        dense = np.zeros((nrows, o.n))
        np.add.at(dense, (r, c), vals)
        back = np.zeros((nrows, o.n))
        for j in range(o.n):
            back[rowidx[colptr[j]:colptr[j + 1]], j] = cv[colptr[j]:colptr[j + 1]]
        assert np.array_equal(back, dense)
        if which == 0:
            assert colptr[-1] == r.size  # J has no duplicate (row, col)
        else:
            assert colptr[-1] < r.size and np.all(rowidx >= np.repeat(np.arange(o.n), np.diff(colptr)))
        assert np.all(np.diff(colptr) >= 0)
        for j in range(o.n):
            assert np.all(np.diff(rowidx[colptr[j]:colptr[j + 1]]) > 0)


# ---------------------------------------------------------------------------
# Bounds of the standard form (Eq. 3) from the limits of Eq. 1f-1k
# ---------------------------------------------------------------------------
def _bounds_network(qramp):
    """Three buses, three branches (one parallel pair), three generators on two
    buses; every limit distinct and asymmetric, so that a swapped pair, a
    borrowed limit or a dropped sign changes some bound."""
    net = H.network(3, [0, 1, 0], [1, 2, 1], [0.01, 0.02, 0.03], [0.1, 0.12, 0.15], [0.01, 0.02, 0.0],
                    gen_bus=[0, 2, 2], load_bus=[1, 2], ref=1)
    net.bus_vmin[:] = [0.91, 0.93, 0.95]
    net.bus_vmax[:] = [1.07, 1.08, 1.09]
    net.br_angmin[:] = [-0.41, -0.52, -0.23]
    net.br_angmax[:] = [0.37, 0.28, 0.19]
    net.gen_pmin[:] = [0.1, 0.25, 0.0]
    net.gen_pmax[:] = [2.5, 3.5, 1.5]
    net.gen_qmin[:] = [-0.4, -0.9, -0.2]
    net.gen_qmax[:] = [0.7, 1.1, 0.6]
    net.gen_ramp[:] = [0.31, 0.47, 0.13]
    if qramp:
        net.gen_qramp = np.array([0.17, 0.29, 0.05])
    return net


@pytest.mark.parametrize("qramp", [False, True])
@pytest.mark.parametrize("T", [1, 2, 3])
def test_bounds_written_out_from_the_model(qramp, T):
    """xl/xu/gl/gu row by row from the model, written out independently of the
    oracle: vm in [vmin, vmax] (Eq. 1i), pg in [pmin, pmax] (Eq. 1g), qg in
    [qmin, qmax] (Eq. 1h), va, p, q free; the reference row, the four flow
    definitions and both balances are equalities (0, 0); the angle difference
    in [angmin, angmax] (Eq. 1j); the squared thermal rows at both ends in
    (-inf, 0] (Eq. 1f); the P ramp in [-ramp, ramp] for t >= 1 (Eq. 1k); the
    reactive ramp, when present, in [-qramp, qramp]."""
    net = _bounds_network(qramp)
    N, L, G = net.n_bus, net.n_branch, net.n_gen
    o = oracle.Oracle(H.instance(net, T))
    xl, xu, gl, gu = o.bounds()
    inf = math.inf
    exl, exu = [], []
    for _ in range(T):                       # va
        exl += [-inf] * N; exu += [inf] * N
    for _ in range(T):                       # vm
        exl += list(net.bus_vmin); exu += list(net.bus_vmax)
    for _ in range(T):                       # pg
        exl += list(net.gen_pmin); exu += list(net.gen_pmax)
    for _ in range(T):                       # qg
        exl += list(net.gen_qmin); exu += list(net.gen_qmax)
    for _ in range(2 * T):                   # p, q of both arcs of every branch
        exl += [-inf] * (2 * L); exu += [inf] * (2 * L)
    egl, egu = [0.0] * T, [0.0] * T          # K0 reference angle
    for _ in range(4 * T):                   # K1..K4 flow definitions
        egl += [0.0] * L; egu += [0.0] * L
    for _ in range(T):                       # K5 angle difference
        egl += list(net.br_angmin); egu += list(net.br_angmax)
    for _ in range(2 * T):                   # K6, K7 thermal
        egl += [-inf] * L; egu += [0.0] * L
    for _ in range(2 * T):                   # K8, K9 balances
        egl += [0.0] * N; egu += [0.0] * N
    for _ in range(T - 1):                   # K10 ramp, t = 1 .. T-1
        egl += [-r for r in net.gen_ramp]; egu += list(net.gen_ramp)
    if qramp:
        for _ in range(T - 1):               # K11 reactive ramp
            egl += [-r for r in net.gen_qramp]; egu += list(net.gen_qramp)
    assert (o.n, o.m) == (len(exl), len(egl))
    for got, exp in ((xl, exl), (xu, exu), (gl, egl), (gu, egu)):
        assert np.array_equal(got, np.array(exp)), np.nonzero(got != np.array(exp))[0][:8]
    assert G == 3


def test_bounds_match_the_network_arrays_cfg1():
    """The same statement on cfg1 (with and without the reactive ramp), checked
    by kind blocks against the network arrays."""
    for qramp in (False, True):
        inst = synth.config_instance("cfg1")
        if qramp:
            inst = synth.with_reactive_ramp(inst)
        net, T = inst.net, inst.T
        o = oracle.Oracle(inst)
        xl, xu, gl, gu = o.bounds()
        sl = H.var_slices(net, T)
        assert np.all(xl[sl["va"]] == -np.inf) and np.all(xu[sl["va"]] == np.inf)
        assert np.array_equal(xl[sl["vm"]], np.tile(net.bus_vmin, T))
        assert np.array_equal(xu[sl["vm"]], np.tile(net.bus_vmax, T))
        assert np.array_equal(xl[sl["pg"]], np.tile(net.gen_pmin, T))
        assert np.array_equal(xu[sl["pg"]], np.tile(net.gen_pmax, T))
        assert np.array_equal(xl[sl["qg"]], np.tile(net.gen_qmin, T))
        assert np.array_equal(xu[sl["qg"]], np.tile(net.gen_qmax, T))
        for k in ("p", "q"):
            assert np.all(xl[sl[k]] == -np.inf) and np.all(xu[sl[k]] == np.inf)
        ro = H.row_offsets(net, T)
        eq = np.r_[ro[0]:ro[5], ro[8]:ro[10]]
        assert np.all(gl[eq] == 0.0) and np.all(gu[eq] == 0.0)
        assert np.array_equal(gl[ro[5]:ro[6]], np.tile(net.br_angmin, T))
        assert np.array_equal(gu[ro[5]:ro[6]], np.tile(net.br_angmax, T))
        assert np.all(gl[ro[6]:ro[8]] == -np.inf) and np.all(gu[ro[6]:ro[8]] == 0.0)
        assert np.array_equal(gl[ro[10]:ro[11]], np.tile(-net.gen_ramp, T - 1))
        assert np.array_equal(gu[ro[10]:ro[11]], np.tile(net.gen_ramp, T - 1))
        if qramp:
            assert o.m == ro[11] + (T - 1) * net.n_gen
            assert np.array_equal(gl[ro[11]:], np.tile(-net.gen_qramp, T - 1))
            assert np.array_equal(gu[ro[11]:], np.tile(net.gen_qramp, T - 1))
        else:
            assert o.m == ro[11]
