"""Parity over many small seeded random instances: shapes from a single bus to a
few hundred branches, T from 1 to 7, dense chords (parallel branches, high
degrees), off-nominal taps and phase shifts on a random subset of branches,
shunts, generators and loads from none to one per bus, and the reactive ramp
on or off.  Every output of the sweep, the derivative products, the
interior-point algebra and the CSC compression is compared with the oracle bit
for bit (the objective within 1e-12 relative: tree vs sequential sum)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _instance(k):
    rng = np.random.default_rng(300 + k)
    N = int(rng.integers(1, 90))
    L = int(rng.integers(max(N - 1, 0), (N - 1) + 3 * N + 1)) if N > 1 else 0
    G = int(rng.integers(0, N + 2))
    D = int(rng.integers(0, N + 2))
    T = int(rng.integers(1, 8))
    inst = synth.make_instance(400 + k, N, L, G, D, T)
    net = inst.net
    if L:
        sel = rng.uniform(size=L) < 0.3
        net = dataclasses.replace(net, br_tap=np.where(sel, rng.uniform(0.9, 1.1, L), 1.0),
                                  br_shift=np.where(rng.uniform(size=L) < 0.3, rng.uniform(-0.2, 0.2, L), 0.0))
    if G and rng.uniform() < 0.5:
        net = dataclasses.replace(net, gen_qramp=0.2 * np.asarray(net.gen_qmax))
    return synth.Instance(net=net, T=inst.T, pd=inst.pd, qd=inst.qd)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("k", range(24))
def test_random_instance_bitwise(k):
    from paper_2405_14032_b300 import mpopf
    inst = _instance(k)
    o = oracle.Oracle(inst)
    h = mpopf.Handle(inst)
    pt = synth.make_point(500 + k, inst)
    tag = f"instance {k}: N={inst.net.n_bus} L={inst.net.n_branch} G={inst.net.n_gen} T={inst.T}"

    # patterns and the full sweep
    pat = {kk: _np(v) for kk, v in h.pattern().items()}
    jr, jc = o.jac_pattern()
    hr, hc = o.hess_pattern()
    assert np.array_equal(pat["jac_row"], jr) and np.array_equal(pat["jac_col"], jc), tag
    assert np.array_equal(pat["hess_row"], hr) and np.array_equal(pat["hess_col"], hc), tag
    out = h.sweep(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    ref = o.eval(pt.x, pt.lam, pt.sigma)
    rowptr, cols, kv = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    assert np.array_equal(pat["kkt_rowptr"], rowptr) and np.array_equal(pat["kkt_col"], cols), tag
    for key, r in (("grad", ref["g"]), ("c", ref["c"]), ("jv", ref["jv"]), ("hv", ref["hv"]), ("kv", kv)):
        assert np.array_equal(_np(out[key]), r), (tag, key)
    assert abs(_np(out["f"])[0] - ref["f"]) <= 1e-12 * max(abs(ref["f"]), 1e-300), tag

    # derivative products
    rng = np.random.default_rng(600 + k)
    y, v = rng.standard_normal(o.m), rng.standard_normal(o.n)
    gx, gpd, gqd = h.vjp(_dev(pt.x), _dev(y))
    rgx, rgpd, rgqd = o.vjp(pt.x, y)
    assert np.array_equal(_np(gx), rgx) and np.array_equal(_np(gpd), rgpd) and np.array_equal(_np(gqd), rgqd), tag
    assert np.array_equal(_np(h.jvp(_dev(pt.x), _dev(v))), o.jvp(pt.x, v)), tag
    # the same products reading the sweep's J values
    gxs = h.vjp(_dev(pt.x), _dev(y), loads=False, jv=out["jv"])[0]
    assert np.array_equal(_np(gxs), rgx), tag
    assert np.array_equal(_np(h.jvp(_dev(pt.x), _dev(v), jv=out["jv"])), o.jvp(pt.x, v)), tag
    assert np.array_equal(_np(h.hvp(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(v))),
                          o.hvp(pt.x, pt.lam, pt.sigma, v)), tag

    # interior-point algebra
    eps, mu, dw, dc = 1e-2, 0.05, 1e-3, 1e-4
    x, s, yy, zlx, zux, zls, zus, *_ = H.ipm_point(inst, o, 700 + k, eps)
    dz = [_dev(a) for a in (zlx, zux, zls, zus)]
    sigx, dvec, cvec, recip = h.ipm_prepare(_dev(x), _dev(s), *dz, dw, dc, eps)
    rsigx, rdvec, rcvec, _, rrecip = o.ipm_prepare(x, s, zlx, zux, zls, zus, dw, dc, eps)
    for got, want in ((sigx, rsigx), (dvec, rdvec), (cvec, rcvec), (recip, rrecip)):
        assert np.array_equal(_np(got), want), tag
    r = o.eval(x, -yy, 1.0)
    rhs = h.ipm_rhs(_dev(x), _dev(s), _dev(yy), _dev(r["g"]), _dev(r["c"]), recip, dvec, cvec, mu)
    assert np.array_equal(_np(rhs), o.ipm_rhs(x, s, yy, zlx, zux, zls, zus, r["g"], r["c"], mu, dw, dc, eps)[0]), tag
    dx = rng.standard_normal(o.n)
    rec = h.ipm_recover(_dev(x), _dev(s), _dev(yy), *dz, _dev(r["c"]), recip, cvec, _dev(dx), mu, dw, dc)
    rrec = o.ipm_recover(x, s, yy, zlx, zux, zls, zus, r["c"], dx, mu, dw, dc, eps)
    for key, rk in (("ds", "ds"), ("dy", "dy"), ("dzl_x", "dzlx"), ("dzu_x", "dzux"), ("dzl_s", "dzls"),
                    ("dzu_s", "dzus")):
        assert np.array_equal(_np(rec[key]), rrec[rk]), (tag, key)

    # CSC compression of the sweep's J and W
    for which, key in ((mpopf.CSC_JAC, "jv"), (mpopf.CSC_HESS, "hv")):
        cpat = h.csc_pattern(which)
        vals = h.coo_to_csc(which, out[key])
        colptr, rowidx, cref = o.csc(which, _np(out[key]))
        assert np.array_equal(_np(cpat["colptr"]), colptr) and np.array_equal(_np(cpat["rowidx"]), rowidx), tag
        assert np.array_equal(_np(vals), cref), tag
    h.close()
