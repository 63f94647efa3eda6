"""The CUDA path against the mathematics directly, not through the oracle's
operation sequence.

Every other GPU parity test compares the kernels with the oracle bit for bit,
which shows that the two run the same binary64 program.  This file compares
the kernels' outputs with references that share nothing with that program:
the textbook constraint values (C-library sin/cos, no fused operations), the
complex-step derivatives of that textbook c(x) and of the textbook gradient of
the Lagrangian (Jacobian and Hessian columns, exact to rounding for analytic
functions), and the condensed matrix M = W + diag(Sigma_x + delta_w) + J^T D J
(Sec. III-B) formed densely in numpy from those complex-step J and W.  The
tolerances are the rounding error of the compared terms, as in the oracle's
own pins; the networks cover the benchmark shape (cfg1), the reactive ramp
rows, and off-nominal taps and phase shifts (asymmetric branches).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _asymmetric():
    """A 40-bus network with taps on a third and phase shifts on a quarter of
    its branches (the asymmetric branch kernel instantiation), T = 3."""
    inst = synth.make_instance(41, 40, 70, 9, 22, 3)
    rng = np.random.default_rng(41)
    L = inst.net.n_branch
    net = dataclasses.replace(inst.net, br_tap=np.where(rng.uniform(size=L) < 0.33, rng.uniform(0.9, 1.1, L), 1.0),
                              br_shift=np.where(rng.uniform(size=L) < 0.25, rng.uniform(-0.2, 0.2, L), 0.0))
    return synth.Instance(net=net, T=inst.T, pd=inst.pd, qd=inst.qd)


CASES = {
    "cfg1": lambda: synth.config_instance("cfg1"),
    "cfg1_reactive_ramp": lambda: synth.with_reactive_ramp(synth.config_instance("cfg1")),
    "asymmetric_40_bus": _asymmetric,
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    from paper_2405_14032_b300 import mpopf
    inst = CASES[request.param]()
    pt = synth.make_point(11, inst)
    o = oracle.Oracle(inst)
    h = mpopf.Handle(inst)
    out = h.sweep(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    torch.cuda.synchronize()
    out = {k: _np(v) for k, v in out.items()}
    pat = {k: _np(v) for k, v in h.pattern().items()}
    # complex-step Jacobian of the textbook c(x) and Hessian of the textbook
    # Lagrangian, one column per unit vector
    n, m = o.n, o.m
    Jcs = np.empty((m, n))
    Wcs = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Jcs[:, j] = o.cons_cstep(pt.x, e)
        Wcs[:, j] = o.gradlag_cstep(pt.x, pt.lam, pt.sigma, e)
    yield request.param, inst, pt, o, h, out, pat, Jcs, Wcs
    h.close()


def test_objective_and_gradient_from_their_formulas(case):
    name, inst, pt, o, h, out, pat, Jcs, Wcs = case
    f_tb = o.obj_textbook(pt.x)
    assert abs(out["f"][0] - f_tb) <= 1e-13 * abs(f_tb), name
    sl = H.var_slices(inst.net, inst.T)
    pg = pt.x[sl["pg"]].reshape(inst.T, -1)
    g = out["grad"]
    np.testing.assert_allclose(g[sl["pg"]].reshape(inst.T, -1), 2 * inst.net.gen_c2 * pg + inst.net.gen_c1,
                               rtol=1e-15, atol=0)
    rest = np.ones(o.n, bool)
    rest[sl["pg"]] = False
    assert np.all(g[rest] == 0.0), name


def test_constraints_equal_the_textbook_values(case):
    """c(x) from the kernels against the textbook flows and balances (libm
    sin/cos, no fma), to a few ulps of the largest term."""
    name, inst, pt, o, h, out, pat, Jcs, Wcs = case
    c_tb = o.cons_textbook(pt.x)
    scale = max(60.0, 4.0 * np.abs(c_tb).max())
    assert np.abs(out["c"] - c_tb).max() <= 64 * np.spacing(scale), name


def test_jacobian_equals_the_complex_step_derivative(case):
    name, inst, pt, o, h, out, pat, Jcs, Wcs = case
    J = H.dense_jac(pat["jac_row"], pat["jac_col"], out["jv"], o.m, o.n)
    mask = np.zeros_like(J, dtype=bool)
    mask[pat["jac_row"], pat["jac_col"]] = True
    assert np.all(Jcs[~mask] == 0.0), name  # the pattern holds every nonzero derivative
    assert (np.abs(J - Jcs) / (1.0 + np.abs(Jcs))).max() <= 2e-14, name


def test_hessian_equals_the_complex_step_derivative(case):
    name, inst, pt, o, h, out, pat, Jcs, Wcs = case
    hr, hc = pat["hess_row"], pat["hess_col"]
    assert np.all(hr >= hc), name
    W = H.dense_sym(hr, hc, out["hv"], o.n)
    mask = np.zeros_like(W, dtype=bool)
    mask[hr, hc] = True
    mask |= mask.T
    assert np.all(Wcs[~mask] == 0.0), name
    scale = 1.0 + np.abs(Wcs)
    assert (np.abs(W - Wcs) / scale).max() <= 2e-14, name


def test_condensed_matrix_equals_its_definition(case):
    """M = W + diag(Sigma_x + delta_w) + J^T D J with J and W the complex-step
    derivatives, formed densely; the bound is the rounding of the terms plus
    the complex-step derivatives' own error carried through the products."""
    name, inst, pt, o, h, out, pat, Jcs, Wcs = case
    Md = Wcs + np.diag(pt.sigma_x + pt.delta_w) + Jcs.T @ (pt.dvec[:, None] * Jcs)
    aJ = np.abs(Jcs) + 1.0 * (Jcs != 0)
    mag = (np.abs(Wcs) + 1.0 * (Wcs != 0)) + np.diag(pt.sigma_x + pt.delta_w) + aJ.T @ (pt.dvec[:, None] * aJ)
    rowptr, cols = pat["kkt_rowptr"], pat["kkt_col"].astype(np.int64)
    rows = np.repeat(np.arange(o.n), np.diff(rowptr))
    assert np.all(cols <= rows), name
    err = np.abs(out["kv"] - Md[rows, cols])
    assert np.all(err <= 1e-13 * mag[rows, cols]), (name, float((err / mag[rows, cols]).max()))
    # outside the pattern the definition gives exact zeros
    inside = np.zeros((o.n, o.n), bool)
    inside[rows, cols] = True
    inside |= inside.T
    assert np.all(Md[~inside] == 0.0), name


def test_products_equal_the_complex_step_matrices(case):
    """The matrix-free J^T y, J v and W v kernels against the products with the
    complex-step J and W."""
    name, inst, pt, o, h, out, pat, Jcs, Wcs = case
    rng = np.random.default_rng(12)
    y, v = rng.standard_normal(o.m), rng.standard_normal(o.n)
    gx = _np(h.vjp(_dev(pt.x), _dev(y), loads=False)[0])
    mag = (np.abs(Jcs) + 1.0).T @ np.abs(y)
    assert np.all(np.abs(gx - Jcs.T @ y) <= 1e-13 * mag), name
    jv = _np(h.jvp(_dev(pt.x), _dev(v)))
    mag = (np.abs(Jcs) + 1.0) @ np.abs(v)
    assert np.all(np.abs(jv - Jcs @ v) <= 1e-13 * mag), name
    wv = _np(h.hvp(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(v)))
    mag = (np.abs(Wcs) + 1.0) @ np.abs(v)
    assert np.all(np.abs(wv - Wcs @ v) <= 1e-13 * mag), name
