"""Matrix-free derivative products on the GPU (J^T y with the load adjoint,
J v with load tangents, W v) and their autograd wrappers.

Parity: the kernels against the oracle's element-order products on the same
seeded inputs (tolerance |gpu - ref| <= max(1e-12 |ref|, 1e-14); bitwise in
practice).  Independent checks: central finite differences (h = 1e-6) of the
GPU's own c(x) and grad L(x), the dot-product identity, and torch's gradcheck
and gradgradcheck through the autograd.Function.
"""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H
from tests.test_gpu_parity import _edge_network, assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


CASES = {
    "cfg1": lambda: (synth.config_instance("cfg1"), 1),
    "edge_T5": lambda: (H.instance(_edge_network(), 5), 43),
    "ragged_T3": lambda: (synth.make_instance(41, 333, 530, 67, 200, 3), 41),
    "single_bus": lambda: (H.instance(H.network(1, [], [], [], [], [], gen_bus=[0, 0], load_bus=[0]), 3), 44),
    "qramp_T4": lambda: (synth.with_reactive_ramp(synth.make_instance(50, 120, 190, 25, 70, 4)), 50),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    from paper_2405_14032_b300 import mpopf
    inst, seed = CASES[request.param]()
    return request.param, inst, synth.make_point(seed, inst), mpopf.Handle(inst), oracle.Oracle(inst)


def test_products_match_oracle(case):
    name, inst, pt, h, o = case
    rng = np.random.default_rng(11)
    y = rng.standard_normal(o.m)
    v = rng.standard_normal(o.n)
    T, D = inst.T, inst.net.n_load
    dpd, dqd = rng.standard_normal(T * D), rng.standard_normal(T * D)
    gx, gpd, gqd = h.vjp(_dev(pt.x), _dev(y))
    rgx, rgpd, rgqd = o.vjp(pt.x, y)
    assert_close(f"{name}:vjp", _np(gx), rgx)
    assert np.array_equal(_np(gpd), rgpd) and np.array_equal(_np(gqd), rgqd)
    jv = h.jvp(_dev(pt.x), _dev(v))
    assert_close(f"{name}:jvp", _np(jv), o.jvp(pt.x, v))
    if D:
        jvl = h.jvp(_dev(pt.x), _dev(v), dpd=_dev(dpd), dqd=_dev(dqd))
        assert_close(f"{name}:jvp_loads", _np(jvl), o.jvp(pt.x, v, dpd=dpd, dqd=dqd))
    hv = h.hvp(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(v))
    assert_close(f"{name}:hvp", _np(hv), o.hvp(pt.x, pt.lam, pt.sigma, v))


def test_products_from_stored_jacobian(case):
    """With J's values from the sweep at the same x, J^T y and J v read them
    instead of recomputing the branch rows: bit for bit the same results."""
    from paper_2405_14032_b300 import mpopf
    name, inst, pt, h, o = case
    rng = np.random.default_rng(15)
    y, v = rng.standard_normal(o.m), rng.standard_normal(o.n)
    xd = _dev(pt.x)
    jv = h.eval(mpopf.OUT_JAC, xd)["jv"]
    gx, gpd, gqd = h.vjp(xd, _dev(y), jv=jv)
    rgx, rgpd, rgqd = o.vjp(pt.x, y)
    assert np.array_equal(_np(gx), rgx) and np.array_equal(_np(gpd), rgpd) and np.array_equal(_np(gqd), rgqd)
    assert np.array_equal(_np(h.jvp(xd, _dev(v), jv=jv)), o.jvp(pt.x, v))
    if inst.net.n_load:
        T, D = inst.T, inst.net.n_load
        dpd, dqd = rng.standard_normal(T * D), rng.standard_normal(T * D)
        assert np.array_equal(_np(h.jvp(xd, _dev(v), dpd=_dev(dpd), dqd=_dev(dqd), jv=jv)),
                              o.jvp(pt.x, v, dpd=dpd, dqd=dqd))


def test_dot_product_identity(case):
    name, inst, pt, h, o = case
    rng = np.random.default_rng(12)
    y, v = rng.standard_normal(o.m), rng.standard_normal(o.n)
    gx = _np(h.vjp(_dev(pt.x), _dev(y), loads=False)[0])
    jv = _np(h.jvp(_dev(pt.x), _dev(v)))
    mag = np.abs(y) @ np.abs(jv) + np.abs(gx) @ np.abs(v)
    assert abs(y @ jv - gx @ v) <= 1e-13 * mag


def test_finite_differences_of_gpu_callbacks(case):
    """J v and W v against central differences of the GPU's own c(x) and
    grad L(x) = sigma grad f + J^T lambda."""
    from paper_2405_14032_b300 import mpopf
    name, inst, pt, h, o = case
    rng = np.random.default_rng(13)
    v = rng.standard_normal(o.n)
    eps = 1e-6
    xp, xm = _dev(pt.x + eps * v), _dev(pt.x - eps * v)
    fd = (_np(h.eval(mpopf.OUT_CONS, xp)["c"]) - _np(h.eval(mpopf.OUT_CONS, xm)["c"])) / (2 * eps)
    jv = _np(h.jvp(_dev(pt.x), _dev(v)))
    np.testing.assert_allclose(jv, fd, rtol=1e-6, atol=1e-6)
    lam = _dev(pt.lam)

    def gradL(x):
        g = h.eval(mpopf.OUT_GRAD, x)["grad"]
        return pt.sigma * _np(g) + _np(h.vjp(x, lam, loads=False)[0])

    fd2 = (gradL(xp) - gradL(xm)) / (2 * eps)
    hv = _np(h.hvp(_dev(pt.x), lam, pt.sigma, _dev(v)))
    np.testing.assert_allclose(hv, fd2, rtol=1e-6, atol=1e-6)


def test_autograd_gradcheck_small():
    from paper_2405_14032_b300 import autograd as ag
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(51, 6, 8, 2, 3, 2)
    h = mpopf.Handle(inst)
    pt = synth.make_point(51, inst)
    x = _dev(pt.x).requires_grad_(True)
    pd = _dev(inst.pd).requires_grad_(True)
    qd = _dev(inst.qd).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b, c: ag.constraints(h, a, b, c), (x, pd, qd), eps=1e-6, atol=1e-6,
                                    rtol=1e-5)
    assert torch.autograd.gradgradcheck(lambda a, b, c: ag.constraints(h, a, b, c), (x, pd, qd), eps=1e-6,
                                        atol=1e-5, rtol=1e-4)
    assert torch.autograd.gradcheck(lambda a: ag.objective(h, a), (x,), eps=1e-6, atol=1e-6, rtol=1e-5)
    assert torch.autograd.gradgradcheck(lambda a: ag.objective(h, a), (x,), eps=1e-6, atol=1e-5, rtol=1e-4)


def test_autograd_matches_oracle_products():
    """Backward of a scalar loss through constraints() gives the oracle's
    J^T y and load adjoint; the Hessian-vector product through double
    backward gives the oracle's W v (lambda = y, sigma = 0)."""
    from paper_2405_14032_b300 import autograd as ag
    from paper_2405_14032_b300 import mpopf
    inst = synth.config_instance("cfg1")
    h = mpopf.Handle(inst)
    o = oracle.Oracle(inst)
    pt = synth.make_point(1, inst)
    rng = np.random.default_rng(14)
    y, v = rng.standard_normal(o.m), rng.standard_normal(o.n)
    x = _dev(pt.x).requires_grad_(True)
    pd, qd = _dev(inst.pd).requires_grad_(True), _dev(inst.qd).requires_grad_(True)
    c = ag.constraints(h, x, pd, qd)
    (gx,) = torch.autograd.grad((c * _dev(y)).sum(), x, create_graph=True)
    rgx, rgpd, _ = o.vjp(pt.x, y)
    assert_close("autograd:vjp", _np(gx), rgx)
    (hv,) = torch.autograd.grad((gx * _dev(v)).sum(), x)
    assert_close("autograd:hvp", _np(hv), o.hvp(pt.x, y, 0.0, v))
    c = ag.constraints(h, x, pd, qd)
    (gpd,) = torch.autograd.grad((c * _dev(y)).sum(), pd)
    assert np.array_equal(_np(gpd).ravel(), rgpd)


def test_diff_config_256_vectors_sampled():
    """The differentiation workload (2,000-bus network, T = 24, seed 5): 16 of
    its 256 (y, v) vectors checked against the oracle."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(5, 2000, 3200, 400, 1200, 24)
    h = mpopf.Handle(inst)
    o = oracle.Oracle(inst)
    pt = synth.make_point(5, inst)
    xd, lamd = _dev(pt.x), _dev(pt.lam)
    for k in range(0, 256, 16):
        y = synth.uniform(5, 5000 + k, o.m, -1.0, 1.0)
        v = synth.normal(5, 9000 + 2 * k, o.n)
        assert_close(f"diff:vjp{k}", _np(h.vjp(xd, _dev(y), loads=False)[0]), o.vjp(pt.x, y)[0])
        assert_close(f"diff:hvp{k}", _np(h.hvp(xd, lamd, pt.sigma, _dev(v))), o.hvp(pt.x, pt.lam, pt.sigma, v))
