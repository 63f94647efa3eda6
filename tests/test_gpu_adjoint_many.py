"""Derivative products for many vectors at one point (mpopf_vjp_many,
mpopf_jvp_many, mpopf_hvp_many): each vector's result equals the single
product's bit for bit, with the branch rows recomputed or read from the stored
J / W; the first vector's results equal the oracle's element-order products;
the 256-vector differentiation workload (2,000 buses x 24) is checked against
the single products on sampled vectors and against the oracle on two."""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H
from tests.test_gpu_adjoint import CASES
from tests.test_gpu_parity import assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MANY_CASES = dict(CASES)
MANY_CASES["no_gens_no_loads"] = lambda: (H.instance(H.network(
    5, [0, 1, 2, 3], [1, 2, 3, 4], [0.01] * 4, [0.1] * 4, [0.02] * 4, ref=2), 2, pd=np.zeros(0), qd=np.zeros(0)), 45)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _check_many(h, inst, pt, k, seed, o=None, name="", sample=None):
    rng = np.random.default_rng(seed)
    T, D = inst.T, inst.net.n_load
    Y, V = _dev(rng.standard_normal((k, h.m))), _dev(rng.standard_normal((k, h.n)))
    DP, DQ = _dev(rng.standard_normal((k, T * D))), _dev(rng.standard_normal((k, T * D)))
    xd, lam = _dev(pt.x), _dev(pt.lam)
    out = h.sweep(xd, lam, pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    jv, hw = out["jv"], out["hv"]
    many = {}
    for stored in (False, True):
        gx, gpd, gqd = h.vjp_many(xd, Y, jv=jv if stored else None)
        jvp = h.jvp_many(xd, V, jv=jv if stored else None)
        jvl = h.jvp_many(xd, V, dpd=DP, dqd=DQ, jv=jv if stored else None) if D else None
        hvp = h.hvp_many(xd, lam, pt.sigma, V, hw=hw if stored else None)
        torch.cuda.synchronize()
        many[stored] = (_np(gx), _np(gpd), _np(gqd), _np(jvp), None if jvl is None else _np(jvl), _np(hvp))
    for a, b in zip(many[False], many[True]):
        assert (a is None and b is None) or np.array_equal(a, b), name
    gx, gpd, gqd, jvp, jvl, hvp = many[False]
    for j in (range(k) if sample is None else sample):
        sgx, sgpd, sgqd = h.vjp(xd, Y[j])
        assert np.array_equal(gx[j], _np(sgx)), (name, j)
        assert np.array_equal(gpd[j], _np(sgpd)) and np.array_equal(gqd[j], _np(sgqd)), (name, j)
        assert np.array_equal(jvp[j], _np(h.jvp(xd, V[j]))), (name, j)
        if D:
            assert np.array_equal(jvl[j], _np(h.jvp(xd, V[j], dpd=DP[j], dqd=DQ[j]))), (name, j)
        assert np.array_equal(hvp[j], _np(h.hvp(xd, lam, pt.sigma, V[j]))), (name, j)
    if o is not None:
        for j in (0, k - 1):
            y, v = _np(Y[j]), _np(V[j])
            rgx, rgpd, rgqd = o.vjp(pt.x, y)
            assert_close(f"{name}:vjp[{j}]", gx[j], rgx)
            assert np.array_equal(gpd[j], rgpd) and np.array_equal(gqd[j], rgqd)
            assert_close(f"{name}:jvp[{j}]", jvp[j], o.jvp(pt.x, v))
            if D:
                assert_close(f"{name}:jvp_loads[{j}]", jvl[j],
                             o.jvp(pt.x, v, dpd=_np(DP[j]), dqd=_np(DQ[j])))
            assert_close(f"{name}:hvp[{j}]", hvp[j], o.hvp(pt.x, pt.lam, pt.sigma, v))


@pytest.mark.parametrize("name", sorted(MANY_CASES))
def test_many_vectors_equal_single_products(name):
    from paper_2405_14032_b300 import mpopf
    inst, seed = MANY_CASES[name]()
    pt = synth.make_point(seed, inst)
    h = mpopf.Handle(inst)
    _check_many(h, inst, pt, 4, seed + 100, oracle.Oracle(inst), name)
    h.close()


def test_differentiation_workload_256_vectors():
    """The 2,000-bus / 3,200-branch / 400-generator network at T = 24 with 256
    vectors, after a smaller call (the scratch grows): every product of all 256
    vectors in one call each; sampled vectors against the single products, the
    first and last against the oracle."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(5, 2000, 3200, 400, 1200, 24)
    pt = synth.make_point(5, inst)
    h = mpopf.Handle(inst)
    _check_many(h, inst, pt, 3, 7, None, "diff k=3")
    _check_many(h, inst, pt, 256, 8, oracle.Oracle(inst), "diff k=256", sample=(0, 1, 77, 128, 254, 255))
    h.close()


def test_many_argument_errors():
    from paper_2405_14032_b300 import mpopf
    inst = synth.config_instance("cfg1")
    h = mpopf.Handle(inst)
    pt = synth.make_point(1, inst)
    xd = _dev(pt.x)
    Y = torch.zeros(2, h.m, dtype=torch.float64, device="cuda")
    V = torch.zeros(2, h.n, dtype=torch.float64, device="cuda")
    G = torch.zeros(2, h.n, dtype=torch.float64, device="cuda")
    lib = mpopf.lib()
    p = lambda t: t.data_ptr()
    assert lib.mpopf_vjp_many(h.h, 0, p(xd), None, p(Y), p(G), None, None, None) == -1
    assert lib.mpopf_vjp_many(h.h, 2, p(xd), None, p(Y), p(G), p(G), None, None) == -1  # gpd without gqd
    assert lib.mpopf_jvp_many(h.h, 65536, p(xd), None, p(V), None, None, p(Y), None) == -1
    assert lib.mpopf_hvp_many(h.h, 2, p(xd), None, 1.0, None, p(V), p(G), None) == -1  # NULL lam
    with pytest.raises(ValueError):
        h.hvp_many(xd, _dev(pt.lam), 1.0, V[:, :-1].contiguous())
    h.close()
    hs = mpopf.Handle(inst, shard=(0, inst.T // 2))
    assert lib.mpopf_hvp_many(hs.h, 1, p(xd), p(_dev(pt.lam)), 1.0, None, p(V), p(G), None) == -1
    hs.close()
