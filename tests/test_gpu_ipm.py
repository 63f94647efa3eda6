"""Interior-point algebra around the condensed matrix on the GPU (Sec. III-B):
Sigma_x, D, C from the bounds and duals, the condensed right-hand side, and
the step recovery, against the oracle on the same seeded interior points
(tolerance |gpu - ref| <= max(1e-12 |ref|, 1e-14), and bit for bit: the
rounding order of every value is the oracle's).  The composition prepare -> assemble -> dense solve ->
recover on the GPU is checked against the full block system of Eq. (5)."""
import numpy as np
import pytest

from paper_2405_14032_b300 import synth
from tests import helpers as H
from tests.test_gpu_parity import CASES, Case, assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MU, DW, DC, EPS = 0.05, 1e-3, 1e-4, 1e-2


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


ALL = dict(CASES)
ALL["cfg2"] = lambda: Case(synth.config_instance("cfg2"), 2)


@pytest.fixture(scope="module", params=sorted(ALL))
def case(request):
    return request.param, ALL[request.param]()


def _point(cs, seed):
    x, s, y, zlx, zux, zls, zus, *_ = H.ipm_point(cs.inst, cs.o, seed, EPS)
    return dict(x=x, s=s, y=y, zlx=zlx, zux=zux, zls=zls, zus=zus)


@pytest.mark.parametrize("stored_j", [False, True])
@pytest.mark.parametrize("dw,dc", [(DW, DC), (0.0, 0.0), (0.5, 2.0)])
def test_prepare_rhs_recover_match_oracle(case, dw, dc, stored_j):
    name, cs = case
    o, h = cs.o, cs.h
    P = _point(cs, 71)
    D = {k: _dev(v) for k, v in P.items()}
    ref = o.eval(P["x"], P["y"], 1.0)
    rng = np.random.default_rng(72)
    dx = rng.standard_normal(o.n)

    sigx, dvec, cvec, recip = h.ipm_prepare(D["x"], D["s"], D["zlx"], D["zux"], D["zls"], D["zus"], dw, dc, EPS)
    rsigx, rdvec, rcvec, _, rrecip = o.ipm_prepare(P["x"], P["s"], P["zlx"], P["zux"], P["zls"], P["zus"], dw, dc,
                                                   EPS)
    for k, got, want in (("sigx", sigx, rsigx), ("dvec", dvec, rdvec), ("cvec", cvec, rcvec),
                         ("recip", recip, rrecip)):
        assert np.array_equal(_np(got), want), f"{name}:{k}"

    # grad f and c(x) from the oracle on both sides, so that only the algebra is compared
    args = (P["x"], P["s"], P["y"], P["zlx"], P["zux"], P["zls"], P["zus"])
    dx_, ds_, dy_ = D["x"], D["s"], D["y"]
    g, c = _dev(ref["g"]), _dev(ref["c"])
    from paper_2405_14032_b300 import mpopf
    jv = h.eval(mpopf.OUT_JAC, dx_)["jv"] if stored_j else None
    rhs = h.ipm_rhs(dx_, ds_, dy_, g, c, recip, dvec, cvec, MU, jv=jv)
    rrhs, _ = o.ipm_rhs(*args, ref["g"], ref["c"], MU, dw, dc, EPS)
    e, n = assert_close(f"{name}:rhs", _np(rhs), rrhs)
    assert e == n, f"{name}:rhs {e}/{n} bitwise"  # same element order as the oracle's J^T w

    rec = h.ipm_recover(dx_, ds_, dy_, D["zlx"], D["zux"], D["zls"], D["zus"], c, recip, cvec, _dev(dx), MU, dw, dc,
                        jv=jv)
    rrec = o.ipm_recover(*args, ref["c"], dx, MU, dw, dc, EPS)
    for k, rk in (("ds", "ds"), ("dy", "dy"), ("dzl_x", "dzlx"), ("dzu_x", "dzux"), ("dzl_s", "dzls"),
                  ("dzu_s", "dzus")):
        e, n = assert_close(f"{name}:{k}", _np(rec[k]), rrec[rk])
        assert e == n, f"{name}:{k} {e}/{n} bitwise"


def test_recovered_step_solves_lifted_system():
    """GPU prepare -> GPU assemble of M (W at lambda = -y) -> dense solve of
    M dx = rhs -> GPU recover solves the full block system of Eq. (5)."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(73, 12, 18, 3, 6, 3)
    cs = Case(inst, 73)
    o, h = cs.o, cs.h
    x, s, y, zlx, zux, zls, zus, xl, xu, sl, su = H.ipm_point(inst, o, 74, EPS)
    dx_, ds_, dy_ = _dev(x), _dev(s), _dev(y)
    dz = [_dev(a) for a in (zlx, zux, zls, zus)]
    sigx, dvec, cvec, recip = h.ipm_prepare(dx_, ds_, *dz, DW, DC, EPS)
    out = h.eval(mpopf.OUT_ALL, dx_, _dev(-y), 1.0, sigx, dvec, DW)
    rhs = h.ipm_rhs(dx_, ds_, dy_, out["grad"], out["c"], recip, dvec, cvec, MU)
    pat = {k: _np(v) for k, v in h.pattern().items()}
    n, m = o.n, o.m
    M = H.csr_to_dense_sym(pat["kkt_rowptr"], pat["kkt_col"], _np(out["kv"]), n)
    step = np.linalg.solve(M, _np(rhs))
    rec = h.ipm_recover(dx_, ds_, dy_, *dz, out["c"], recip, cvec, _dev(step), MU, DW, DC)
    A = H.dense_jac(pat["jac_row"], pat["jac_col"], _np(out["jv"]), m, n)
    W = H.dense_sym(pat["hess_row"], pat["hess_col"], _np(out["hv"]), n)
    K, p, sl_ = H.lifted_system(W, A, x, s, y, zlx, zux, zls, zus, xl, xu, sl, su, _np(out["grad"]),
                                _np(out["c"]), MU, DW, DC)
    il, iu = np.isfinite(xl), np.isfinite(xu)
    jl, ju = np.isfinite(sl), np.isfinite(su)
    d = np.concatenate([step, _np(rec["ds"]), _np(rec["dy"]), _np(rec["dzl_x"])[il], _np(rec["dzu_x"])[iu],
                        _np(rec["dzl_s"])[jl], _np(rec["dzu_s"])[ju]])
    res = K @ d - p
    scale = np.abs(K).max() * np.abs(d).max() + np.abs(p).max()
    assert np.abs(res).max() <= 1e-10 * scale
    assert np.all(_np(rec["dzl_x"])[~il] == 0) and np.all(_np(rec["dzu_s"])[~ju] == 0)


def test_null_argument_is_rejected():
    from paper_2405_14032_b300 import mpopf
    cs = Case(synth.config_instance("cfg1"), 1)
    lib = mpopf.lib()
    z = torch.zeros(cs.o.n, dtype=torch.float64, device="cuda")
    rc = lib.mpopf_ipm_prepare(cs.h.h, z.data_ptr(), None, None, None, None, None, 0.0, 0.0, 0.0, None, None,
                               None, None, None)
    assert rc == -1 and b"NULL" in lib.mpopf_last_error()
