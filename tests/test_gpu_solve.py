"""The library factorisation of the condensed matrix (cuSOLVER sparse Cholesky
standing in for the paper's cuDSS) inside one interior-point step on the GPU:
prepare -> sweep -> condensed right-hand side -> factor -> solve -> recover.
The solve is checked against a dense solve of the oracle's M (small cases) and
by its residual (the 2,000-bus case); the whole step against the dense lifted
system of Eq. (5).  The library's values are not bitwise: tolerances follow
from the conditioning of M."""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H
from tests.test_gpu_parity import _edge_network

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS, MU, DC = 1e-2, 0.05, 1e-4


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _step(inst, seed, dw):
    """One GPU step at an interior point; returns everything the checks need."""
    from paper_2405_14032_b300 import mpopf
    o = oracle.Oracle(inst)
    h = mpopf.Handle(inst)
    x, s, y, zlx, zux, zls, zus, xl, xu, sl, su = H.ipm_point(inst, o, seed, EPS)
    dz = [_dev(a) for a in (zlx, zux, zls, zus)]
    dx_, ds_, dy_ = _dev(x), _dev(s), _dev(y)
    sigx, dvec, cvec, recip = h.ipm_prepare(dx_, ds_, *dz, dw, DC, EPS)
    out = h.sweep(dx_, _dev(-y), 1.0, sigx, dvec, dw)
    rhs = h.ipm_rhs(dx_, ds_, dy_, out["grad"], out["c"], recip, dvec, cvec, MU)
    pivot = h.kkt_factor(out["kv"])
    step = h.kkt_solve(rhs) if pivot < 0 else None
    rec = h.ipm_recover(dx_, ds_, dy_, *dz, out["c"], recip, cvec, step, MU, dw, DC) if step is not None else None
    torch.cuda.synchronize()
    return dict(o=o, h=h, x=x, s=s, y=y, z=(zlx, zux, zls, zus), bounds=(xl, xu, sl, su), out=out, rhs=rhs,
                pivot=pivot, step=step, rec=rec, sigx=sigx, dvec=dvec)


def _dense_m(h, kv):
    pat = {k: _np(v) for k, v in h.pattern().items()}
    return H.csr_to_dense_sym(pat["kkt_rowptr"], pat["kkt_col"], _np(kv), h.n)


CASES = {
    "cfg1": lambda: synth.config_instance("cfg1"),
    "edge_T5": lambda: H.instance(_edge_network(), 5),
    "qramp_T3": lambda: synth.with_reactive_ramp(synth.make_instance(81, 30, 48, 6, 18, 3)),
    "ragged_T2": lambda: synth.make_instance(82, 120, 190, 24, 70, 2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_factor_solve_against_dense_and_lifted_system(name):
    inst = CASES[name]()
    r = _step(inst, 90, dw=50.0)
    M = _dense_m(r["h"], r["out"]["kv"])
    assert np.all(np.linalg.eigvalsh(M) > 0), "choose a larger delta_w for this case"
    assert r["pivot"] == -1
    rhs, step = _np(r["rhs"]), _np(r["step"])
    ref = np.linalg.solve(M, rhs)
    cond = np.linalg.cond(M)
    assert np.abs(step - ref).max() <= 1e-14 * cond * np.abs(ref).max()
    assert np.abs(M @ step - rhs).max() <= 1e-12 * (np.abs(M).max() * np.abs(step).max() + np.abs(rhs).max())
    # the recovered step solves the full lifted system
    o, out = r["o"], r["out"]
    pat = {k: _np(v) for k, v in r["h"].pattern().items()}
    A = H.dense_jac(pat["jac_row"], pat["jac_col"], _np(out["jv"]), o.m, o.n)
    W = H.dense_sym(pat["hess_row"], pat["hess_col"], _np(out["hv"]), o.n)
    K, p, _ = H.lifted_system(W, A, r["x"], r["s"], r["y"], *r["z"], *r["bounds"], _np(out["grad"]), _np(out["c"]),
                              MU, 50.0, DC)
    xl, xu, sl, su = r["bounds"]
    rec = {k: _np(v) for k, v in r["rec"].items()}
    d = np.concatenate([step, rec["ds"], rec["dy"], rec["dzl_x"][np.isfinite(xl)], rec["dzu_x"][np.isfinite(xu)],
                        rec["dzl_s"][np.isfinite(sl)], rec["dzu_s"][np.isfinite(su)]])
    scale = np.abs(K).max() * np.abs(d).max() + np.abs(p).max()
    assert np.abs(K @ d - p).max() <= 1e-10 * scale
    r["h"].close()


def test_not_positive_definite_is_reported():
    """A strongly negative delta_w makes M indefinite: the factorisation
    reports a pivot row and the solve is refused."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.config_instance("cfg1")
    r = _step(inst, 91, dw=-1e4)
    assert 0 <= r["pivot"] < r["h"].n
    with pytest.raises(mpopf.MpopfError):
        r["h"].kkt_solve(r["rhs"])
    # a later positive definite factorisation works again on the same handle
    h = r["h"]
    o = r["o"]
    x, s, y = r["x"], r["s"], r["y"]
    sigx, dvec, cvec, recip = h.ipm_prepare(_dev(x), _dev(s), *[_dev(a) for a in r["z"]], 50.0, DC, EPS)
    out = h.sweep(_dev(x), _dev(-y), 1.0, sigx, dvec, 50.0)
    assert h.kkt_factor(out["kv"]) == -1
    rhs = torch.ones(o.n, dtype=torch.float64, device="cuda")
    sol = _np(h.kkt_solve(rhs))
    M = _dense_m(h, out["kv"])
    assert np.abs(M @ sol - 1.0).max() <= 1e-10 * np.abs(M).max() * np.abs(sol).max()
    h.close()


def test_factor_solve_2000_bus_residual():
    """The 2,000-bus, T = 24 network: relative residual of the library solve,
    with M applied through a symmetric expansion of its lower CSR."""
    inst = synth.config_instance("cfg2")
    r = _step(inst, 92, dw=50.0)
    assert r["pivot"] == -1
    h = r["h"]
    pat = h.pattern()
    rp, col, kv = pat["kkt_rowptr"], pat["kkt_col"].long(), r["out"]["kv"]
    rows = torch.repeat_interleave(torch.arange(h.n, device="cuda"), rp[1:] - rp[:-1])
    off = rows != col
    idx = torch.cat([torch.stack([rows, col]), torch.stack([col[off], rows[off]])], 1)
    M = torch.sparse_coo_tensor(idx, torch.cat([kv, kv[off]]), (h.n, h.n), check_invariants=True).coalesce()
    res = torch.mv(M, r["step"]) - r["rhs"]
    scale = kv.abs().max() * r["step"].abs().max() + r["rhs"].abs().max()
    assert float(res.abs().max() / scale) <= 1e-10
    h.close()
