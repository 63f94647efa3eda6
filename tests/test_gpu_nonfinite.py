"""Non-finite inputs are data, not faults: NaN and Inf in x (a voltage angle, a
magnitude, a generator output, an arc flow) and in the multipliers propagate
to exactly the outputs that depend on them, at the same positions as in the
CPU oracle, with every other entry unchanged; the call returns MPOPF_OK and
the next call on clean inputs is clean (no sticky error, no trap)."""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _same(got, ref):
    """Equal entries, NaN where the oracle has NaN, +-Inf where it has +-Inf."""
    return np.array_equal(got, ref, equal_nan=True)


def test_nan_and_inf_inputs_match_the_oracle():
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(81, 60, 96, 12, 36, 3)
    pt = synth.make_point(81, inst)
    o = oracle.Oracle(inst)
    h = mpopf.Handle(inst)
    sl = H.var_slices(inst.net, inst.T)
    clean = h.sweep(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    clean = {k: v.cpu().numpy() for k, v in clean.items()}
    x = pt.x.copy()
    lam = pt.lam.copy()
    x[sl["va"].start + 5] = np.nan                # an angle of period 0
    x[sl["vm"].start + inst.net.n_bus + 7] = np.inf  # a magnitude of period 1
    x[sl["pg"].start + 2 * inst.net.n_gen + 1] = -np.inf  # a generator output of period 2
    x[sl["q"].start + 3] = np.nan                 # an arc flow of period 0
    lam[inst.T + 10] = np.nan                     # a flow-row multiplier
    out = h.sweep(_dev(x), _dev(lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    with np.errstate(invalid="ignore", over="ignore"):
        ref = o.eval(x, lam, pt.sigma)
        _, _, kv = o.kkt_csr(x, lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    for key, gkey in (("g", "grad"), ("c", "c"), ("jv", "jv"), ("hv", "hv")):
        assert _same(got[gkey], ref[key]), gkey
        assert not np.isfinite(got[gkey]).all() or gkey in ("grad",), gkey
    assert _same(got["kv"], kv)
    assert not np.isfinite(got["kv"]).all()
    assert np.isnan(got["f"][0]) or np.isinf(got["f"][0])
    # the non-finite values reach only the outputs that depend on them
    for key in ("c", "jv", "hv", "kv"):
        fin = np.isfinite(got[key])
        assert fin.sum() > 0.9 * fin.size, key
        assert np.array_equal(got[key][fin], got[key][fin])
    # the next call with clean inputs is clean
    again = h.sweep(_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
    torch.cuda.synchronize()
    for k in clean:
        assert np.array_equal(again[k].cpu().numpy(), clean[k]), k
    h.close()
