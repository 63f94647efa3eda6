"""COO -> CSC compression of J and the lower W on the GPU (Sec. III-A) against
the oracle's compression of the same COO values: identical colptr / rowidx,
values bit for bit (J is a permutation; W's duplicate entries are summed in
COO order on both sides)."""
import numpy as np
import pytest

from paper_2405_14032_b300 import synth
from tests.test_gpu_parity import CASES, Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALL = dict(CASES)
ALL["cfg2"] = lambda: Case(synth.config_instance("cfg2"), 2)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=sorted(ALL))
def case(request):
    return request.param, ALL[request.param]()


def test_csc_matches_oracle(case):
    from paper_2405_14032_b300 import mpopf
    name, cs = case
    out = cs.h.eval(mpopf.OUT_JAC | mpopf.OUT_HESS, torch.as_tensor(cs.pt.x, device="cuda"),
                    torch.as_tensor(cs.pt.lam, device="cuda"), cs.pt.sigma)
    for which, key in ((mpopf.CSC_JAC, "jv"), (mpopf.CSC_HESS, "hv")):
        pat = cs.h.csc_pattern(which)
        vals = cs.h.coo_to_csc(which, out[key])
        torch.cuda.synchronize()
        colptr, rowidx, ref = cs.o.csc(which, _np(out[key]))
        assert np.array_equal(_np(pat["colptr"]), colptr), (name, which)
        assert np.array_equal(_np(pat["rowidx"]), rowidx), (name, which)
        assert np.array_equal(_np(vals), ref), (name, which)
        again = cs.h.csc_pattern(which)  # built once
        assert again["colptr"].data_ptr() == pat["colptr"].data_ptr()


def test_csc_argument_errors():
    from paper_2405_14032_b300 import mpopf
    cs = Case(synth.config_instance("cfg1"), 1)
    lib = mpopf.lib()
    buf = torch.zeros(cs.o.nnz_jac, dtype=torch.float64, device="cuda")
    assert lib.mpopf_coo_to_csc(cs.h.h, 0, buf.data_ptr(), buf.data_ptr(), None) == -1
    assert b"mpopf_csc_pattern" in lib.mpopf_last_error()
    c = mpopf._Csc()
    import ctypes
    assert lib.mpopf_csc_pattern(cs.h.h, 2, ctypes.byref(c)) == -1
