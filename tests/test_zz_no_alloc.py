"""The allocation-free condensed-matrix entry point, through the C-ABI.

mpopf_assemble_kkt_noalloc serves callers that cannot call cudaMalloc once
they are running (processes that reserve all device memory up front, plugins
inside an application that owns the device's memory).  Its scratch is a fixed array inside the library, shared by
every call, so this test checks two calls in a row against the regular
mpopf_assemble_kkt, with the tolerance the parity tests use.  It sits in a file
of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2405_14032_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _close(got, ref):
    return bool(np.all(np.abs(got - ref) <= np.maximum(1e-12 * np.abs(ref), 1e-14)))


def test_noalloc_matches_assemble_kkt_two_calls():
    from paper_2405_14032_b300 import mpopf
    inst = synth.config_instance("cfg2")
    h = mpopf.Handle(inst)
    kv = torch.full((h.nnz_kkt,), float("nan"), dtype=torch.float64, device="cuda")
    for k, seed in enumerate((2, 77)):
        pt = synth.make_point(seed, inst)
        args = (_dev(pt.x), _dev(pt.lam), pt.sigma, _dev(pt.sigma_x), _dev(pt.dvec), pt.delta_w)
        ref = h.eval(mpopf.OUT_KKT, *args)["kv"]
        h.assemble_kkt_noalloc(*args, kv)
        torch.cuda.synchronize()
        got, want = kv.cpu().numpy(), ref.cpu().numpy()
        assert _close(got, want), f"call {k + 1}"
    h.close()


def test_noalloc_rejects_problems_over_its_static_limit():
    from paper_2405_14032_b300 import mpopf
    # 3,200 branches x 120 periods = 384,000 branch-periods > 349,525
    inst = synth.make_instance(5, 2000, 3200, 400, 1200, 120)
    h = mpopf.Handle(inst)
    # full-size arrays, so that the call would stay in bounds of its inputs
    # and output even if it were (wrongly) accepted
    zn = torch.zeros(h.n, dtype=torch.float64, device="cuda")
    zm = torch.zeros(h.m, dtype=torch.float64, device="cuda")
    kv = torch.zeros(h.nnz_kkt, dtype=torch.float64, device="cuda")
    with pytest.raises(mpopf.MpopfError) as err:
        h.assemble_kkt_noalloc(zn, zm, 1.0, zn, zm, 0.0, kv)
    assert "(-2)" in str(err.value) and "static maximum" in str(err.value)
    h.close()
