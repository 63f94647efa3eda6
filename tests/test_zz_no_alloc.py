"""The allocation-free condensed-matrix entry point, through the C-ABI.

mpopf_assemble_kkt_noalloc serves callers that cannot call cudaMalloc while
they run (work recorded in a stream capture, processes that reserve all device
memory up front).  Its scratch is a fixed array inside the library, shared by
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
    # 3,200 branches x 240 periods = 768,000 branch-periods > 699,050
    inst = synth.make_instance(5, 2000, 3200, 400, 1200, 240)
    h = mpopf.Handle(inst)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mpopf.MpopfError) as err:
        h.assemble_kkt_noalloc(z, z, 1.0, z, z, 0.0, z)
    assert "(-2)" in str(err.value) and "static maximum" in str(err.value)
    h.close()
