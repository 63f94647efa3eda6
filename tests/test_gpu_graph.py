"""Evaluations captured into a CUDA graph.  An evaluation forks its generator
kernels onto the handle's side stream and joins them back with events; under
stream capture that fork becomes a parallel branch of the graph.  Replaying
the graph must give the plain sweep's outputs bit for bit, also for a graph of
several sweeps at different iterates and for the callbacks one by one."""
import numpy as np
import pytest

from paper_2405_14032_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("sched", [(0, 4), (0, 0), (2, 1), (1, 2), (0, 8), (0, 20), (0, 16)])
@pytest.mark.parametrize("shape", [(300, 480, 60, 180, 6), (57, 91, 11, 30, 3), (40, 64, 0, 20, 4)])
def test_graph_replay_equals_plain(shape, sched):
    """sched: the launch schedule (period chunks with the bus kernels on a
    second stream, itself a parallel branch of the captured graph; the bus
    kernel as a programmatic dependent launch, a programmatic edge of the
    graph; the bus-end products' launch before the branch kernel)."""
    from paper_2405_14032_b300 import mpopf
    N, L, G, D, T = shape
    inst = synth.make_instance(71, N, L, G, D, T)
    pt = synth.make_point(71, inst)
    h = mpopf.Handle(inst)
    x0, lam, sx, dv = _dev(pt.x), _dev(pt.lam), _dev(pt.sigma_x), _dev(pt.dvec)
    gen = torch.Generator(device="cuda").manual_seed(5)
    xs = [x0 + 1e-3 * torch.randn(h.n, generator=gen, device="cuda", dtype=torch.float64) for _ in range(3)]
    refs = [h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w) for x in xs]  # plain schedule
    torch.cuda.synchronize()
    h.set_sweep_schedule(*sched)

    outs = [h.new_outputs() for _ in xs]
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            for x, out in zip(xs, outs):
                h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=out, stream=st)
    torch.cuda.synchronize()
    for _ in range(2):
        for out in outs:
            for v in out.values():
                v.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for ref, out in zip(refs, outs):
            for k in ref:
                assert torch.equal(out[k], ref[k]), (shape, k)

    # the callbacks one by one, captured the same way
    single = {}
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g2, stream=st):
            single["f"] = h.eval(mpopf.OUT_OBJ, xs[0], stream=st)["f"]
            single["c"] = h.eval(mpopf.OUT_CONS, xs[0], stream=st)["c"]
            single["hv"] = h.eval(mpopf.OUT_HESS, xs[0], lam, pt.sigma, stream=st)["hv"]
    g2.replay()
    torch.cuda.synchronize()
    for k in single:
        assert torch.equal(single[k], refs[0][k]), (shape, k)
    del g, g2
    h.close()


def test_profiling_times_the_callers_stream_kernels():
    """Per-kernel profiling with the generator work on the side stream: the
    branch and bus launches are timed, the side-stream launches are not, and
    the outputs are those of an unprofiled sweep."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(72, 200, 320, 40, 120, 4)
    pt = synth.make_point(72, inst)
    h = mpopf.Handle(inst)
    x, lam, sx, dv = _dev(pt.x), _dev(pt.lam), _dev(pt.sigma_x), _dev(pt.dvec)
    ref = h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w)
    out = h.new_outputs()
    h.profile_start(4 * 3)
    for _ in range(3):
        h.sweep(x, lam, pt.sigma, sx, dv, pt.delta_w, out=out)
    prof = h.profile_stop()
    assert prof["branch"][1] == 3 and prof["bus"][1] == 3
    assert prof["gen"][1] == 0 and prof["fsum"][1] == 0
    assert prof["branch"][0] > 0 and prof["bus"][0] > 0
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    h.close()


def test_points_and_many_products_in_a_graph():
    """mpopf_sweep_points and the many-vector products captured after a first
    call of the same size (their scratch exists, so the captured calls
    allocate nothing): replays equal the eager results bit for bit."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(73, 300, 480, 60, 180, 6)
    h = mpopf.Handle(inst)
    pts = [synth.make_point(73, inst, stream_offset=100 * j) for j in range(3)]
    st_ = lambda key: torch.as_tensor(np.stack([getattr(p, key) for p in pts]), dtype=torch.float64,
                                      device="cuda").contiguous()
    X, LAM, SX, DV = st_("x"), st_("lam"), st_("sigma_x"), st_("dvec")
    V = torch.randn(5, h.n, generator=torch.Generator(device="cuda").manual_seed(3), device="cuda",
                    dtype=torch.float64)
    ref = h.sweep_points(X, LAM, 1.0, SX, DV, 1e-8)
    ref_h = h.hvp_many(X[0], LAM[0], 1.0, V)
    torch.cuda.synchronize()
    out = h.new_point_outputs(3)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    holder = {}
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            h.sweep_points(X, LAM, 1.0, SX, DV, 1e-8, out=out, stream=st)
            holder["hv"] = h.hvp_many(X[0], LAM[0], 1.0, V, stream=st)
    torch.cuda.synchronize()
    for _ in range(2):
        for v in out.values():
            v.fill_(float("nan"))
        holder["hv"].fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(out[k], ref[k]), k
        assert torch.equal(holder["hv"], ref_h)
    del g
    h.close()


def test_points_scratch_growth_refused_under_capture():
    """A captured sweep_points / hvp_many call whose scratch would have to grow
    returns MPOPF_ERR_ARG (no allocation or device synchronisation inside the
    capture); after an eager call of that size the same capture works."""
    from paper_2405_14032_b300 import mpopf
    inst = synth.make_instance(74, 120, 190, 24, 70, 3)
    h = mpopf.Handle(inst)
    pts = [synth.make_point(74, inst, stream_offset=100 * j) for j in range(3)]
    st_ = lambda key: torch.as_tensor(np.stack([getattr(p, key) for p in pts]), dtype=torch.float64,
                                      device="cuda").contiguous()
    X, LAM, SX, DV = st_("x"), st_("lam"), st_("sigma_x"), st_("dvec")
    out = h.new_point_outputs(3)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with pytest.raises(mpopf.MpopfError, match="stream capture"):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                h.sweep_points(X, LAM, 1.0, SX, DV, 1e-8, out=out, stream=st)
    torch.cuda.synchronize()
    ref = h.sweep_points(X, LAM, 1.0, SX, DV, 1e-8)  # grows the scratch
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            h.sweep_points(X, LAM, 1.0, SX, DV, 1e-8, out=out, stream=st)
    g.replay()
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    del g
    h.close()
