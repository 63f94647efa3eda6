"""Independent handles used at the same time on separate CUDA streams (each
call enqueues on the stream it is given; each handle owns its scratch) give
the same outputs, bit for bit, as the same sweeps run one after the other."""
import numpy as np
import pytest

from paper_2405_14032_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_concurrent_handles_on_separate_streams():
    from paper_2405_14032_b300 import mpopf
    shapes = [(400, 640, 80, 240, 12), (900, 1440, 180, 540, 6), (150, 240, 30, 90, 24), (1200, 1920, 240, 720, 4)]
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    cases = []
    for k, (N, L, G, D, T) in enumerate(shapes):
        inst = synth.make_instance(200 + k, N, L, G, D, T)
        pt = synth.make_point(200 + k, inst)
        h = mpopf.Handle(inst)
        args = (dev(pt.x), dev(pt.lam), pt.sigma, dev(pt.sigma_x), dev(pt.dvec), pt.delta_w)
        ref = h.sweep(*args)
        torch.cuda.synchronize()
        cases.append((h, args, {kk: v.clone() for kk, v in ref.items()}))
    streams = [torch.cuda.Stream() for _ in cases]
    outs = [h.new_outputs() for h, _, _ in cases]
    for rep in range(20):
        for (h, args, _), s, o in zip(cases, streams, outs):
            with torch.cuda.stream(s):
                h.sweep(*args, out=o, stream=s)
                if rep % 5 == 0:  # also the derivative products on the same streams
                    h.vjp(args[0], args[1], loads=False, stream=s)
    torch.cuda.synchronize()
    for (h, _, ref), o in zip(cases, outs):
        for k in ref:
            assert torch.equal(o[k], ref[k]), k
        h.close()
