"""Angle differences at the edges of the sin/cos evaluation, through the whole
sweep: the kernels' flows, J, W and M equal the oracle's bit for bit where
both sides evaluate the same polynomials (|x| < 2^30: no reduction up to
RN(pi/4), Cody-Waite reduction by pi/2 beyond), and within the stated
tolerance where both hand the argument to their math library (|x| >= 2^30,
not a voltage-angle difference any network produces).

A two-bus network with one branch over 48 periods: period t puts the angle
difference x_t on the branch (va_from = x_t, va_to = 0 at the reference bus).
"""
import math

import numpy as np
import pytest

from paper_2405_14032_b300 import synth
from tests import helpers as H
from tests.test_gpu_parity import Case, assert_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

Q = float.fromhex("0x1.921fb54442d18p-1")  # RN(pi/4): the largest argument without reduction
_EDGES = [0.0, 1e-300, 2.0 ** -30, 1e-8, 0.3, Q, math.nextafter(Q, 1.0), math.nextafter(Q, 0.0),
          math.pi / 2, math.nextafter(math.pi / 2, 4.0), math.pi, 3 * math.pi / 4, 2.0, 3.0, 100.0, 1e5,
          2.0 ** 30 - 1.0, math.nextafter(2.0 ** 30, 0.0)]
ANGLES = np.array(_EDGES + [-a for a in _EDGES if a != 0.0] + [2.0 ** 30, -(2.0 ** 30), 1e9, -3e9])


def _case():
    T = ANGLES.size
    net = H.network(2, [0], [1], [0.01], [0.1], [0.02], gen_bus=[0], load_bus=[1], ref=1)
    inst = H.instance(net, T)
    pt = synth.make_point(61, inst)
    sl = H.var_slices(net, T)
    va = pt.x[sl["va"]].reshape(T, 2)
    va[:, 0] = ANGLES
    va[:, 1] = 0.0
    pt.x[sl["va"]] = va.ravel()
    return Case(inst, 61, pt)


def test_sincos_edges_match_oracle():
    cs = _case()
    pt, o = cs.pt, cs.o
    out = cs.run()
    ref = o.eval(pt.x, pt.lam, pt.sigma)
    _, _, kv = o.kkt_csr(pt.x, pt.lam, pt.sigma, pt.sigma_x, pt.dvec, pt.delta_w)
    for k, r in (("c", ref["c"]), ("jv", ref["jv"]), ("hv", ref["hv"]), ("kv", kv)):
        assert_close(f"edges:{k}", out[k], r)
    # the four flow rows of period t sit at T + (k - 1) T + t (one branch)
    T = ANGLES.size
    same = np.abs(ANGLES) < 2.0 ** 30
    for k in range(4):
        rows = T + k * T + np.arange(T)
        got, want = out["c"][rows], ref["c"][rows]
        bad = np.nonzero(same & (got != want))[0]
        assert bad.size == 0, (k + 1, ANGLES[bad], got[bad], want[bad])
