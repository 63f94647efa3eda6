"""The pins are strong enough to catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle source (a dropped term, a
wrong sign, a wrong index, a transposed operand, a wrong coefficient),
compiles it, and checks that at least one pin written against the paper and
the mathematics (closed forms, an independently written textbook model,
complex-step derivatives, dense brute force, scipy, the C library, a dense
solve of the block system of Eq. 5) fails on it.  No GPU is involved.
"""
import numpy as np
import pytest

import oracle
from paper_2405_14032_b300 import synth
from tests import test_oracle_pins as P


def _cfg1():
    inst = synth.config_instance("cfg1")
    return inst, synth.make_point(1, inst), oracle.Oracle(inst)


def _cfg1_ramp():
    inst = synth.with_reactive_ramp(synth.config_instance("cfg1"))
    return inst, synth.make_point(1, inst), oracle.Oracle(inst)


# name: (exact source text, replacement, occurrence to replace (0-based), pin that must fail)
MUTATIONS = {
    "flow term sign": ("q.A1 = fmaS(S(gft), cs, S(bft) * sn);", "q.A1 = fmaS(S(gft), cs, -(S(bft) * sn));", 0,
                       lambda: P.test_constraints_match_textbook(_cfg1())),
    "arc flow sign in the balance": ("acc = acc - x[P ? v_p(M, t, a) : v_q(M, t, a)];",
                                     "acc = acc + x[P ? v_p(M, t, a) : v_q(M, t, a)];", 0,
                                     lambda: P.test_constraints_match_textbook(_cfg1())),
    "shunt sign": ("acc = fmaS(S(P ? -M.gs[n] : M.bs[n]), vm2, acc);",
                   "acc = fmaS(S(P ? M.gs[n] : M.bs[n]), vm2, acc);", 0,
                   lambda: P.test_constraints_match_textbook(_cfg1())),
    "thermal limit not squared": ("const double smax2 = M.smax[l] * M.smax[l];", "const double smax2 = M.smax[l];",
                                  0, lambda: P.test_constraints_match_textbook(_cfg1())),
    "ramp difference sign": ("*cval = x[jt] - x[jp];", "*cval = x[jt] + x[jp];", 0,
                             lambda: P.test_constraints_match_textbook(_cfg1_ramp())),
    "Jacobian entry sign": ("push(jvf, -q.dPfr_vf);", "push(jvf, q.dPfr_vf);", 0,
                            lambda: P.test_jacobian_complex_step(_cfg1())),
    "Hessian coefficient": ("std::fma(l2, 2.0 * M.bff[l], -(l1 * (2.0 * M.gff[l])))",
                            "std::fma(l2, M.bff[l], -(l1 * (2.0 * M.gff[l])))", 0,
                            lambda: P.test_hessian_complex_step_and_symmetry(_cfg1())),
    "condensed matrix operand": ("slot = std::fma(w, vals_i[q], slot);", "slot = std::fma(w, vals_i[p], slot);", 0,
                                 lambda: P.test_kkt_dense_brute_force(_cfg1())),
    "transposed product row": ("slot = std::fma(vals_i[p], y[i], slot);",
                               "slot = std::fma(vals_i[p], y[std::min<int64_t>(i + 1, M.m - 1)], slot);", 0,
                               lambda: P.test_vjp_jvp_hvp(_cfg1())),
    "sine coefficient": ("kP2 = -0x1.a01a019e6dedep-13", "kP2 = 0x1.a01a019e6dedep-13", 0,
                         lambda: P.test_sincos_against_c_library(-3.0, 3.0)),
    "slack right-hand side sign": ("const double qs = std::fma(mu, r.ru - r.rl, y[i]);",
                                   "const double qs = std::fma(mu, r.rl - r.ru, y[i]);", 0,
                                   lambda: P.test_ipm_condensation_solves_full_lifted_system(1e-3, 1e-4)),
    "reactive limits swapped": ("xl[v_qg(M, t, g)] = M.qmin[g]; xu[v_qg(M, t, g)] = M.qmax[g];",
                                "xl[v_qg(M, t, g)] = M.qmax[g]; xu[v_qg(M, t, g)] = M.qmin[g];", 0,
                                lambda: P.test_bounds_written_out_from_the_model(False, 2)),
    "angle limits taken as symmetric": ("lo = M.angmin[comp]; hi = M.angmax[comp];",
                                        "lo = -M.angmax[comp]; hi = M.angmax[comp];", 0,
                                        lambda: P.test_bounds_written_out_from_the_model(False, 1)),
    "reactive ramp limit from the P ramp": ("lo = -M.qramp[comp]; hi = M.qramp[comp];",
                                            "lo = -M.ramp[comp]; hi = M.ramp[comp];", 0,
                                            lambda: P.test_bounds_written_out_from_the_model(True, 3)),
    "condensed-matrix diagonal without delta_w": ("contrib.push_back({{j, j}, sigx[j] + delta_w});",
                                                  "contrib.push_back({{j, j}, sigx[j]});", 0,
                                                  lambda: P.test_kkt_dense_brute_force(_cfg1())),
    "W v with a transposed entry": ("b = std::fma(e.v, v[e.r], b);", "b = std::fma(e.v, v[e.c], b);", 0,
                                    lambda: P.test_vjp_jvp_hvp(_cfg1())),
    "load tangent sign": ("acc = acc - dl[t * M.D + d];", "acc = acc + dl[t * M.D + d];", 0,
                          lambda: P.test_jvp_load_tangent_finite_difference()),
    "load adjoint sign": ("if (gpd) gpd[t * M.D + d] = -y[r_k8(M, t, M.lbus[d])];",
                          "if (gpd) gpd[t * M.D + d] = y[r_k8(M, t, M.lbus[d])];", 0,
                          lambda: P.test_load_adjoint_complex_step()),
    "Sigma with the bound reciprocals swapped": ("return std::fma(zl, r.rl, zu * r.ru);",
                                                "return std::fma(zl, r.ru, zu * r.rl);", 0,
                                                lambda: P.test_ipm_condensation_solves_full_lifted_system(1e-3, 1e-4)),
    "multiplier step without delta_w": ("dy[i] = std::fma(sg + delta_w, d, -qs);", "dy[i] = std::fma(sg, d, -qs);", 0,
                                        lambda: P.test_ipm_condensation_solves_full_lifted_system(0.3, 0.7)),
    "cost constant dropped": ("acc = acc + std::fma(std::fma(M.c2[g], pg, M.c1[g]), pg, M.c0[g]);",
                              "acc = acc + std::fma(std::fma(M.c2[g], pg, M.c1[g]), pg, 0.0);", 0,
                              lambda: P.test_objective_with_constant_cost()),
    "ramp rows of a window's first period skipped": (
        "const int64_t a = std::max<int64_t>(t0, 1), b = std::max<int64_t>(t1, 1);",
        "const int64_t a = t0 + 1, b = std::max<int64_t>(t1, 1);", 0,
        lambda: P.test_windowed_outputs_agree_with_full()),
    "CSC drops a duplicate": ("vals[k] = vals[k] + coo[v[p].e];", "vals[k] = coo[v[p].e];", 0,
                              lambda: P.test_csc_compression_matches_scipy_and_dense(1)),
}


def _plant(old, new, occurrence):
    src = open(oracle._SRC).read()
    pos = -1
    for _ in range(occurrence + 1):
        pos = src.index(old, pos + 1)
    return src[:pos] + new + src[pos + len(old):]


def test_every_mutation_site_exists():
    src = open(oracle._SRC).read()
    for name, (old, _, occurrence, _) in MUTATIONS.items():
        assert src.count(old) > occurrence, name


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new, occurrence, pin = MUTATIONS[name]
    path = oracle.build_variant(_plant(old, new, occurrence), str(tmp_path))
    with oracle.using(path):
        with pytest.raises(AssertionError):
            pin()
    # the unmodified oracle passes the same pin
    pin()


def test_unmodified_oracle_is_restored():
    inst, pt, o = _cfg1()
    assert o._lib is oracle.load()
    assert np.isfinite(o.eval(pt.x, pt.lam, pt.sigma)["c"]).all()
