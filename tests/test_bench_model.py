"""The benchmark's speedup model (the paper's reciprocal-speedup formulas evaluated with
measured phase times) against cases the formulas fix by themselves:

- Eq. LinSpeedup (Alg. 1): free homogeneous problems give s = N; homogeneous problems as
  slow as the inhomogeneous ones give s = 1; the limit for many subintervals is
  (tau_I + tau_I') / (tau_H + tau_H').
- Eq. hybridSpeedup (Sec. 3.3, equal partition so that T_N - T_{N-1} = T/N): a chain as
  slow as the serial adjoint over T_H = T (N-1)/N gives s = 1; a free chain leaves
  s^-1 = (tau_I + tau_I'/N) / (tau_I + tau_I'); the limit is
  (tau_I + tau_I') / (tau_I + tau_H').

The phase times are built from chosen rates tau (ms per unit of simulated time) the way a
run would measure them: serial sweeps over [0, T], Paraexp chains over their spans.
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def linear_phases(T, P, tI, tIa, tH, tHa, lanes_ms=1.0):
    span = T * (P - 1) / P
    ser = {"ms_direct_inhom": T * tI, "ms_adjoint_inhom": T * tIa, "ms_direct_hom": 0.0,
           "ms_adjoint_hom": 0.0, "ms_total": T * (tI + tIa)}
    par = {"ms_direct_inhom": lanes_ms, "ms_adjoint_inhom": lanes_ms, "ms_direct_hom": span * tH,
           "ms_adjoint_hom": span * tHa, "ms_total": 2 * lanes_ms + span * (tH + tHa)}
    return {"paraexp": par, "serial": ser}


def hybrid_phases(T, P, tI, tIa, tHa, T_H):
    ser = {"ms_direct_inhom": T * tI, "ms_adjoint_inhom": T * tIa, "ms_direct_hom": 0.0,
           "ms_adjoint_hom": 0.0, "ms_total": T * (tI + tIa)}
    par = {"ms_direct_inhom": T * tI, "ms_adjoint_inhom": (T / P) * tIa, "ms_direct_hom": 0.0,
           "ms_adjoint_hom": T_H * tHa, "ms_total": T * tI + (T / P) * tIa + T_H * tHa}
    return {"paraexp": par, "serial": ser}


@pytest.mark.parametrize("P", [2, 8, 64])
def test_linear_free_homogeneous_problems_give_the_subinterval_count(P):
    m = bench.speedup_model("linear", linear_phases(1.0, P, 3.0, 2.0, 0.0, 0.0), 1.0, P)
    assert m["predicted"] == pytest.approx(P, rel=1e-14)


@pytest.mark.parametrize("P", [2, 8, 64])
def test_linear_homogeneous_as_slow_as_stepping_gives_no_speedup(P):
    m = bench.speedup_model("linear", linear_phases(2.0, P, 3.0, 2.0, 3.0, 2.0), 2.0, P)
    assert m["predicted"] == pytest.approx(1.0, rel=1e-14)
    assert m["limit"] == pytest.approx(1.0, rel=1e-14)


def test_linear_limit_and_monotone_in_the_subintervals():
    tI, tIa, tH, tHa = 4.0, 3.0, 0.5, 0.2
    preds = [bench.speedup_model("linear", linear_phases(1.0, P, tI, tIa, tH, tHa), 1.0, P)["predicted"]
             for P in (2, 4, 16, 256, 65536)]
    assert all(b > a for a, b in zip(preds, preds[1:]))
    lim = (tI + tIa) / (tH + tHa)
    assert preds[-1] == pytest.approx(lim, rel=1e-3) and preds[-1] < lim


def test_linear_lanes_efficiency_is_one_for_ideal_lanes():
    T, P, tI, tIa = 1.0, 8, 3.0, 2.0
    ph = linear_phases(T, P, tI, tIa, 0.1, 0.1, lanes_ms=0.0)
    ph["paraexp"]["ms_direct_inhom"] = (T / P) * tI
    ph["paraexp"]["ms_adjoint_inhom"] = (T / P) * tIa
    m = bench.speedup_model("linear", ph, T, P)
    assert m["lanes_efficiency"] == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("P", [4, 32, 64])
def test_hybrid_chain_as_slow_as_the_serial_adjoint_gives_no_speedup(P):
    T, tI, tIa = 1.0, 3.2, 2.9
    T_H = T * (P - 1) / P
    m = bench.speedup_model("hybrid", hybrid_phases(T, P, tI, tIa, tIa, T_H), T, P, T_H=T_H)
    assert m["predicted"] == pytest.approx(1.0, rel=1e-14)
    assert m["measured"] == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("P", [4, 32, 64])
def test_hybrid_free_chain_leaves_the_serial_direct_and_one_lane(P):
    T, tI, tIa = 2.0, 3.2, 2.9
    m = bench.speedup_model("hybrid", hybrid_phases(T, P, tI, tIa, 0.0, T), T, P, T_H=T)
    assert 1.0 / m["predicted"] == pytest.approx((tI + tIa / P) / (tI + tIa), rel=1e-14)
    assert m["predicted"] == pytest.approx(m["measured"], rel=1e-14)


def test_hybrid_limit():
    tI, tIa, tHa = 3.2, 2.9, 0.9
    m = bench.speedup_model("hybrid", hybrid_phases(1.0, 64, tI, tIa, tHa, 1.0), 1.0, 64, T_H=1.0)
    assert m["limit"] == pytest.approx((tI + tIa) / (tI + tHa), rel=1e-14)
    assert m["predicted"] < m["limit"]
