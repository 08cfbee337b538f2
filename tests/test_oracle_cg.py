"""Pins for the oracle's conjugate-gradient loop (Algorithm 1's CGsolver with
the search interval of Section IV-A).

  * the first direction is steepest descent: x_1 - x_0 is -grad f(x_0)
    scaled so that the farthest unclamped cell moves by a_0, with grad f
    taken from an independent evaluation (W~ and N gradients, lambda_0 =
    |grad W~|_1 / |grad N|_1);
  * every step lies in [0.01 a_max_k, a_max_k] with a_max_0 = 0.044 w_b and
    a_max_{k+1} = max(a_max_0, 2 a_k);
  * the loop reaches the overflow target tau <= 0.1 on the small design and
    reduces the energy it was started from.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def tiny():
    return synth.make_instance("tiny")


def test_first_step_is_steepest_descent(tiny):
    inst = tiny
    x, y, rows, ran = oracle.cg(inst, 1, gamma_fixed=inst.gamma)
    assert ran == 1
    ev = oracle.eval_instance(inst)
    lam = ev["gW_l1"] / ev["gN_l1"]
    gx = ev["gWx"] + lam * ev["gNx"]
    gy = ev["gWy"] + lam * ev["gNy"]
    ginf = max(np.abs(gx).max(), np.abs(gy).max())
    a0 = rows[0]["alpha"]
    x0 = inst.x.astype(np.float64); y0 = inst.y.astype(np.float64)
    L = inst.region[2]
    lox, hix = 0.5 * inst.w[:inst.m_mov], L - 0.5 * inst.w[:inst.m_mov]
    loy, hiy = 0.5 * inst.h[:inst.m_mov], L - 0.5 * inst.h[:inst.m_mov]
    ex = np.clip(x0 - a0 * gx / ginf, lox, hix)
    ey = np.clip(y0 - a0 * gy / ginf, loy, hiy)
    # positions are float32 at the end of the loop
    np.testing.assert_allclose(x, ex, rtol=0, atol=2e-5 * L)
    np.testing.assert_allclose(y, ey, rtol=0, atol=2e-5 * L)
    assert rows[0]["lam"] == pytest.approx(lam, rel=1e-12)


def test_step_interval_and_recurrence(tiny):
    inst = tiny
    wb = (inst.region[2] - inst.region[0]) / inst.n
    _, _, rows, ran = oracle.cg(inst, 40, gamma_fixed=inst.gamma)
    amax0 = 0.044 * wb
    amax = amax0
    for r in rows:
        a = r["alpha"]
        assert 0.01 * amax * (1 - 1e-12) <= a <= amax * (1 + 1e-12)
        assert r["step_max"] == a
        amax = max(amax0, 2.0 * a)


def test_reaches_overflow_target(tiny):
    inst = tiny
    _, _, rows, ran = oracle.cg(inst, 300, gamma_fixed=0.0, stop_on_tau=True)
    assert ran < 300 and rows[-1]["tau"] <= 0.1
    assert rows[-1]["N"] < rows[0]["N"]
