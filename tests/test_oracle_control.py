"""Pins of the oracle's parameter control (Section IV-A) and placement loop.

The scalar formulas are checked at values worked out by hand from the
paper's constants (tests/golden/control_constants.txt); the loop against a
separate Python restatement of one and two Nesterov iterations built on the
(separately pinned) evaluation, and against its own invariants.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "control_constants.txt")


def golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_mu_values(orc):
    g = golden()
    ref = g["dw_ref"]
    assert orc.mu(0.0, ref) == pytest.approx(1.1)          # exponent 1
    assert orc.mu(ref, ref) == pytest.approx(1.0)          # exponent 0
    assert orc.mu(-5 * ref, ref) == pytest.approx(g["mu_hi"])   # clamped above
    assert orc.mu(10 * ref, ref) == pytest.approx(g["mu_lo"])   # clamped below
    assert orc.mu(2 * ref, ref) == pytest.approx(1 / 1.1)


def test_gamma_schedule(orc):
    g = golden()
    wb = 1.5
    assert orc.gamma_schedule(0.1, wb) == pytest.approx(g["gamma_at_tau_0.1_bins"] * wb)
    assert orc.gamma_schedule(1.0, wb) == pytest.approx(g["gamma_at_tau_1.0_bins"] * wb)
    assert orc.gamma_schedule(0.55, wb) == pytest.approx(8.0 * wb * 10 ** (0.0))


def test_nesterov_sequence(orc):
    a1 = orc.nesterov_a(1.0)
    assert a1 == pytest.approx((1 + math.sqrt(5)) / 2)
    # a_k grows like (k+1)/2
    a = 1.0
    for _ in range(1000):
        a = orc.nesterov_a(a)
    assert 500 < a < 503


def _py_loop(orc, inst, iters, lam0, gamma, amax0_bins=0.044):
    """Plain restatement of the loop in numpy on top of eval_instance."""
    x0, y0, x1, y1 = inst.region
    m = inst.m_mov
    w, h = inst.w[:m].astype(np.float64), inst.h[:m].astype(np.float64)
    lo = np.concatenate([x0 + w / 2, y0 + h / 2]); hi = np.concatenate([x1 - w / 2, y1 - h / 2])
    u = np.clip(np.concatenate([inst.x, inst.y]).astype(np.float64), lo, hi)
    v = u.copy()
    wb = inst.wb
    a, lam, amax0 = 1.0, lam0, amax0_bins * wb
    amax, alpha = amax0, 0.0
    vp = gp = None
    hp_prev = None
    for k in range(iters):
        r = orc.eval_instance(inst, x=v[:m].astype(np.float32), y=v[m:].astype(np.float32), gamma=gamma)
        gN = np.concatenate([r["gNx"], r["gNy"]]); gW = np.concatenate([r["gWx"], r["gWy"]])
        if k == 0 and lam <= 0:
            lam = r["gW_l1"] / r["gN_l1"]
        if k >= 1:
            lam *= orc.mu(r["hpwl"] - hp_prev, 3.5e5)
        hp_prev = r["hpwl"]
        g = gW + lam * gN
        ginf = np.abs(g).max()
        if k == 0:
            alpha = amax0 / ginf
        else:
            dg = np.linalg.norm(g - gp)
            if dg > 0:
                alpha = np.linalg.norm(v - vp) / dg
        alpha = min(alpha, amax / ginf)
        alpha = max(alpha, 0.01 * amax / ginf)
        an = 0.5 * (1 + math.sqrt(1 + 4 * a * a))
        beta = (a - 1) / an
        un = np.clip(v - alpha * g, lo, hi)
        step = np.abs(un - v).max()
        vn = np.clip(un + beta * (un - u), lo, hi)
        vp, gp, u, v, a = v, g, un, vn, an
        amax = max(amax0, 2 * step)
    return u


def test_loop_matches_restatement(orc):
    import synth
    inst = synth.make_instance("tiny")
    for iters in (1, 2, 4):
        x, y, rows, ran = orc.nesterov(inst, iters)
        assert ran == iters
        u = _py_loop(orc, inst, iters, 0.0, inst.gamma)
        np.testing.assert_allclose(np.concatenate([x, y]), u, rtol=0, atol=1e-4)
    # first step moves the farthest cell by alpha_max_0 = 0.044 w_b (unless clamped)
    assert rows[0]["step_max"] == pytest.approx(0.044 * inst.wb, rel=1e-9)


def test_loop_invariants(orc):
    """Positions stay inside the region; density overflow falls and the
    energy N drops over a short run (Fig. 3(a): tau and N move together)."""
    import synth
    inst = synth.make_instance("tiny")
    x, y, rows, ran = orc.nesterov(inst, 60)
    m = inst.m_mov
    assert np.all(x - inst.w[:m] / 2 >= inst.region[0] - 1e-4)
    assert np.all(x + inst.w[:m] / 2 <= inst.region[2] + 1e-4)
    assert np.all(y - inst.h[:m] / 2 >= inst.region[1] - 1e-4)
    assert rows[-1]["tau"] < 0.6 * rows[0]["tau"]
    assert rows[-1]["N"] < 0.5 * rows[0]["N"]
