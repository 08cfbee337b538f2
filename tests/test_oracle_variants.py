"""Pins for the oracle's model variants: the log-sum-exp wirelength that
Section II names, and the Helmholtz smoothing of Eq. 4.

LSE per net and axis: g ln sum exp(p/g) + g ln sum exp(-p/g) (the usual
definition; the paper gives no formula).  Pinned by the two-pin closed form
|d| + 2g ln(1 + exp(-|d|/g)) with gradient tanh(d / 2g), by
span <= LSE <= span + 2g ln(deg), by translation invariance (gradients of a
net sum to zero), by the g -> 0 limit (HPWL) and by central differences.

Helmholtz (laplacian psi - eps psi = -rho, Neumann): every cosine mode is
divided by w_u^2 + w_v^2 + eps, so a single mode and a constant have exact
solutions, and eps -> 0 gives the Poisson solution of a zero-mean density.
"""
import math

import numpy as np
import pytest

import oracle


def two_pin(x1, x2, y=5.0):
    return dict(net_ptr=np.array([0, 2], np.int32), pin_cell=np.array([0, 1], np.int32),
                dx=np.zeros(2, np.float32), dy=np.zeros(2, np.float32), m_mov=2,
                x=np.array([x1, x2], np.float32), y=np.array([y, y], np.float32))


@pytest.mark.parametrize("d,g", [(3.0, 1.0), (0.25, 2.0), (-7.5, 0.5), (0.0, 1.5)])
def test_lse_two_pins_closed_form(d, g):
    net = two_pin(10.0 + d, 10.0)
    r = oracle.wa(**net, gamma=g, model=oracle.WL_LSE)
    ad = abs(d)
    # x axis: |d| + 2g ln(1 + e^{-|d|/g}); y axis (coincident): 2g ln 2
    want = ad + 2 * g * math.log1p(math.exp(-ad / g)) + 2 * g * math.log(2.0)
    assert r["W"] == pytest.approx(want, rel=1e-13, abs=1e-13)
    t = math.tanh(d / (2 * g))
    assert r["gcx"][0] == pytest.approx(t, abs=1e-13)
    assert r["gcx"][1] == pytest.approx(-t, abs=1e-13)
    assert abs(r["gcy"][0]) < 1e-15 and abs(r["gcy"][1]) < 1e-15
    assert r["hpwl"] == pytest.approx(ad, abs=1e-12)


def random_nets(seed, E=60, m=40, dmax=9):
    rng = np.random.default_rng(seed)
    deg = rng.integers(2, dmax + 1, E)
    net_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    pin_cell = np.concatenate([rng.choice(m, d, replace=False) for d in deg]).astype(np.int32)
    P = pin_cell.size
    return dict(net_ptr=net_ptr, pin_cell=pin_cell,
                dx=rng.uniform(-0.5, 0.5, P).astype(np.float32),
                dy=rng.uniform(-0.5, 0.5, P).astype(np.float32), m_mov=m,
                x=rng.uniform(0, 50, m).astype(np.float32),
                y=rng.uniform(0, 50, m).astype(np.float32)), deg


def test_lse_bounds_and_invariance():
    net, deg = random_nets(3)
    g = 1.7
    r = oracle.wa(**net, gamma=g, model=oracle.WL_LSE, per_pin=True)
    hp = oracle.wa(**net, gamma=1e-9, model=oracle.WL_WA)  # per-net spans via a tiny-g WA
    spans = hp["net_w"]
    # span <= LSE_e <= span + 2 g ln(deg) per axis (two axes)
    assert np.all(r["net_w"] >= spans - 1e-9)
    assert np.all(r["net_w"] <= spans + 4 * g * np.log(deg) + 1e-9)
    # the gradients of each net sum to zero along each axis
    for e in range(len(deg)):
        b, c = net["net_ptr"][e], net["net_ptr"][e + 1]
        assert abs(r["gpx"][b:c].sum()) < 1e-12 and abs(r["gpy"][b:c].sum()) < 1e-12
        # and each lies in [-1, 1] (a difference of two softmax weights)
        assert np.all(np.abs(r["gpx"][b:c]) <= 1 + 1e-15)


def test_lse_tends_to_hpwl():
    net, deg = random_nets(4)
    hp = oracle.wa(**net, gamma=1.0)["hpwl"]
    prev = None
    for g in (1.0, 0.1, 0.01, 0.001):
        w = oracle.wa(**net, gamma=g, model=oracle.WL_LSE)["W"]
        assert w >= hp - 1e-9
        err = w - hp
        assert err <= 4 * g * np.log(deg).sum() + 1e-9
        if prev is not None:
            assert err < prev
        prev = err


def test_lse_gradient_matches_central_differences():
    net, _ = random_nets(5, E=30, m=20)
    g = 2.0
    r = oracle.wa(**net, gamma=g, model=oracle.WL_LSE)
    h = 1.0 / 64  # exact in float32 at these magnitudes
    for c in range(0, 20, 3):
        for axis in ("x", "y"):
            lo = dict(net); hi = dict(net)
            lo[axis] = net[axis].copy(); hi[axis] = net[axis].copy()
            lo[axis][c] -= h; hi[axis][c] += h
            fd = (oracle.wa(**hi, gamma=g, model=oracle.WL_LSE)["W"] -
                  oracle.wa(**lo, gamma=g, model=oracle.WL_LSE)["W"]) / (2 * h)
            an = r["gcx" if axis == "x" else "gcy"][c]
            # central difference error O(h^2 / g^2) relative to the gradient scale
            assert fd == pytest.approx(an, abs=2e-4)


def mode(n, u, v):
    x = np.arange(n)
    cu = np.cos(np.pi * u * (2 * x + 1) / (2 * n))
    cv = np.cos(np.pi * v * (2 * x + 1) / (2 * n))
    return np.outer(cv, cu)  # [y][x]


@pytest.mark.parametrize("u,v", [(1, 0), (3, 5), (0, 7), (15, 15)])
def test_helmholtz_single_mode(u, v):
    n, Lx, Ly, eps = 16, 24.0, 40.0, 0.03
    rho = mode(n, u, v)
    _, psi, ex, ey = oracle.solve(rho, Lx, Ly, eps)
    wu, wv = np.pi * u / Lx, np.pi * v / Ly
    d = wu * wu + wv * wv + eps
    x = np.arange(n)
    su = np.sin(np.pi * u * (2 * x + 1) / (2 * n))
    sv = np.sin(np.pi * v * (2 * x + 1) / (2 * n))
    cu = np.cos(np.pi * u * (2 * x + 1) / (2 * n))
    cv = np.cos(np.pi * v * (2 * x + 1) / (2 * n))
    np.testing.assert_allclose(psi, rho / d, rtol=0, atol=1e-12 / d)
    np.testing.assert_allclose(ex, wu * np.outer(cv, su) / d, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ey, wv * np.outer(sv, cu) / d, rtol=0, atol=1e-12)


def test_helmholtz_constant_density():
    n, eps = 32, 0.25
    rho = np.full((n, n), 1.7)
    _, psi, ex, ey = oracle.solve(rho, 48.0, 48.0, eps)
    np.testing.assert_allclose(psi, 1.7 / eps, rtol=1e-13)
    assert np.abs(ex).max() < 1e-12 and np.abs(ey).max() < 1e-12


def test_helmholtz_small_eps_is_poisson():
    rng = np.random.default_rng(9)
    n = 32
    rho = rng.random((n, n))
    rho -= rho.mean()                      # zero mean: no (0,0) mode
    _, p0, x0, y0 = oracle.solve(rho, 40.0, 40.0)
    _, p1, x1, y1 = oracle.solve(rho, 40.0, 40.0, 1e-10)
    # smallest divisor (pi/40)^2 ~ 6e-3: relative change ~ eps / 6e-3
    for a, b in ((p0, p1), (x0, x1), (y0, y1)):
        assert np.abs(a - b).max() <= 1e-7 * np.abs(a).max()


def test_eval_variants_run_and_differ():
    import synth
    inst = synth.make_instance("tiny")
    base = oracle.eval_instance(inst, maps=True)
    lse = oracle.eval_instance(inst, maps=True, wirelength=oracle.WL_LSE)
    hel = oracle.eval_instance(inst, maps=True, helmholtz_eps=1e-3)
    # LSE >= HPWL >= WA (WA underestimates, LSE overestimates)
    assert lse["W"] >= base["hpwl"] >= base["W"]
    assert lse["hpwl"] == base["hpwl"]
    # the density side does not depend on the wirelength model
    np.testing.assert_array_equal(lse["gNx"], base["gNx"])
    # Helmholtz: N = 1/2 A_b sum rho psi with the DC mode kept
    Ab = (inst.region[2] - inst.region[0]) * (inst.region[3] - inst.region[1]) / inst.n ** 2
    assert hel["N"] == pytest.approx(0.5 * Ab * float((hel["rho"] * hel["psi"]).sum()), rel=1e-12)
    assert hel["N"] > base["N"]
