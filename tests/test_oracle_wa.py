"""Pins of the oracle's wirelength (Eq. 1 HPWL, Eq. 3 weighted-average model).

Checked against: the two-pin closed form derived from Eq. 3
(W~ = |d| tanh(|d| / 2 gamma)); the bound W~ <= HPWL and convergence to HPWL
as gamma -> 0 (stated after Eq. 3); translation invariance (the pin gradient
sums to zero); homogeneity W~(c p; c gamma) = c W~(p; gamma); coincident pins;
and central finite differences on a dyadic grid where every perturbed pin
coordinate is exact in float32.
"""
import numpy as np
import pytest


def one_net(px, py=None):
    """A single net whose pins sit on distinct movable cells at the given
    centres with zero offsets."""
    d = len(px)
    py = np.zeros(d) if py is None else py
    return (np.array([0, d], np.int32), np.arange(d, dtype=np.int32),
            np.zeros(d, np.float32), np.zeros(d, np.float32),
            np.asarray(px, np.float32), np.asarray(py, np.float32))


@pytest.mark.parametrize("d,g", [(0.5, 1.0), (3.0, 0.75), (10.0, 2.0), (1e-3, 1.0), (7.25, 0.1)])
def test_two_pin_closed_form(orc, d, g):
    net_ptr, pc, dx, dy, x, y = one_net([1.0, 1.0 + d])
    r = orc.wa(net_ptr, pc, dx, dy, 2, x, y, g, per_pin=True)
    dd = float(np.float32(1.0 + d) - np.float32(1.0))
    t = np.tanh(dd / (2 * g))
    assert r["W"] == pytest.approx(dd * t, rel=1e-13, abs=1e-14)
    dW = t + dd / (2 * g) * (1 - t * t)
    assert r["gpx"][1] == pytest.approx(dW, rel=1e-12, abs=1e-14)
    assert r["gpx"][0] == pytest.approx(-dW, rel=1e-12, abs=1e-14)
    assert r["hpwl"] == pytest.approx(dd, rel=1e-15)


def test_bound_and_limit(orc):
    """W~ <= HPWL for every net and W~ -> HPWL as gamma -> 0 (Section II)."""
    import synth
    inst = synth.make_instance("tiny")
    prev = None
    for g in (4.0, 1.0, 0.25, 0.05, 0.01):
        r = orc.wa(inst.net_ptr, inst.pin_cell, inst.pin_dx, inst.pin_dy, inst.m_mov,
                   inst.x, inst.y, g)
        assert r["W"] <= r["hpwl"] * (1 + 1e-12)
        gap = r["hpwl"] - r["W"]
        if prev is not None:
            assert gap < prev
        prev = gap
    assert prev < 1e-3 * r["hpwl"]


def test_translation_invariance_and_homogeneity(orc):
    rng = np.random.default_rng(0)
    for deg in (2, 3, 7, 50):
        px = rng.uniform(0, 40, deg); py = rng.uniform(0, 40, deg)
        net_ptr, pc, dx, dy, x, y = one_net(px, py)
        r = orc.wa(net_ptr, pc, dx, dy, deg, x, y, 1.5, per_pin=True)
        assert abs(r["gpx"].sum()) < 1e-12 * np.abs(r["gpx"]).sum()
        assert abs(r["gpy"].sum()) < 1e-12 * np.abs(r["gpy"]).sum()
        # homogeneity with a power-of-two scale keeps float32 coordinates exact
        r2 = orc.wa(net_ptr, pc, dx, dy, deg, x * 4, y * 4, 6.0)
        assert r2["W"] == pytest.approx(4 * r["W"], rel=1e-13)


def test_coincident_pins_and_degree_one(orc):
    net_ptr, pc, dx, dy, x, y = one_net([3.0] * 5, [7.0] * 5)
    r = orc.wa(net_ptr, pc, dx, dy, 5, x, y, 0.5, per_pin=True)
    assert r["W"] == 0.0 and np.all(r["gpx"] == 0) and np.all(r["gpy"] == 0)
    net_ptr = np.array([0, 1, 3], np.int32)
    pc = np.array([0, 1, 2], np.int32)
    z = np.zeros(3, np.float32)
    x = np.array([5.0, 1.0, 4.0], np.float32)
    r = orc.wa(net_ptr, pc, z, z, 3, x, z, 1.0)
    assert r["net_w"][0] == 0.0 and r["gcx"][0] == 0.0
    assert r["gcx"][1] == pytest.approx(-r["gcx"][2])


def test_finite_differences(orc):
    """Central differences with dyadic coordinates and step: every perturbed
    pin coordinate is exact in float32, so the only error is O(h^2)."""
    rng = np.random.default_rng(2)
    m, E = 30, 12
    deg = rng.integers(2, 8, E)
    net_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    P = int(net_ptr[-1])
    pc = rng.integers(0, m, P).astype(np.int32)
    dx = (rng.integers(-8, 9, P) / 16.0).astype(np.float32)
    dy = (rng.integers(-8, 9, P) / 16.0).astype(np.float32)
    x = (rng.integers(0, 512, m) / 32.0).astype(np.float32)
    y = (rng.integers(0, 512, m) / 32.0).astype(np.float32)
    g = 1.25
    r = orc.wa(net_ptr, pc, dx, dy, m, x, y, g)
    h = 2.0 ** -9
    for i in range(m):
        for arr, grad in ((x, r["gcx"]), (y, r["gcy"])):
            old = arr[i]
            arr[i] = old + h
            wp = orc.wa(net_ptr, pc, dx, dy, m, x, y, g)["W"]
            arr[i] = old - h
            wm = orc.wa(net_ptr, pc, dx, dy, m, x, y, g)["W"]
            arr[i] = old
            fd = (wp - wm) / (2 * h)
            assert abs(fd - grad[i]) < 1e-6 * max(1.0, abs(grad[i])), (i, fd, grad[i])


def test_macro_pins_use_fixed_positions(orc):
    """A pin on a fixed cell reads the macro centre and sends no gradient to
    any movable cell."""
    net_ptr = np.array([0, 2], np.int32)
    pc = np.array([0, 3], np.int32)  # m_mov = 3, so 3 is macro 0
    z = np.zeros(2, np.float32)
    x = np.array([1.0, 50.0, 50.0], np.float32)
    y = np.zeros(3, np.float32)
    r = orc.wa(net_ptr, pc, z, z, 3, x, y, 1.0, fx=np.array([9.0], np.float32),
               fy=np.array([0.0], np.float32))
    assert r["hpwl"] == pytest.approx(8.0)
    assert r["gcx"][1] == 0.0 and r["gcx"][2] == 0.0 and r["gcx"][0] < 0
