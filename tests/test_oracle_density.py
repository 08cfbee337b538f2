"""Pins of the oracle's density map, field gather, exact adjoint and overflow.

The density map (Section II bin density; Section III charges q_i = A_i) is
checked against exact rational arithmetic over every bin, against area
conservation and the one-bin case; the gather (q.E of Eq. 7) against its
adjoint relation with the scatter; the edge-difference derivative against
central finite differences of the binned energy N (Eq. 6), which are exact
because N is quadratic in rho and rho is linear in a cell's position between
bin crossings.
"""
from fractions import Fraction

import numpy as np
import pytest


def f32(v):
    return np.float32(v)


def exact_edges(x, w):
    h = f32(0.5) * f32(w)
    return Fraction(float(f32(x) - h)), Fraction(float(f32(x) + h))


def brute_area(region, n, x, y, w, h):
    """Exact overlap of every cell with every bin, rational arithmetic."""
    x0, y0, x1, y1 = [Fraction(v) for v in region]
    wb, hb = (x1 - x0) / n, (y1 - y0) / n
    area = [[Fraction(0)] * n for _ in range(n)]
    touched = []
    for i in range(len(x)):
        xl, xh = exact_edges(x[i], w[i])
        yl, yh = exact_edges(y[i], h[i])
        t = set()
        for j in range(n):
            oy = min(yh, y0 + (j + 1) * hb) - max(yl, y0 + j * hb)
            if oy <= 0:
                continue
            for k in range(n):
                ox = min(xh, x0 + (k + 1) * wb) - max(xl, x0 + k * wb)
                if ox <= 0:
                    continue
                area[j][k] += ox * oy
                t.add((j, k))
        touched.append(t)
    return area, touched


def edge_cases(region, n):
    """Cells on bin edges, on the region boundary, partly or wholly outside,
    wider than many bins, and tiny."""
    x0, y0, x1, y1 = region
    wb = (x1 - x0) / n
    xs = [x0 + 1.0 * wb, x0 + 0.5, x1 - 0.5, x0 - 0.3, x1 + 5.0, 0.5 * (x0 + x1), x0 + 2.5 * wb, x0 + 3 * wb + 1e-3]
    ws = [2 * wb, 1.0, 1.0, 1.0, 1.0, 6.5 * wb, 1e-3, wb]
    ys = [y0 + 1.0 * wb, y0 + 0.5, y1 - 0.5, y0 + 3.0, y0 + 3.0, y0 + wb, y0 + 2.5 * wb, y1 - 0.25]
    hs = [wb, 1.0, 1.0, 2.0, 2.0, 1.0, 1e-3, 1.0]
    return [np.array(v, np.float32) for v in (xs, ys, ws, hs)]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_density_exact_rational(orc, seed):
    """Overlap areas and bin ranges agree with exact rational arithmetic,
    including cells on bin edges and outside the region."""
    rng = np.random.default_rng(seed)
    n, region = 8, (0.0, 0.0, 12.0, 12.0)
    m = 40
    x = rng.uniform(-2, 14, m).astype(np.float32)
    y = rng.uniform(-2, 14, m).astype(np.float32)
    w = rng.uniform(0.1, 7.0, m).astype(np.float32)
    h = rng.uniform(0.1, 3.0, m).astype(np.float32)
    ex, ey, ew, eh = edge_cases(region, n)
    x, y, w, h = [np.concatenate([a, b]) for a, b in ((x, ex), (y, ey), (w, ew), (h, eh))]
    area, touched = brute_area(region, n, x, y, w, h)
    D = orc.overlap_map(region, n, x, y, w, h)
    ref = np.array([[float(v) for v in row] for row in area])
    np.testing.assert_allclose(D, ref, rtol=1e-14, atol=1e-14)
    ranges, pairs = orc.bin_ranges(region, n, x, y, w, h)
    total = 0
    for i, t in enumerate(touched):
        ilo, ihi, jlo, jhi = ranges[i]
        got = {(j, k) for j in range(jlo, jhi + 1) for k in range(ilo, ihi + 1)}
        assert got == t, (i, ranges[i], sorted(t))
        total += len(t)
    assert pairs == total


def test_rectangular_bins(orc):
    """A region with different x and y bin sizes and an offset origin."""
    rng = np.random.default_rng(11)
    n, region = 4, (-3.0, 5.0, 9.0, 7.0)
    x = rng.uniform(-4, 10, 20).astype(np.float32)
    y = rng.uniform(4.5, 7.5, 20).astype(np.float32)
    w = rng.uniform(0.1, 5, 20).astype(np.float32)
    h = rng.uniform(0.05, 1, 20).astype(np.float32)
    area, _ = brute_area(region, n, x, y, w, h)
    D = orc.overlap_map(region, n, x, y, w, h)
    np.testing.assert_allclose(D, np.array([[float(v) for v in r] for r in area]), atol=1e-14)


def test_area_conservation_and_one_bin(orc):
    """Cells inside the region deposit exactly their area; a cell inside one
    bin gives rho = q / A_b there and zero elsewhere."""
    import synth
    inst = synth.make_instance("tiny")
    rho, D, F = orc.density(inst.region, inst.n, 1.0, inst.x, inst.y, inst.w, inst.h)
    # the deposited area is that of the float32-rounded rectangle
    hw, hh = np.float32(0.5) * inst.w, np.float32(0.5) * inst.h
    q = float(np.sum(((inst.x + hw).astype(np.float64) - (inst.x - hw)) *
                           ((inst.y + hh).astype(np.float64) - (inst.y - hh))))
    assert abs(q - float(np.sum(inst.w.astype(np.float64) * inst.h))) < 1e-6 * q
    assert abs(D.sum() - q) < 1e-12 * q
    Ab = inst.wb * inst.hb
    assert abs(rho.sum() * Ab - q) < 1e-9 * q
    x = np.array([5.0], np.float32); y = np.array([3.0], np.float32)
    w = np.array([1.5], np.float32); h = np.array([1.0], np.float32)
    rho1, _, _ = orc.density((0, 0, 16, 16), 8, 1.0, x, y, w, h)
    assert rho1[1, 2] == pytest.approx(1.5 / 4.0, abs=1e-15)
    assert np.count_nonzero(rho1) == 1


def test_fixed_area_scaled_by_target_density(orc):
    """Section III-B: fixed (macro) area enters rho scaled by rho_t."""
    region, n = (0, 0, 8, 8), 4
    x = np.array([1.0], np.float32); y = np.array([1.0], np.float32)
    w = np.array([2.0], np.float32); h = np.array([2.0], np.float32)
    fx = np.array([5.0], np.float32); fy = np.array([5.0], np.float32)
    fw = np.array([2.0], np.float32); fh = np.array([2.0], np.float32)
    rho, D, F = orc.density(region, n, 0.9, x, y, w, h, fx, fy, fw, fh)
    assert rho[0, 0] == pytest.approx(1.0)
    assert rho[2, 2] == pytest.approx(0.9)
    assert F[2, 2] == pytest.approx(4.0) and D[2, 2] == 0.0


def test_quantised_map_matches_and_is_order_free(orc):
    """The int64 fixed-point map equals the FP64 map to float32 accuracy and
    does not depend on cell order."""
    import synth
    inst = synth.make_instance("medium")
    m = inst.m_mov
    Q = orc.overlap_map_q(inst.region, inst.n, inst.x, inst.y, inst.w[:m], inst.h[:m])
    D = orc.overlap_map(inst.region, inst.n, inst.x, inst.y, inst.w[:m], inst.h[:m])
    np.testing.assert_allclose(Q * 2.0 ** -32, D, rtol=3e-7, atol=1e-9)
    perm = np.random.default_rng(0).permutation(m)
    Q2 = orc.overlap_map_q(inst.region, inst.n, inst.x[perm], inst.y[perm],
                           inst.w[:m][perm], inst.h[:m][perm])
    assert np.array_equal(Q, Q2)


def test_gather_is_adjoint_of_scatter(orc):
    """sum_b D_b(x) phi_b = -sum_i gather_i(phi): the gather uses exactly the
    scatter's weights (q.E of Eq. 7 with E averaged over the overlap)."""
    import synth
    inst = synth.make_instance("tiny")
    rng = np.random.default_rng(1)
    phx = rng.standard_normal((inst.n, inst.n))
    phy = rng.standard_normal((inst.n, inst.n))
    D = orc.overlap_map(inst.region, inst.n, inst.x, inst.y, inst.w, inst.h)
    gx, gy = orc.gather(inst.region, inst.n, inst.x, inst.y, inst.w, inst.h, phx, phy)
    assert abs((D * phx).sum() + gx.sum()) < 1e-10 * np.abs(gx).sum()
    assert abs((D * phy).sum() + gy.sum()) < 1e-10 * np.abs(gy).sum()


def test_gather_single_bin_cell(orc):
    """A cell covering exactly one bin feels -A_b E_b."""
    n, region = 8, (0.0, 0.0, 16.0, 16.0)
    rng = np.random.default_rng(2)
    ex, ey = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    x = np.array([7.0], np.float32); y = np.array([11.0], np.float32)
    w = np.array([2.0], np.float32); h = np.array([2.0], np.float32)
    gx, gy = orc.gather(region, n, x, y, w, h, ex, ey)
    assert gx[0] == pytest.approx(-4.0 * ex[5, 3]) and gy[0] == pytest.approx(-4.0 * ey[5, 3])


def _energy(orc, region, n, x, y, w, h, fx=None, fy=None, fw=None, fh=None, rho_t=1.0):
    rho, _, _ = orc.density(region, n, rho_t, x, y, w, h, fx, fy, fw, fh)
    L = region[2] - region[0]
    _, psi, _, _ = orc.solve(rho, L, region[3] - region[1])
    return orc.energy(rho, psi, (L / n) * ((region[3] - region[1]) / n)), rho, psi


def test_adjoint_equals_central_differences(orc):
    """The edge-difference gradient is the exact derivative of the binned N.
    Positions, sizes and the step are dyadic, so every shifted edge is exact
    in float32, and no edge crosses a bin edge within the step: the central
    difference of the quadratic N is then exact up to FP64 rounding."""
    rng = np.random.default_rng(4)
    n, L = 16, 32.0
    region = (0.0, 0.0, L, L)
    m = 60
    x = (rng.integers(64, 30 * 64, m) / 64.0).astype(np.float32)
    y = (rng.integers(64, 30 * 64, m) / 64.0).astype(np.float32)
    w = (rng.integers(1, 12, m) / 2.0).astype(np.float32)
    h = np.ones(m, np.float32)
    step = 1.0 / 256.0
    wb = L / n
    N0, rho, psi = _energy(orc, region, n, x, y, w, h)
    gx, gy = orc.adjoint(region, n, x, y, w, h, psi)
    checked = 0
    for i in range(m):
        edges = [float(x[i] - w[i] / 2), float(x[i] + w[i] / 2), float(y[i] - h[i] / 2), float(y[i] + h[i] / 2)]
        if any(abs(e / wb - round(e / wb)) * wb < 2 * step for e in edges):
            continue
        for axis, g in ((0, gx), (1, gy)):
            xp, xm, yp, ym = x.copy(), x.copy(), y.copy(), y.copy()
            if axis == 0:
                xp[i] += step; xm[i] -= step
            else:
                yp[i] += step; ym[i] -= step
            Np, _, _ = _energy(orc, region, n, xp, yp, w, h)
            Nm, _, _ = _energy(orc, region, n, xm, ym, w, h)
            fd = (Np - Nm) / (2 * step)
            assert abs(fd - g[i]) <= 1e-8 * max(1.0, abs(N0)) / step * 1e-3 + 1e-9 * abs(g[i]), (i, axis, fd, g[i])
            checked += 1
    assert checked >= 40


def test_gather_approaches_adjoint_for_smooth_fields(orc):
    """The paper's q.E gather is not the exact derivative of the binned N, but
    on a smooth background (one cosine mode) their gap shrinks with the bin
    width at first order."""
    gaps = []
    for n in (16, 32, 64):
        L = 32.0
        c = np.arange(n)
        rho = 1.0 + 0.5 * np.outer(np.cos(np.pi * 1 * (2 * c + 1) / (2 * n)),
                                   np.cos(np.pi * 2 * (2 * c + 1) / (2 * n)))
        _, psi, ex, ey = orc.solve(rho, L, L)
        rng = np.random.default_rng(0)
        x = rng.uniform(4, 28, 50).astype(np.float32)
        y = rng.uniform(4, 28, 50).astype(np.float32)
        w = np.full(50, 3.0, np.float32); h = np.full(50, 3.0, np.float32)
        gx, _ = orc.gather((0, 0, L, L), n, x, y, w, h, ex, ey)
        ax, _ = orc.adjoint((0, 0, L, L), n, x, y, w, h, psi)
        gaps.append(np.linalg.norm(gx - ax) / np.linalg.norm(ax))
    assert gaps[0] > gaps[1] > gaps[2] and gaps[2] < 0.1, gaps


def test_overflow_hand_example(orc):
    """tau = sum_b max(0, D_b - rho_t (A_b - F_b)) / sum q on a 2x2 grid."""
    region, n = (0, 0, 4, 4), 2
    # two 2x2 cells stacked on bin (0,0), one 2x1 cell in bin (1,1), a 2x1 macro in bin (1,1)
    x = np.array([1, 1, 3], np.float32); y = np.array([1, 1, 2.5], np.float32)
    w = np.array([2, 2, 2], np.float32); h = np.array([2, 2, 1], np.float32)
    fx = np.array([3], np.float32); fy = np.array([3.5], np.float32)
    fw = np.array([2], np.float32); fh = np.array([1], np.float32)
    for rho_t, expect in ((1.0, (8 - 4) / 10.0), (0.5, ((8 - 2) + (2 - 0.5 * 2)) / 10.0)):
        _, D, F = orc.density(region, n, rho_t, x, y, w, h, fx, fy, fw, fh)
        tau = orc.overflow(D, F, 4.0, rho_t, 10.0)
        assert tau == pytest.approx(expect, abs=1e-15)
