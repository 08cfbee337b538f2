"""Pins of the oracle's spectral Poisson solve (Section III-E, Eqs. 8-12).

Each test checks the oracle against something other than its own formula:
closed forms of a single cosine mode, invariants the paper states (zero
integral of psi, Neumann boundary, DC removal), symmetry of the energy form,
Parseval, a library DCT, and the PDE itself (-laplacian psi = rho - mean,
E = -grad psi) by finite differences with second-order convergence.
"""
import numpy as np
import pytest
import scipy.fft


def basis(n, k):
    x = np.arange(n)
    return np.cos(np.pi * k * (2 * x + 1) / (2 * n))


def sbasis(n, k):
    x = np.arange(n)
    return np.sin(np.pi * k * (2 * x + 1) / (2 * n))


@pytest.mark.parametrize("n,p,q,L", [(8, 1, 0, 16.0), (16, 3, 5, 32.0), (32, 0, 7, 48.0),
                                     (32, 31, 31, 24.0), (64, 2, 9, 128.0)])
def test_single_mode_closed_form(orc, n, p, q, L):
    """rho = cos(w_p x) cos(w_q y) has a = delta_{pq}, psi = rho/(w_p^2+w_q^2),
    E_x = w_p/(w^2) sin cos, E_y = w_q/(w^2) cos sin (Eqs. 9-12)."""
    rho = np.outer(basis(n, q), basis(n, p))
    a, psi, ex, ey = orc.solve(rho, L, L)
    expect = np.zeros((n, n)); expect[q, p] = 1.0
    np.testing.assert_allclose(a, expect, atol=1e-12)
    wp, wq = np.pi * p / L, np.pi * q / L
    d = wp * wp + wq * wq
    np.testing.assert_allclose(psi, rho / d, atol=1e-12 / d)
    np.testing.assert_allclose(ex, wp / d * np.outer(basis(n, q), sbasis(n, p)), atol=1e-12)
    np.testing.assert_allclose(ey, wq / d * np.outer(sbasis(n, q), basis(n, p)), atol=1e-12)


def test_rectangular_region_units(orc):
    """w_u = pi u / Lx and w_v = pi v / Ly are separate in a non-square region."""
    n, p, q, Lx, Ly = 16, 2, 3, 20.0, 50.0
    rho = np.outer(basis(n, q), basis(n, p))
    _, psi, ex, ey = orc.solve(rho, Lx, Ly)
    wp, wq = np.pi * p / Lx, np.pi * q / Ly
    d = wp * wp + wq * wq
    np.testing.assert_allclose(psi, rho / d, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(ex, wp / d * np.outer(basis(n, q), sbasis(n, p)), atol=1e-12)


def test_constant_density_has_no_field(orc):
    """DC removal (Section III-A): a uniform density gives psi = E = 0."""
    rho = np.full((16, 16), 0.73)
    a, psi, ex, ey = orc.solve(rho, 16.0, 16.0)
    assert np.abs(a).max() < 1e-13
    for f in (psi, ex, ey):
        assert np.abs(f).max() < 1e-13


def test_zero_integral_and_neumann(orc):
    """Eq. 8: the integral of psi vanishes; the normal field vanishes on the
    boundary.  With the mirror at the region edge the sine series of E_x is
    zero at x = 0 and x = L; sampling the same series half a bin outside the
    first and last centres shows it."""
    rng = np.random.default_rng(3)
    n, L = 32, 32.0
    rho = rng.random((n, n))
    a, psi, ex, ey = orc.solve(rho, L, L)
    assert abs(psi.sum()) < 1e-10 * np.abs(psi).sum()
    # evaluate E_x at the left and right region edges from the coefficients
    u = np.arange(n); v = np.arange(n)
    wu = np.pi * u / L; wv = np.pi * v / L
    W = wu[None, :] ** 2 + wv[:, None] ** 2
    W[0, 0] = 1.0
    hat = a / W; hat[0, 0] = 0.0
    yc = (np.arange(n) + 0.5) * L / n
    for xb in (0.0, L):
        exb = np.einsum("vu,u,yv->y", hat * wu[None, :], np.sin(wu * xb), np.cos(np.outer(yc, wv)))
        assert np.abs(exb).max() < 1e-12 * max(1.0, np.abs(ex).max())


def test_scipy_dct_library_pin(orc):
    """The coefficients equal scipy's DCT-II (norm=None: 2 sum x cos) rescaled
    by eps_u eps_v / (4 n^2), with the (0,0) mode dropped."""
    rng = np.random.default_rng(5)
    n = 24
    rho = rng.standard_normal((n, n))
    a = orc.dct_coeffs(rho)
    ref = scipy.fft.dctn(rho, type=2)
    eps = np.where(np.arange(n) == 0, 1.0, 2.0)
    ref = ref * eps[:, None] * eps[None, :] / (4.0 * n * n)
    ref[0, 0] = 0.0
    np.testing.assert_allclose(a, ref, atol=1e-12)


def test_scipy_idct_library_pin(orc):
    """psi is scipy's inverse DCT (type-III) of a/(w_u^2+w_v^2)."""
    rng = np.random.default_rng(6)
    n, Lx, Ly = 16, 24.0, 40.0
    rho = rng.random((n, n))
    a, psi, _, _ = orc.solve(rho, Lx, Ly)
    wu = np.pi * np.arange(n) / Lx; wv = np.pi * np.arange(n) / Ly
    W = wv[:, None] ** 2 + wu[None, :] ** 2
    W[0, 0] = 1.0
    hat = a / W; hat[0, 0] = 0.0
    # scipy dct type 3 norm=None: y[k] = x0 + 2 sum_{n>=1} x_n cos(pi n (2k+1)/2N)
    eps = np.where(np.arange(n) == 0, 1.0, 2.0)
    ref = scipy.fft.dctn(hat / (eps[:, None] * eps[None, :]), type=3)
    np.testing.assert_allclose(psi, ref, atol=1e-12 * np.abs(ref).max())


def test_linearity_and_energy_symmetry(orc):
    """psi is linear in rho and the energy form is symmetric:
    rho1 . psi(rho2) = rho2 . psi(rho1); N >= 0."""
    rng = np.random.default_rng(7)
    n, L = 16, 20.0
    r1, r2 = rng.random((n, n)), rng.random((n, n))
    _, p1, ex1, _ = orc.solve(r1, L, L)
    _, p2, ex2, _ = orc.solve(r2, L, L)
    _, p12, ex12, _ = orc.solve(2.0 * r1 - 3.0 * r2, L, L)
    np.testing.assert_allclose(p12, 2 * p1 - 3 * p2, atol=1e-11)
    np.testing.assert_allclose(ex12, 2 * ex1 - 3 * ex2, atol=1e-11)
    s12, s21 = (r1 * p2).sum(), (r2 * p1).sum()
    assert abs(s12 - s21) < 1e-11 * abs(s12)
    Ab = (L / n) ** 2
    assert orc.energy(r1, p1, Ab) > 0


def test_mirror_symmetry(orc):
    """Mirroring rho in x keeps psi mirrored and flips the sign of E_x."""
    rng = np.random.default_rng(8)
    n, L = 16, 16.0
    rho = rng.random((n, n))
    _, psi, ex, ey = orc.solve(rho, L, L)
    _, psim, exm, eym = orc.solve(rho[:, ::-1], L, L)
    np.testing.assert_allclose(psim, psi[:, ::-1], atol=1e-12)
    np.testing.assert_allclose(exm, -ex[:, ::-1], atol=1e-12)
    np.testing.assert_allclose(eym, ey[:, ::-1], atol=1e-12)


def test_parseval_energy(orc):
    """N = 1/2 A_b sum_b rho psi = 1/2 A_b sum_uv (n^2/(eps_u eps_v)) a^2/(w^2)."""
    rng = np.random.default_rng(9)
    n, Lx, Ly = 32, 48.0, 40.0
    rho = rng.random((n, n))
    a, psi, _, _ = orc.solve(rho, Lx, Ly)
    Ab = (Lx / n) * (Ly / n)
    N = orc.energy(rho, psi, Ab)
    eps = np.where(np.arange(n) == 0, 1.0, 2.0)
    wu = np.pi * np.arange(n) / Lx; wv = np.pi * np.arange(n) / Ly
    W = wv[:, None] ** 2 + wu[None, :] ** 2
    W[0, 0] = np.inf
    Np = 0.5 * Ab * np.sum(n * n / (eps[:, None] * eps[None, :]) * a * a / W)
    assert abs(N - Np) < 1e-10 * abs(N)


def _smooth_rho(n, L):
    c = (np.arange(n) + 0.5) * L / n
    X, Y = np.meshgrid(c, c)
    return np.exp(-((X - 0.37 * L) ** 2 + (Y - 0.58 * L) ** 2) / (2 * (0.12 * L) ** 2)) \
        + 0.5 * np.exp(-((X - 0.7 * L) ** 2 + (Y - 0.3 * L) ** 2) / (2 * (0.08 * L) ** 2))


def test_poisson_residual_second_order(orc):
    """Eq. 8: -laplacian psi = rho - mean(rho) (DC removed).  The 5-point
    stencil with mirrored (Neumann) ghost cells has an O(h^2) residual, so
    halving the bin width divides it by about 4; and E = -grad psi, checked
    with central differences at the same order."""
    L = 10.0
    res, eres = [], []
    for n in (32, 64, 128):
        rho = _smooth_rho(n, L)
        _, psi, ex, ey = orc.solve(rho, L, L)
        h = L / n
        P = np.pad(psi, 1, mode="symmetric")
        lap = (P[1:-1, 2:] + P[1:-1, :-2] + P[2:, 1:-1] + P[:-2, 1:-1] - 4 * P[1:-1, 1:-1]) / (h * h)
        r = -lap - (rho - rho.mean())
        res.append(np.abs(r[4:-4, 4:-4]).max())
        dpsi_dx = (psi[:, 2:] - psi[:, :-2]) / (2 * h)
        dpsi_dy = (psi[2:, :] - psi[:-2, :]) / (2 * h)
        eres.append(max(np.abs(ex[:, 1:-1] + dpsi_dx).max(), np.abs(ey[1:-1, :] + dpsi_dy).max()))
    assert res[0] / res[1] > 3.3 and res[1] / res[2] > 3.3, res
    assert eres[0] / eres[1] > 3.3 and eres[1] / eres[2] > 3.3, eres
    assert res[2] < 2e-3 * np.abs(_smooth_rho(128, L)).max()


def test_energy_decreases_when_spread(orc):
    """Spreading a lump lowers the energy N (the equilibrium of Section III-A
    has zero energy at uniform density)."""
    n, L = 32, 32.0
    lump = np.zeros((n, n)); lump[12:20, 12:20] = 4.0
    spread = np.zeros((n, n)); spread[8:24, 8:24] = 1.0
    Ab = (L / n) ** 2
    Ns = []
    for r in (lump, spread, np.full((n, n), 0.25)):
        _, psi, _, _ = orc.solve(r, L, L)
        Ns.append(orc.energy(r, psi, Ab))
    assert Ns[0] > Ns[1] > 0 and abs(Ns[2]) < 1e-9 * Ns[1]


@pytest.mark.parametrize("n,Lx,Ly", [(8, 16.0, 16.0), (16, 20.0, 50.0), (32, 48.0, 24.0)])
def test_potential_at_equals_full_field(orc, n, Lx, Ly):
    """orc_potential_at (the pointwise series used to check large grids)
    agrees with the full-map series at every bin of small grids, for random
    coefficients with a nonzero (0,0) entry that both must ignore, in a
    non-square region (w_u and w_v differ): a swapped sine/cosine or axis, a
    kept (0,0) term or a wrong divisor would differ by O(1)."""
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n))
    a[0, 0] = 5.0
    psi, ex, ey = orc.potential_field(a, Lx, Ly)
    ys, xs = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    p, qx, qy = orc.potential_at(a, Lx, Ly, xs.ravel(), ys.ravel())
    scale = max(np.abs(psi).max(), np.abs(ex).max(), np.abs(ey).max())
    for got, ref in ((p, psi), (qx, ex), (qy, ey)):
        assert np.abs(got - ref.ravel()).max() <= 1e-13 * scale


@pytest.mark.parametrize("p,q", [(3, 0), (0, 5), (7, 11), (255, 1)])
def test_potential_at_single_mode_large_grid(orc, p, q):
    """n = 256 with a single coefficient a[q][p] = 1: at sampled bins psi,
    E_x and E_y equal the closed forms of Eqs. 11-12 for one mode."""
    n, Lx, Ly = 256, 384.0, 192.0
    a = np.zeros((n, n))
    a[q, p] = 1.0
    rng = np.random.default_rng(p * 1000 + q)
    xs = rng.integers(0, n, 40); ys = rng.integers(0, n, 40)
    psi, ex, ey = orc.potential_at(a, Lx, Ly, xs, ys)
    wp, wq = np.pi * p / Lx, np.pi * q / Ly
    d = wp * wp + wq * wq
    cx, sx = basis(n, p)[xs], sbasis(n, p)[xs]
    cy, sy = basis(n, q)[ys], sbasis(n, q)[ys]
    np.testing.assert_allclose(psi, cx * cy / d, rtol=0, atol=1e-12 / d)
    np.testing.assert_allclose(ex, wp / d * sx * cy, rtol=0, atol=1e-12 / d)
    np.testing.assert_allclose(ey, wq / d * cx * sy, rtol=0, atol=1e-12 / d)
