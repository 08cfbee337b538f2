"""Pins of the oracle's Nesterov loop (orc_nesterov_run, the loop behind
orc_nesterov) on objectives whose iterates can be worked out by hand.

Section IV-A and Algorithm 1 fix the control: alpha_max_0 bounds the first
move, the Barzilai-Borwein ratio ||dv|| / ||dg|| gives the later steps (on a
quadratic with curvature c it is exactly 1/c), alpha ||g||_inf is kept in
[0.01 alpha_max, alpha_max] with alpha_max doubling the last move, the
penalty grows by mu = 1.1^(1 - dW/dw_ref) with dW the HPWL change between the
evaluated points, and gamma follows the overflow of the previous point.
Every expected value below is written out step by step from those rules and
Nesterov's sequence a_{k+1} = (1 + sqrt(1 + 4 a_k^2)) / 2; none comes from
running a loop.
"""
import math

import numpy as np
import pytest

PHI = (1 + math.sqrt(5)) / 2                # a_1
A2 = (1 + math.sqrt(1 + 4 * PHI ** 2)) / 2  # a_2
A3 = (1 + math.sqrt(1 + 4 * A2 ** 2)) / 2   # a_3
B1 = (PHI - 1) / A2                         # beta_1 (beta_0 = 0 since a_0 = 1)
B2 = (A2 - 1) / A3


def quad(c, lam_grad=0.0, hpwl=lambda v: 0.0, tau=lambda v: 0.5):
    """f = c v^2 / 2 as the wirelength, lam_grad * v as the density gradient."""
    def objective(v, gamma):
        gW = c * v
        gN = lam_grad * v
        return dict(gW=gW, gN=gN, W=0.5 * c * float(v @ v), hpwl=hpwl(v), N=0.0, tau=tau(v),
                    gW_l1=float(np.abs(gW).sum()), gN_l1=float(np.abs(gN).sum()))
    return objective


def test_quadratic_steps(orc):
    """c = 2 from x_0 = 10, alpha_max_0 = 1:
    k=0: g = 20, alpha = 1/20, u_1 = 9 = v_1 (beta_0 = 0), move 1 -> alpha_max 2
    k=1: g = 18, BB ratio 1/2 but alpha g = 9 > 2: alpha = 2/18, u_2 = 7,
         v_2 = 7 + beta_1 (7 - 9), move 2 -> alpha_max 4
    k=2: g = 2 v_2, alpha g = v_2 > 4: alpha = 4 / g, u_3 = v_2 - 4,
         v_3 = u_3 + beta_2 (u_3 - u_2), move 4 -> alpha_max 8
    k=3: g = 2 v_3 with v_3 < 8: the BB ratio 1/2 stands, u_4 = v_3 - v_3 = 0."""
    u, rows, ran = orc.nesterov_run([10.0], [-100.0], [100.0], 1.0, quad(2.0), 4,
                                    lambda0=1.0, alpha_max0_bins=1.0)
    assert ran == 4
    v2 = 7 - 2 * B1
    u3 = v2 - 4
    v3 = u3 + B2 * (u3 - 7)
    alphas = [1 / 20, 2 / 18, 4 / (2 * v2), 0.5]
    moves = [1.0, 2.0, 4.0, v3]
    for k in range(4):
        assert rows[k]["alpha"] == pytest.approx(alphas[k], rel=1e-12), k
        assert rows[k]["step_max"] == pytest.approx(moves[k], rel=1e-12), k
    assert abs(u[0]) < 1e-12
    # the momentum step of iteration 2 lands where the sign and index of
    # (u_{k+1} - u_k) say: v_3 = 3 - 2 beta_1 - beta_2 (4 + 2 beta_1)
    assert v3 == pytest.approx(3 - 2 * B1 - B2 * (4 + 2 * B1), rel=1e-15)
    assert 0.45 < v3 < 0.46


def test_step_bounds(orc):
    """alpha ||g||_inf is kept in [0.01 alpha_max, alpha_max], alpha_max_0 = 1.
    Cap: c = 2000 from x_0 = 10.  k=0: alpha = 1/20000, u_1 = 9.  k=1: the BB
    ratio 1/2000 would move 9, above alpha_max = 2, so alpha = 2 / 18000.
    Floor: c = 2 from x_0 = 1.001.  k=0: alpha = 1/2.002, u_1 = 0.001 (move 1,
    alpha_max 2).  k=1: the BB ratio 1/2 would move 0.001, below
    0.01 alpha_max = 0.02, so alpha = 0.02 / 0.002 = 10 and u_2 = -0.019."""
    _, rows, _ = orc.nesterov_run([10.0], [-100.0], [100.0], 1.0, quad(2000.0), 2,
                                  lambda0=1.0, alpha_max0_bins=1.0)
    assert rows[0]["alpha"] == pytest.approx(1 / 20000, rel=1e-12)
    assert rows[1]["alpha"] == pytest.approx(2 / 18000, rel=1e-12)
    u, rows, _ = orc.nesterov_run([1.001], [-100.0], [100.0], 1.0, quad(2.0), 2,
                                  lambda0=1.0, alpha_max0_bins=1.0)
    assert rows[0]["alpha"] == pytest.approx(1 / 2.002, rel=1e-12)
    assert rows[1]["alpha"] == pytest.approx(10.0, rel=1e-9)
    assert rows[1]["step_max"] == pytest.approx(0.02, rel=1e-9)
    assert u[0] == pytest.approx(-0.019, rel=1e-9)


def test_projection(orc):
    """The bounds clamp both the step and the momentum point: lower bound 7.5.
    k=0: u_1 = v_1 = 9.  k=1: alpha = 2/18 would reach 7, clamped to 7.5
    (move 1.5); v_2 = Pi(7.5 + beta_1 (7.5 - 9)) = 7.5; alpha_max = 3.
    k=2: g = 15, BB ratio |7.5 - 9| / |15 - 18| = 1/2, alpha g = 7.5 > 3:
    alpha = 3/15 and u_3 = Pi(4.5) = 7.5 (move 0)."""
    u, rows, ran = orc.nesterov_run([10.0], [7.5], [100.0], 1.0, quad(2.0), 3,
                                    lambda0=1.0, alpha_max0_bins=1.0)
    assert ran == 3
    assert [r["alpha"] for r in rows] == pytest.approx([1 / 20, 1 / 9, 0.2], rel=1e-12)
    assert [r["step_max"] for r in rows] == pytest.approx([1.0, 1.5, 0.0], abs=1e-12)
    assert u[0] == 7.5
    # a start outside the bounds is projected first: Pi(10) = 8.5
    u, rows, _ = orc.nesterov_run([10.0], [0.0], [8.5], 1.0, quad(2.0), 1,
                                  lambda0=1.0, alpha_max0_bins=1.0)
    assert rows[0]["alpha"] == pytest.approx(1 / 17, rel=1e-12)
    assert u[0] == pytest.approx(7.5, rel=1e-12)


def test_two_variables_use_norms(orc):
    """With two variables the step uses ||g||_inf and the BB ratio the 2-norms:
    c = 2, x_0 = (10, -5).  k=0: g = (20, -10), alpha = 1/20, u_1 = (9, -4.5),
    move 1.  k=1: g = (18, -9), dv = (1, 0.5), dg = (2, 1): BB = 1/2; alpha g_inf
    = 9 > 2: alpha = 2/18, moves (2, 1)."""
    u, rows, _ = orc.nesterov_run([10.0, -5.0], [-100.0] * 2, [100.0] * 2, 1.0, quad(2.0), 2,
                                  lambda0=1.0, alpha_max0_bins=1.0)
    assert [r["alpha"] for r in rows] == pytest.approx([1 / 20, 1 / 9], rel=1e-12)
    assert [r["step_max"] for r in rows] == pytest.approx([1.0, 2.0], rel=1e-12)
    np.testing.assert_allclose(u, [7.0, -3.5], rtol=1e-12)


def test_penalty_and_gamma_control(orc):
    """lambda and gamma.  gW = 2v, gN = v, HPWL(v) = 1e6 - H v with
    H = 1.75e5 and dw_ref = 3.5e5, tau(v) = 0.1 + 0.045 v, gamma scheduled,
    w_b = 1, alpha_max_0 = 1, x_0 = 10.
    k=0: lambda_0 = ||gW||_1 / ||gN||_1 = 2; g = 40, alpha = 1/40, u_1 = v_1 = 9.
         gamma_0 = gamma(tau(v_0) = 0.55) = 8 (exponent (20/9) 0.45 - 1 = 0).
    k=1: dW = HPWL(v_1) - HPWL(v_0) = H, mu = 1.1^(1 - 0.5) -> lambda_1 = 2 sqrt(1.1);
         gamma_1 = gamma(tau(v_0)) = 8 again; g = (2 + lambda_1) 9,
         alpha = 2 / g (BB ratio 1/|g_1 - 40| moves above alpha_max = 2);
         u_2 = 7, v_2 = 7 - 2 beta_1.
    k=2: dW = H (v_1 - v_2) = H (2 + 2 beta_1): taken at the look-ahead
         points v, not at u (u_2 - u_1 = -2 would give mu = 1 exactly);
         gamma_2 = gamma(tau(v_1) = 0.505) = 8 * 10^(0.9 - 1)."""
    H, ref = 1.75e5, 3.5e5
    obj = quad(2.0, lam_grad=1.0, hpwl=lambda v: 1e6 - H * float(v[0]),
               tau=lambda v: 0.1 + 0.045 * float(v[0]))
    _, rows, ran = orc.nesterov_run([10.0], [-100.0], [100.0], 1.0, obj, 3, lambda0=0.0,
                                    gamma_fixed=0.0, dw_ref=ref, alpha_max0_bins=1.0)
    assert ran == 3
    lam0 = 2.0
    lam1 = lam0 * 1.1 ** 0.5
    v2 = 7 - 2 * B1
    lam2 = lam1 * 1.1 ** (1 - H * (9 - v2) / ref)
    assert [r["lam"] for r in rows] == pytest.approx([lam0, lam1, lam2], rel=1e-12)
    assert [r["gamma"] for r in rows] == pytest.approx([8.0, 8.0, 8.0 * 10 ** -0.1], rel=1e-12)
    assert rows[1]["alpha"] == pytest.approx(2 / ((2 + lam1) * 9), rel=1e-12)
    assert rows[2]["step_max"] == pytest.approx(4.0, rel=1e-12)
    # the reading that would take dW at u instead: mu = 1.1^(1 - 2H/ref) = 1
    assert abs(lam2 - lam1) > 1e-3


def test_stop_on_overflow(orc):
    """The stop test uses the overflow of the evaluated point: tau(v) = v / 100
    from x_0 = 10 with tau_stop 0.085 stops after the iteration at v_2 = 7 - 2 beta_1
    (tau 0.064), having run iterations 0, 1, 2 (tau 0.1, 0.09, 0.064)."""
    obj = quad(2.0, tau=lambda v: float(v[0]) / 100.0)
    _, rows, ran = orc.nesterov_run([10.0], [-100.0], [100.0], 1.0, obj, 10, lambda0=1.0,
                                    alpha_max0_bins=1.0, stop_on_tau=True, tau_stop=0.085)
    assert ran == 3
    assert [r["tau"] for r in rows] == pytest.approx([0.1, 0.09, (7 - 2 * B1) / 100], rel=1e-12)


def test_adaptive_restart(orc):
    """Scripted gradients g = -1, -1, 0.001, -1, -1 from x_0 = 0 (alpha_max_0 = 1):
    k=0: alpha = 1, u_1 = v_1 = 1.  k=1: dg = 0 keeps alpha = 1, u_2 = 2,
    v_2 = 2 + beta_1.  k=2: the BB ratio moves 0.00128, below 0.01 alpha_max =
    0.02, so alpha = 20 and u_3 = v_2 - 0.02 = 1.98 + beta_1 > u_2: the step went
    up the gradient (g_2 (u_3 - u_2) > 0), so the sequence restarts after
    v_3 = u_3 + beta_2 (u_3 - u_2) is formed: a_3 = 1, and the momentum weight
    of iteration 3 is 0, so v_4 = u_4 exactly (without the restart it would be
    u_4 + (a_3 - 1)/a_4 (u_4 - u_3))."""
    grads = [-1.0, -1.0, 0.001, -1.0, -1.0]
    seen = []

    def objective(v, gamma):
        k = len(seen)
        seen.append(float(v[0]))
        g = np.array([grads[k]])
        return dict(gW=g, gN=np.zeros(1), W=0.0, hpwl=0.0, N=0.0, tau=0.5, gW_l1=1.0, gN_l1=1.0)

    u, rows, ran = orc.nesterov_run([0.0], [-100.0], [100.0], 1.0, objective, 5, lambda0=1.0,
                                    alpha_max0_bins=1.0)
    assert ran == 5
    u3 = 2 + B1 - 0.02
    v3 = u3 + B2 * (u3 - 2)
    assert seen[:4] == pytest.approx([0.0, 1.0, 2 + B1, v3], rel=1e-12, abs=1e-15)
    assert rows[2]["alpha"] == pytest.approx(20.0, rel=1e-9)
    # iteration 3: BB ratio |v_3 - v_2| / |g_3 - g_2|, inside [0.01, 1] alpha_max
    a3 = abs(v3 - (2 + B1)) / 1.001
    u4 = v3 + a3
    assert rows[3]["alpha"] == pytest.approx(a3, rel=1e-12)
    assert seen[4] == pytest.approx(u4, rel=1e-12)


def test_step_bound_ceiling(orc):
    """alpha_max doubles with the last largest move but not past the ceiling:
    c = 2 from x_0 = 10, alpha_max_0 = 1, ceiling 3 bins (w_b = 1).
    k=0: move 1 -> alpha_max 2.  k=1: alpha = 2/18, move 2 -> alpha_max
    min(4, 3) = 3.  k=2: alpha = 3 / g_2 with g_2 = 2 v_2, move 3 -> alpha_max
    min(6, 3) = 3 again (without the ceiling: 4, then 8)."""
    _, rows, _ = orc.nesterov_run([10.0], [-100.0], [100.0], 1.0, quad(2.0), 4, lambda0=1.0,
                                  alpha_max0_bins=1.0, alpha_max_cap_bins=3.0)
    v2 = 7 - 2 * B1
    assert [r["step_max"] for r in rows[:3]] == pytest.approx([1.0, 2.0, 3.0], rel=1e-12)
    assert rows[2]["alpha"] == pytest.approx(3.0 / (2 * v2), rel=1e-12)
    u3 = v2 - 3.0
    v3 = u3 + B2 * (u3 - 7.0)
    # k=3: the BB ratio 1/2 moves |v_3| (about 1.9), inside [0.03, 3]
    assert rows[3]["alpha"] == pytest.approx(0.5, rel=1e-12)
    assert rows[3]["step_max"] == pytest.approx(abs(v3), rel=1e-12)
