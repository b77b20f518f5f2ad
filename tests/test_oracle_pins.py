"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names the fact it checks and where it comes from.  A plausible slip
in the oracle (a sign in K_i, a transposed exponential, a dropped 1/4 in the
conjugate, a wrong node time or weight, a missing term in the gap) fails at
least one of them.
"""
import numpy as np
import pytest
from scipy.linalg import expm

from inputs import workloads as wl
from oracle import hopf as oh
from tests import _independent as ind


# ----------------------------------------------------------------- quadrature
def test_nodes_left_riemann_and_trapezoid_integrate_polynomials():
    # Left Riemann (Eq. 17) integrates constants exactly; trapezoid also
    # integrates linear functions exactly.
    t, w = oh.nodes(3.0, 12, oh.LEFT_RIEMANN)
    assert np.isclose(w.sum(), 3.0) and np.isclose(t[0], 0.0) and np.isclose(t[-1], 3.0 - 0.25)
    t, w = oh.nodes(3.0, 13, oh.TRAPEZOID)
    assert np.isclose(w.sum(), 3.0) and np.isclose((w * t).sum(), 4.5)
    assert np.isclose(t[-1], 3.0) and np.isclose(w[0], 0.125)


def test_simpson_weights_integrate_cubics_and_reject_even_counts():
    # composite Simpson's rule (named in §III.A) is exact for cubics
    t, w = oh.nodes(2.0, 9, oh.SIMPSON)
    for k in range(4):
        assert np.isclose((w * t ** k).sum(), 2.0 ** (k + 1) / (k + 1), rtol=1e-13)
    assert not np.isclose((w * t ** 4).sum(), 2.0 ** 5 / 5, rtol=1e-6)
    with pytest.raises(ValueError):
        oh.nodes(2.0, 8, oh.SIMPSON)


def test_simpson_value_converges_at_fourth_order():
    # For a smooth Hamiltonian along the optimal p (ball control, K_i p != 0)
    # the quadrature error of phi_N is that of the integral at p*: halving the
    # step divides it by 16 with Simpson's rule and by 4 with the trapezoid
    # rule.  A wrong Simpson weight pattern drops the order.
    sysd = wl.random_system(5, 3, 2)
    x = np.array([[4.2, -3.7, 3.9]])
    ref = oh.value(sysd, x, 1.5, 1025, oh.SIMPSON, 0.5, tol=1e-13)["phi"][0]
    for rule, order in ((oh.SIMPSON, 16.0), (oh.TRAPEZOID, 4.0)):
        e = [abs(oh.value(sysd, x, 1.5, N, rule, 0.5, tol=1e-13)["phi"][0] - ref) for N in (9, 17, 33)]
        assert all(abs(e[i] / e[i + 1] - order) < 0.1 * order for i in range(2)), (rule, e)


# ----------------------------------------------------- double integrator table
def test_di_node_matrices_closed_form():
    # §VI.A: A = [[0,1],[0,0]] is nilpotent, e^{-sA} B = [-s, 1]^T, so
    # K_i = -(e^{-s_i A} B)^T = [s_i, -1] with s_i = T - t_i.
    sysd = wl.double_integrator(0.2)
    for rule in (oh.LEFT_RIEMANN, oh.TRAPEZOID):
        K = oh.node_matrices(sysd, 1.7, 9, rule)
        t, _ = oh.nodes(1.7, 9, rule)
        s = 1.7 - t
        assert np.allclose(K[:, 0, 0], s, atol=1e-14)
        assert np.allclose(K[:, 0, 1], -1.0, atol=1e-14)


def test_di_terminal_variable_node_matrices_closed_form():
    # After p = e^{T A^T} q the node matrices are (-e^{t_i A} B)^T; for the
    # double integrator e^{tA} B = [t, 1]^T, so K'_i = [-t_i, -1], and M' = W.
    sysd = wl.double_integrator(0.2)
    for rule in (oh.LEFT_RIEMANN, oh.TRAPEZOID):
        prob = oh.setup(sysd, 1.7, 9, rule, 1.0, variables="terminal")
        t, _ = oh.nodes(1.7, 9, rule)
        assert np.allclose(prob["K"][:, 0, 0], -t, atol=1e-14)
        assert np.allclose(prob["K"][:, 0, 1], -1.0, atol=1e-14)
        assert np.allclose(prob["M"], 0.04 * np.eye(2)) and np.allclose(prob["E"], [[1.0, 1.7], [0.0, 1.0]])


def test_terminal_matrices_closed_form_di():
    # M = e^{-TA} W e^{-TA}^T with e^{-TA} = [[1, -T], [0, 1]].
    sysd = wl.double_integrator(0.3)
    M, V = oh.terminal_matrices(sysd, 2.0)
    E = np.array([[1.0, -2.0], [0.0, 1.0]])
    assert np.allclose(M, 0.09 * E @ E.T, atol=1e-14)
    assert np.allclose(V @ M, np.eye(2), atol=1e-12)


def test_expm_library_against_closed_forms():
    # The oracle relies on scipy's expm; pin it on a rotation generator
    # (e^{sJ} = [[cos, sin], [-sin, cos]]) and a diagonal matrix.
    J = np.array([[0.0, 1.0], [-1.0, 0.0]])
    s = 0.7
    assert np.allclose(expm(s * J), [[np.cos(s), np.sin(s)], [-np.sin(s), np.cos(s)]], atol=1e-15)
    d = np.array([0.3, -1.2, 2.0])
    assert np.allclose(expm(np.diag(d)), np.diag(np.exp(d)), rtol=1e-14)


# ------------------------------------------------------- single integrator
@pytest.mark.parametrize("kind", [oh.BALL, oh.BOX])
def test_single_integrator_value_closed_form(kind):
    # A = 0, B = I: every K_i = -Q^T, the quadrature is exact for any N, and the
    # basic Hopf formula (Eq. 6) gives phi = min over the reachable set of J:
    #   ball: max(|x| - rho T, 0)^2 / r^2 - 1;  box: |softthresh(x, T b)|^2 / r^2 - 1.
    n, rho, r = 3, 0.8, 0.5
    sysd = wl.single_integrator(n, kind, radius=rho, radius_target=r)
    x = wl.normal_points(7, 6, n, 1.5)
    T = 0.9
    res = oh.value(sysd, x, T, 16, oh.LEFT_RIEMANN, tau=1.0, tol=1e-11)
    assert np.all(res["status"] == oh.OK)
    if kind == oh.BALL:
        nx = np.linalg.norm(x, axis=1)
        exact = np.maximum(nx - rho * T, 0.0) ** 2 / r ** 2 - 1.0
        grad = 2.0 * np.maximum(nx - rho * T, 0.0)[:, None] / r ** 2 * x / nx[:, None]
    else:
        st = np.sign(x) * np.maximum(np.abs(x) - rho * T, 0.0)
        exact = np.sum(st ** 2, axis=1) / r ** 2 - 1.0
        grad = 2.0 * st / r ** 2
    assert np.allclose(res["phi"], exact, rtol=1e-9, atol=1e-9)
    # Eq. 24: the minimiser is the gradient of the value
    assert np.allclose(res["p"], grad, rtol=1e-5, atol=1e-5)


def test_single_integrator_time_to_reach_closed_form():
    # Ball control of radius rho, ball target of radius r: T* = max(|x| - r, 0) / rho.
    n, rho, r = 2, 1.0, 0.5
    sysd = wl.single_integrator(n, oh.BALL, radius=rho, radius_target=r)
    x = np.array([[1.5, 0.2], [0.1, 0.2], [-2.0, 2.5]])
    res = oh.time_to_reach(sysd, x, 6.0, 8, oh.LEFT_RIEMANN, tau=1.0, tol_T=1e-7)
    exact = np.maximum(np.linalg.norm(x, axis=1) - r, 0.0) / rho
    assert np.allclose(res["T"], exact, rtol=2e-6, atol=1e-9)
    assert res["T"][1] == 0.0


# ---------------------------------------------- strong duality, other solvers
@pytest.mark.parametrize("variables", ["initial", "terminal"])
def test_value_equals_independent_projected_gradient_box_di(variables):
    # phi_N from the PDHG (dual form) equals the discrete-control minimum
    # computed by an unrelated algorithm (FISTA on the primal control form),
    # in the paper's variable p and in the terminal-time variable q.
    sysd = wl.double_integrator(0.1)
    for T, x0 in [(1.0, np.array([0.6, -0.3])), (2.0, np.array([-1.2, 0.9]))]:
        res = oh.value(sysd, x0, T, 32, oh.TRAPEZOID, tau=2.0, tol=1e-12, variables=variables)
        ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x0, T, 32, "box", trapezoid=True)
        assert abs(res["phi"][0] - ref) <= 1e-8 * max(1.0, abs(ref))


@pytest.mark.parametrize("variables", ["initial", "terminal"])
def test_value_equals_independent_projected_gradient_ball_random(variables):
    sysd = wl.random_system(11, 4, 2)
    x = wl.normal_points(12, 3, 4, 1.0)
    res = oh.value(sysd, x, 0.8, 24, oh.LEFT_RIEMANN, tau=0.2, tol=1e-12, variables=variables)
    for k in range(3):
        ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x[k], 0.8, 24, "ball")
        assert abs(res["phi"][k] - ref) <= 1e-8 * max(1.0, abs(ref)), (k, res["phi"][k], ref)


@pytest.mark.parametrize("variables", ["initial", "terminal"])
def test_value_equals_brute_force_enumeration(variables):
    # Exhaustive active-set enumeration is exact on N <= 8 scalar-control nodes.
    sysd = wl.double_integrator(0.2)
    for T, x0, rule in [(1.3, np.array([0.5, 0.4]), oh.LEFT_RIEMANN),
                        (0.7, np.array([-0.3, 0.8]), oh.TRAPEZOID)]:
        res = oh.value(sysd, x0, T, 6, rule, tau=2.0, tol=1e-13, variables=variables)
        ref = ind.brute_force_value(sysd["A"], sysd["B"], sysd["W"], x0, T, 6,
                                    trapezoid=(rule == oh.TRAPEZOID))
        assert abs(res["phi"][0] - ref) <= 1e-9 * max(1.0, abs(ref)), (res["phi"][0], ref)


@pytest.mark.parametrize("variables", ["initial", "terminal"])
def test_duality_gap_certifies_interval(variables):
    # Weak duality: D(y) <= phi <= ... i.e. -P <= phi <= -D for any feasible pair,
    # and the independent optimum lies inside [-P, -D] at every tolerance.
    sysd = wl.double_integrator(0.1)
    x0 = np.array([0.9, 0.2])
    ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x0, 1.0, 16, "box", trapezoid=True)
    for tol in (1e-2, 1e-4, 1e-6):
        r = oh.value(sysd, x0, 1.0, 16, oh.TRAPEZOID, tau=2.0, tol=tol, variables=variables)
        assert -r["P"][0] - 1e-12 <= ref <= -r["D"][0] + 1e-12
        assert r["gap"][0] <= tol


# ----------------------------------------------------------- calculus pins
@pytest.mark.parametrize("variables", ["initial", "terminal"])
def test_gradient_identity_finite_differences(variables):
    # Eq. 24: p* = grad_z phi (= grad_x phi at t = 0).  In terminal-time
    # variables this also pins the map back p = e^{T A^T} q.
    sysd = wl.random_system(5, 3, 1)
    x0 = np.array([0.8, -0.5, 0.3])
    T, N = 0.6, 20
    base = oh.value(sysd, x0, T, N, oh.LEFT_RIEMANN, tau=0.3, tol=1e-13, variables=variables)
    h = 1e-4
    fd = np.zeros(3)
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fp = oh.value(sysd, x0 + e, T, N, oh.LEFT_RIEMANN, tau=0.3, tol=1e-13)["phi"][0]
        fm = oh.value(sysd, x0 - e, T, N, oh.LEFT_RIEMANN, tau=0.3, tol=1e-13)["phi"][0]
        fd[j] = (fp - fm) / (2 * h)
    assert np.allclose(base["p"][0], fd, rtol=1e-5, atol=1e-6), (base["p"][0], fd)


def test_hj_identity_time_derivative():
    # §IV: d phi / dT = -H_x(p*, x0), H_x(p, x0) = -x0^T A^T p + |-Q^T B^T p|_*.
    # The discretised phi_N matches it up to the quadrature error.
    sysd = wl.double_integrator(0.2)
    x0 = np.array([0.9, 0.3])
    T, N, h = 1.0, 400, 1e-3
    r0 = oh.value(sysd, x0, T, N, oh.TRAPEZOID, tau=2.0, tol=1e-12)
    fp = oh.value(sysd, x0, T + h, N, oh.TRAPEZOID, tau=2.0, tol=1e-12)["phi"][0]
    fm = oh.value(sysd, x0, T - h, N, oh.TRAPEZOID, tau=2.0, tol=1e-12)["phi"][0]
    dphi = (fp - fm) / (2 * h)
    H = oh.hamiltonian_x(sysd, r0["p"][0], x0)
    assert abs(dphi + H) <= 1e-2 * max(1.0, abs(H)), (dphi, H)


def test_value_monotone_in_time_di():
    # A larger horizon can only enlarge the set of reachable end states here.
    sysd = wl.double_integrator(0.1)
    x0 = np.array([1.0, 0.0])
    vals = [oh.value(sysd, x0, T, 64, oh.TRAPEZOID, tau=2.0, tol=1e-10)["phi"][0]
            for T in (0.5, 1.0, 1.5, 2.0, 2.5)]
    assert all(a >= b - 1e-9 for a, b in zip(vals, vals[1:])), vals


# ------------------------------------------------------------- trajectory
def test_trajectory_endpoint_is_conjugate_gradient():
    # Eq. 29 with Eq. 35: the optimal end state in z is (1/2) V^-1 p* = M p* / 2,
    # i.e. x(T) = e^{TA} M p*/2.  The node controls carried by the dual reach
    # it exactly; the argmax controls of Eq. 27 reach it up to the nodes where
    # K_i p* = 0 (a switch falls on a node and the maximiser is not unique),
    # each of which moves the end point by at most 2 w_i |e^{-s_i A} B Q|.
    sysd = wl.random_system(21, 3, 1)
    x0 = np.array([1.2, -0.4, 0.7])
    T, N = 0.9, 30
    prob = oh.setup(sysd, T, N, oh.LEFT_RIEMANN, 0.3)
    r = oh.pdhg(prob, x0[None], tol=1e-12)
    M, _ = oh.terminal_matrices(sysd, T)
    end = expm(T * sysd["A"]) @ (0.5 * M @ r["p"][0])
    s_d, x_d = oh.trajectory_from_dual(sysd, x0, prob, r["y"][0])
    assert np.isclose(s_d[-1], T) and np.allclose(x_d[-1], end, atol=1e-8), (x_d[-1], end)
    assert abs(oh.terminal_cost(sysd, x_d[-1][None])[0] - r["phi"][0]) < 1e-8
    xs, us = oh.trajectory(sysd, x0, T, r["p"][0], N)
    Kp = np.einsum("imn,n->im", prob["K"], r["p"][0])
    on_switch = np.sum(np.linalg.norm(Kp, axis=1) < 1e-6)
    bound = on_switch * 2.0 * (T / N) * np.exp(T * np.linalg.norm(sysd["A"], 2)) * \
        np.linalg.norm(sysd["B"], 2) * np.linalg.norm(expm(T * sysd["A"]), 2)
    assert np.linalg.norm(xs[-1] - end) <= bound + 1e-8
    assert np.all(np.abs(us) <= 1.0 + 1e-12)
    # the two constructions agree at every node that is not on a switch
    if on_switch == 0:
        assert np.allclose(xs, x_d, atol=1e-8)


def test_trajectory_di_reaches_target_boundary_at_time_to_reach():
    # §IV: at T* the end state lies on the target boundary (J_x = 0).  The dual
    # node controls reach it exactly; the argmax controls of Eq. 27 differ only
    # at a node that carries the switch, by at most 2 w_i |e^{-s_i A} B| there.
    sysd = wl.double_integrator(0.2)
    x0 = np.array([1.0, 0.0])
    N = 100
    tt = oh.time_to_reach(sysd, x0, 6.0, N, oh.LEFT_RIEMANN, tau=2.0, tol_T=1e-9, tol_gap=1e-11)
    T = tt["T"][0]
    prob = oh.setup(sysd, T, N, oh.LEFT_RIEMANN, 2.0)
    r = oh.pdhg(prob, x0[None], tol=1e-12)
    _, x_d = oh.trajectory_from_dual(sysd, x0, prob, r["y"][0])
    assert abs(oh.terminal_cost(sysd, x_d[-1][None])[0]) < 1e-6
    xs, _ = oh.trajectory(sysd, x0, T, tt["p"][0], N)
    assert np.linalg.norm(xs[-1] - x_d[-1]) <= 2.0 * (T / N) * (1.0 + T) * (1.0 + T) + 1e-9


def test_di_time_to_reach_against_switching_curve():
    # Time to reach a ball of radius r is below the bang-bang time to the origin
    # T0(x), and T0(x) - T*(r) is at most the worst time to the origin from
    # inside the ball (<= r + 2 sqrt(r + r^2/2)); it shrinks as r -> 0 (§II.B remark).
    x0 = np.array([1.0, 0.5])
    T0 = ind.di_min_time_to_origin(x0)
    prev = -np.inf
    for r in (0.2, 0.1, 0.05):
        sysd = wl.double_integrator(r)
        T = oh.time_to_reach(sysd, x0, 8.0, 200, oh.TRAPEZOID, tau=2.0, tol_T=1e-6)["T"][0]
        slack = r + 2.0 * np.sqrt(r + 0.5 * r * r)
        assert T <= T0 + 1e-3 and T0 - T <= slack + 1e-2, (r, T, T0)
        assert T > prev
        prev = T


def test_di_control_sign_matches_switching_curve():
    # Away from the switching curve the first control is -sign(x1 + x2|x2|/2).
    sysd = wl.double_integrator(0.05)
    for x0 in (np.array([1.0, 0.5]), np.array([-1.2, 0.3]), np.array([0.4, -1.5])):
        tt = oh.time_to_reach(sysd, x0, 8.0, 200, oh.TRAPEZOID, tau=2.0, tol_T=1e-6)
        u0 = oh.optimal_control(sysd, tt["p"][0], 1e-3)
        sw = x0[0] + 0.5 * x0[1] * abs(x0[1])
        assert np.sign(u0[0]) == -np.sign(sw)


def test_accelerated_iteration_reaches_the_same_value():
    # Chambolle-Pock Algorithm 2 (strongly convex G, §III) converges to the same
    # discretised value; pinned against the independent projected-gradient solver.
    sysd = wl.random_system(11, 4, 2)
    x = wl.normal_points(12, 3, 4, 1.0)
    res = oh.value(sysd, x, 0.8, 24, oh.LEFT_RIEMANN, tau=2.0, tol=1e-12, accel=True)
    assert np.all(res["status"] == oh.OK)
    for k in range(3):
        ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x[k], 0.8, 24, "ball")
        assert abs(res["phi"][k] - ref) <= 1e-8 * max(1.0, abs(ref))
    sysd = wl.double_integrator(0.1)
    x0 = np.array([0.6, -0.3])
    r1 = oh.value(sysd, x0, 1.0, 32, oh.TRAPEZOID, tau=2.0, tol=1e-12, accel=True)
    ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x0, 1.0, 32, "box", trapezoid=True)
    assert abs(r1["phi"][0] - ref) <= 1e-8 * max(1.0, abs(ref))


def test_terminal_variables_time_to_reach_matches_switching_curve_bound():
    # The bisection in terminal-time variables finds the same T* as in the
    # paper's variables, inside the switching-curve bound of the double integrator.
    sysd = wl.double_integrator(0.1)
    x = np.array([[1.0, 0.5], [-1.2, 0.3]])
    rt = oh.time_to_reach(sysd, x, 8.0, 64, oh.TRAPEZOID, tau=2.0, tol_T=1e-8, variables="terminal")
    ri = oh.time_to_reach(sysd, x, 8.0, 64, oh.TRAPEZOID, tau=2.0, tol_T=1e-8)
    assert np.allclose(rt["T"], ri["T"], rtol=1e-7), (rt["T"], ri["T"])
    for k in range(2):
        T0 = ind.di_min_time_to_origin(x[k])
        assert 0.0 <= T0 - rt["T"][k] <= 0.1 + 2.0 * np.sqrt(0.1 + 0.005) + 1e-2
    # p* at gap 1e-8 is fixed only to about sqrt(gap / lambda_min(M)) here
    assert np.allclose(rt["p"], ri["p"], rtol=1e-3, atol=1e-6)


def test_newton_time_to_reach_matches_closed_form_and_bisection():
    # §IV hybrid Newton/bisection: single integrator closed form T* = |x| - r,
    # and the double integrator against the bisection result.
    sysd = wl.single_integrator(2, oh.BALL, radius=1.0, radius_target=0.5)
    x = np.array([[1.5, 0.2], [0.1, 0.2], [-2.0, 2.5]])
    r = oh.time_to_reach_newton(sysd, x, 6.0, 8, oh.LEFT_RIEMANN, tau=1.0, tol_T=1e-9)
    assert np.allclose(r["T"], np.maximum(np.linalg.norm(x, axis=1) - 0.5, 0.0), rtol=1e-7, atol=1e-9)
    sysd = wl.double_integrator(0.1)
    x = np.array([[1.0, 0.5], [-1.2, 0.3], [0.4, -1.5]])
    rn = oh.time_to_reach_newton(sysd, x, 10.0, 64, oh.TRAPEZOID, tau=2.0, tol_T=1e-8)
    rb = oh.time_to_reach(sysd, x, 10.0, 64, oh.TRAPEZOID, tau=2.0, tol_T=1e-8)
    assert np.allclose(rn["T"], rb["T"], rtol=1e-6), (rn["T"], rb["T"])
    assert rn["steps"] < rb["steps"]


# ------------------------------------------- stacked copies (§VI.B, §VI.C)
def test_unscented_samples_reproduce_mean_and_covariance():
    mu = np.array([0.7, -1.2])
    chi, w = wl.unscented_samples(mu, 0.3)
    assert chi.shape == (5, 2) and np.isclose(w.sum(), 1.0)
    assert np.allclose(w @ chi, mu)
    d = chi - mu
    assert np.allclose((w[:, None] * d).T @ d, 0.09 * np.eye(2))


def test_identical_stacked_copies_reduce_to_the_base_problem():
    # All copies at the same state under one shared control: the weighted mean
    # square distance is the base distance, so phi of the stacked problem
    # equals phi of the base problem with target radius sqrt(ell), for any
    # copy weights summing to 1.
    w = wl.workload_unscented(3, std=0.0)
    base = wl.double_integrator(np.sqrt(w["ell"]))
    for T in (1.0, 2.5):
        a = oh.value(w["system"], w["x"], T, 40, oh.LEFT_RIEMANN, 0.5, tol=1e-11)["phi"]
        b = oh.value(base, w["mu"], T, 40, oh.LEFT_RIEMANN, 0.5, tol=1e-11)["phi"]
        assert np.allclose(a, b, rtol=1e-8), (a, b)


@pytest.mark.parametrize("variables", ["initial", "terminal"])
def test_adaptive_steps_reach_the_independent_value(variables):
    # Residual-balanced steps (§III.B residuals, Goldstein et al.'s adaptive
    # PDHG) change tau and sigma as they go but converge to the same
    # discretised value; pinned against the projected-gradient solver, ball
    # and box control
    sysd = wl.random_system(11, 4, 2)
    x = wl.normal_points(12, 3, 4, 1.0)
    res = oh.value(sysd, x, 0.8, 24, oh.LEFT_RIEMANN, tau=0.2, tol=1e-12, adaptive=True, variables=variables)
    assert np.all(res["status"] == oh.OK)
    for k in range(3):
        ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x[k], 0.8, 24, "ball")
        assert abs(res["phi"][k] - ref) <= 1e-8 * max(1.0, abs(ref))
    sysd = wl.double_integrator(0.1)
    x0 = np.array([0.6, -0.3])
    r1 = oh.value(sysd, x0, 1.0, 32, oh.TRAPEZOID, tau=2.0, tol=1e-12, adaptive=True, variables=variables)
    ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x0, 1.0, 32, "box", trapezoid=True)
    assert abs(r1["phi"][0] - ref) <= 1e-8 * max(1.0, abs(ref))


# ------------------------------------------------ fixed-step quadrature rule
def test_fixed_step_nodes_are_the_partition_and_reduce_to_eq17():
    # The nodes of horizon T are the left ends of the partition {0, dt, ...,
    # t_last, T} (walked independently here); at T = k dt they are Eq. 17 with
    # k nodes; the weights always sum to T.
    rule = oh.FixedStep(4.0, 64)
    for T in (0.01, 0.0625, 0.3, 1.0, 1.23456, 3.99, 4.0):
        t, w = oh.nodes(T, 64, rule)
        tr, wr = ind.fixed_step_nodes(T, 4.0 / 64)
        assert t.size == tr.size and np.allclose(t, tr, rtol=0, atol=1e-15) and np.allclose(w, wr, rtol=1e-12)
        assert abs(w.sum() - T) <= 1e-14 * T and np.all(w > 0) and np.all(t < T)
    for k in (1, 5, 17, 64):
        t, w = oh.nodes(k * rule.dt, 64, rule)
        tl, wl = oh.nodes(k * rule.dt, k, oh.LEFT_RIEMANN)
        assert np.allclose(t, tl, rtol=1e-15, atol=0) and np.allclose(w, wl, rtol=1e-15)
    with pytest.raises(ValueError):
        oh.nodes(4.5, 64, rule)


def test_fixed_step_single_integrator_time_to_reach_closed_form():
    # A = 0: the value depends on the weights only through their sum, so the
    # fixed-step rule is exact at every T, not only at multiples of the step:
    # T* = max(|x| - r, 0) / rho.  A wrong last weight moves T* off it.
    n, rho, r = 2, 1.0, 0.5
    sysd = wl.single_integrator(n, oh.BALL, radius=rho, radius_target=r)
    x = np.array([[1.5, 0.2], [0.1, 0.2], [-2.0, 2.5], [0.7, -0.45]])
    for variables in ("initial", "terminal"):
        res = oh.time_to_reach(sysd, x, 6.0, 8, oh.FixedStep(6.0, 8), tau=1.0, tol_T=1e-8,
                               variables=variables)
        exact = np.maximum(np.linalg.norm(x, axis=1) - r, 0.0) / rho
        assert np.allclose(res["T"], exact, rtol=2e-7, atol=1e-9), (variables, res["T"], exact)


@pytest.mark.parametrize("variables", ["initial", "terminal"])
def test_fixed_step_value_equals_independent_projected_gradient(variables):
    # phi with the fixed-step nodes against FISTA on the primal control form
    # with the partition nodes built independently, at horizons between
    # multiples of the step (a partial last node).
    sysd = wl.random_system(11, 4, 2)
    x = wl.normal_points(12, 2, 4, 1.0)
    rule = oh.FixedStep(2.0, 40)
    for T in (0.77, 1.313):
        res = oh.value(sysd, x, T, 40, rule, tau=0.2, tol=1e-12, variables=variables)
        for k in range(2):
            ref, _ = ind.fista_value(sysd["A"], sysd["B"], sysd["W"], x[k], T, 0, "ball",
                                     tw=ind.fixed_step_nodes(T, rule.dt))
            assert abs(res["phi"][k] - ref) <= 1e-8 * max(1.0, abs(ref)), (T, k, res["phi"][k], ref)


def test_fixed_step_di_time_to_reach_within_switching_curve_bound():
    # The double integrator's time to reach a ball of radius r lies below the
    # bang-bang time to the origin by at most the worst time from inside the
    # ball; the fixed-step bisection lands there and agrees with the
    # uniform-step rule to the quadrature error.
    sysd = wl.double_integrator(0.1)
    x = np.array([[1.0, 0.5], [-1.2, 0.3]])
    rf = oh.time_to_reach(sysd, x, 8.0, 512, oh.FixedStep(8.0, 512), tau=2.0, tol_T=1e-8,
                          variables="terminal")
    ru = oh.time_to_reach(sysd, x, 8.0, 256, oh.LEFT_RIEMANN, tau=2.0, tol_T=1e-8, variables="terminal")
    for k in range(2):
        T0 = ind.di_min_time_to_origin(x[k])
        assert 0.0 <= T0 - rf["T"][k] <= 0.1 + 2.0 * np.sqrt(0.1 + 0.005) + 1e-2
    assert np.allclose(rf["T"], ru["T"], rtol=2e-3), (rf["T"], ru["T"])
