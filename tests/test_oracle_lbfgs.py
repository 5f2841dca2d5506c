"""Pins for the oracle's Phase 1 (batched L-BFGS, Sec. 3.2.1)."""
import numpy as np
import pytest

from oracle import method as M
from paper_2606_26164_gb300 import inputs as I


def _dense_bfgs_inverse(pairs, d):
    """Explicit inverse-BFGS recursion H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T
    from H0 = gamma I (gamma of the newest pair), oldest pair first."""
    s_new, y_new = pairs[0]
    H = (s_new @ y_new) / (y_new @ y_new) * np.eye(d)
    for s, y in reversed(pairs):
        rho = 1.0 / (s @ y)
        V = np.eye(d) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


@pytest.mark.parametrize("d,k", [(2, 1), (3, 2), (4, 4), (4, 3)])
def test_two_loop_equals_dense_bfgs(d, k):
    rng = np.random.default_rng(10 * d + k)
    m = 5
    N = 6
    S = np.zeros((N, m, d))
    Y = np.zeros((N, m, d))
    rho = np.zeros((N, m))
    hlen = np.full(N, k)
    G = rng.standard_normal((N, d))
    for n in range(N):
        B = rng.standard_normal((d, d))
        A = B @ B.T + d * np.eye(d)                       # SPD curvature so s^T y > 0
        for i in range(k):
            s = rng.standard_normal(d)
            y = A @ s
            S[n, i], Y[n, i], rho[n, i] = s, y, 1.0 / (s @ y)
    P = M.lbfgs_direction(G, S, Y, rho, hlen)
    for n in range(N):
        H = _dense_bfgs_inverse([(S[n, i], Y[n, i]) for i in range(k)], d)
        np.testing.assert_allclose(P[n], -H @ G[n], rtol=1e-10, atol=1e-12)


def test_two_loop_empty_history_is_steepest_descent():
    G = np.array([[1.0, -2.0, 3.0]])
    Z = np.zeros((1, 4, 3))
    np.testing.assert_array_equal(M.lbfgs_direction(G, Z, Z, np.zeros((1, 4)), np.zeros(1, int)), -G)


def test_line_search_backtracks_to_first_passing_step():
    """F = x^2/2 (f = -x^2/2) at x=1 with an overshooting direction p=-3:
    alpha=1 lands at x=-2 (F=2 > 0.5 - 3e-4), alpha=1/2 at x=-1/2 (F=1/8 passes)."""
    obj = I.Objective(3, 1, {"center": np.array([0.0]), "Q": np.eye(1), "lam": np.array([0.5])})
    prob = I.Problem(1, 1, np.array([-10.0]), np.array([10.0]), obj, np.zeros((1, 1), np.float32), 1e-6, 1.0)
    P = M.Params()
    X = np.array([[1.0]])
    F = np.array([0.5])
    G = np.array([[1.0]])
    acc, Xn, Fn, trials = M.line_search(prob, X, F, G, np.array([[-3.0]]), np.array([1.0]), P)
    assert acc[0] and trials[0] == 2
    assert Xn[0, 0] == -0.5 and Fn[0] == 0.125


def test_line_search_projects_onto_box():
    obj = I.Objective(3, 1, {"center": np.array([5.0]), "Q": np.eye(1), "lam": np.array([1.0])})
    prob = I.Problem(1, 1, np.array([-1.0]), np.array([1.0]), obj, np.zeros((1, 1), np.float32), 1e-6, 1.0)
    P = M.Params()
    X = np.array([[0.0]])
    F = np.array([25.0])                                  # F = -f = (x-5)^2
    G = np.array([[-10.0]])
    acc, Xn, Fn, _ = M.line_search(prob, X, F, G, np.array([[10.0]]), np.array([1.0]), P)
    assert acc[0] and Xn[0, 0] == 1.0 and Fn[0] == 16.0


def test_curvature_pair_rejected_when_not_positive():
    st = M.new_state(np.zeros((2, 2)), 3)
    s = np.array([[1.0, 0.0], [1.0, 0.0]])
    y = np.array([[1.0, 0.0], [-1.0, 0.0]])
    ok = M.push_pair(st, np.arange(2), s, y, M.Params())
    assert list(ok) == [True, False]
    assert list(st.hlen) == [1, 0] and st.rho[0, 0] == 1.0


def test_phase1_converges_to_quadratic_center():
    """Proposition 1: on a strictly log-concave target every sample converges to theta*."""
    p = I.small_quadratic(4, 16, seed=5, cond=10.0)
    P = M.Params(m=5, grad_mode=M.GRAD_ADJOINT)
    st = M.new_state(p.x0, P.m)
    M.lbfgs_iterations(p, st, P, 40)
    c = p.objective.arrays["center"]
    assert np.abs(st.x - c[None]).max() < 1e-8
    assert np.abs(st.g).max() < 1e-6


def test_phase1_fd_and_adjoint_agree_on_mixture():
    p = I.small_mixture(3, 4, 24, seed=6)
    out = []
    for mode in (M.GRAD_ADJOINT, M.GRAD_FD64):
        P = M.Params(m=5, grad_mode=mode)
        st = M.new_state(p.x0, P.m)
        M.lbfgs_iterations(p, st, P, 30)
        out.append(st.x.copy())
    np.testing.assert_allclose(out[0], out[1], atol=1e-5)
