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


def test_line_search_equals_trials_taken_in_batches():
    """Reading 23: the trials of a search do not depend on one another, so evaluating them
    in batches side by side and taking the first that passes (as the batched evaluator and
    the small-sample device kernels do) gives the sequential search's step, value and trial
    count.  Checked on a noisy mixture with one-trial-at-a-time, batches of 3 and batches of
    8, including searches that fail and samples already at a mode."""
    prob = I.small_mixture(3, 4, 200, seed=9, noise_sigma=0.05)
    P = M.Params(m=5, grad_mode=M.GRAD_ADJOINT, T_ls=11)
    rng = np.random.default_rng(9)
    X = prob.x0.astype(np.float64)
    F = -M.evaluate(prob, X)
    G = -M.gradient(prob, X, P)
    Pd = -G + rng.normal(0, 1.0, G.shape) * np.abs(G).max(axis=1, keepdims=True)   # some ascent steps
    alpha0 = np.minimum(1.0, 1.0 / np.abs(G).max(axis=1))
    acc, Xn, Fn, trials = M.line_search(prob, X, F, G, Pd, alpha0, P)
    assert 0 < acc.sum() < prob.n
    for B in (1, 3, 8):
        for i in range(prob.n):
            got = None
            for t0 in range(0, P.T_ls, B):
                ts = np.arange(t0, min(t0 + B, P.T_ls))
                Xt = np.clip(X[i] + (alpha0[i] * 2.0 ** (-ts))[:, None] * Pd[i], prob.lo, prob.hi)
                Ft = -M.evaluate(prob, Xt)
                ok = Ft <= F[i] + P.c1 * (Xt - X[i]) @ G[i]
                if ok.any():
                    k = int(np.argmax(ok))
                    got = (True, Xt[k], Ft[k], int(ts[k]) + 1)
                    break
            if got is None:
                got = (False, X[i], F[i], P.T_ls)
            assert got[0] == acc[i] and got[3] == trials[i]
            np.testing.assert_array_equal(got[1], Xn[i])
            assert got[2] == Fn[i]


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


def test_curvature_pair_rejected_when_rho_would_overflow():
    """s^T y = 1e-310 (subnormal) passes the angle test but 1 / s^T y is not a
    finite double: the pair is not stored, so no infinite rho enters the history."""
    st = M.new_state(np.zeros((2, 2)), 3)
    s = np.array([[1e-155, 0.0], [1e-150, 0.0]])
    y = np.array([[1e-155, 0.0], [1e-150, 0.0]])
    ok = M.push_pair(st, np.arange(2), s, y, M.Params())
    assert list(ok) == [False, True]
    assert list(st.hlen) == [0, 1] and np.all(np.isfinite(st.rho))


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


def _state_with_pairs(pairs_per_sample, d, m):
    N = len(pairs_per_sample)
    st = M.new_state(np.zeros((N, d)), m)
    for n, pairs in enumerate(pairs_per_sample):
        st.hlen[n] = len(pairs)
        for i, (s, y) in enumerate(pairs):                 # slot 0 = newest
            st.S[n, i], st.Y[n, i], st.rho[n, i] = s, y, 1.0 / (s @ y)
    return st


def test_laplace_widths_eigenvector_pairs_closed_form():
    """Pairs along eigenvectors v_i of an SPD B (y = B s): the inverse update of
    each pair leaves the others alone, so H = sum_i v_i v_i^T / lam_i over the
    stored pairs plus gamma times the projector onto the rest, gamma = 1 / lam of
    the newest pair.  A wrong gamma (oldest pair, or 1) or a dropped rho s s^T term
    changes H."""
    d, m = 6, 4
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.standard_normal((d, d)))
    lam = np.array([0.5, 2.0, 3.0, 7.0, 11.0, 13.0])
    used = [3, 0, 4]                                       # newest first
    pairs = [(2.5 * Qm[:, i], 2.5 * lam[i] * Qm[:, i]) for i in used]
    st = _state_with_pairs([pairs], d, m)
    H, w = M.laplace_widths(st, [0])
    Vu = Qm[:, used]
    P_rest = np.eye(d) - Vu @ Vu.T
    H_ref = Vu @ np.diag(1.0 / lam[used]) @ Vu.T + P_rest / lam[used[0]]
    np.testing.assert_allclose(H[0], H_ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(w[0], np.sqrt(np.diag(H_ref)), rtol=1e-12)


def test_laplace_widths_conjugate_pairs_give_the_inverse_hessian():
    """d pairs along B-conjugate directions (s_i^T B s_j = 0), y = B s: the L-BFGS
    matrix is B^-1 exactly, whatever gamma (the finite-termination property of
    BFGS on a quadratic), so the widths are sqrt(diag B^-1)."""
    d = 5
    rng = np.random.default_rng(8)
    C = rng.standard_normal((d, d))
    B = C @ C.T + 0.3 * np.eye(d)
    S = []
    for v in rng.standard_normal((d, d)):                 # B-orthogonalise (Gram-Schmidt)
        for s in S:
            v = v - (s @ B @ v) / (s @ B @ s) * s
        S.append(v)
    pairs = [(s, B @ s) for s in S[::-1]]
    st = _state_with_pairs([pairs], d, d)
    H, w = M.laplace_widths(st, [0])
    Binv = np.linalg.inv(B)
    np.testing.assert_allclose(H[0], Binv, rtol=1e-9, atol=1e-12 * np.abs(Binv).max())
    np.testing.assert_allclose(w[0], np.sqrt(np.diag(Binv)), rtol=1e-9)


def test_laplace_widths_secant_symmetry_and_empty_history():
    """Any history: H is symmetric positive definite and satisfies the secant
    equation H y = s of the newest pair; no pairs: H = I, widths 1."""
    d, m = 7, 5
    rng = np.random.default_rng(21)
    samples = []
    for n in range(4):
        Cm = rng.standard_normal((d, d))
        A = Cm @ Cm.T + 0.5 * np.eye(d)
        samples.append([(s, A @ s) for s in rng.standard_normal((n + 1, d))])
    samples.append([])
    st = _state_with_pairs(samples, d, m)
    H, w = M.laplace_widths(st, np.arange(5))
    for n in range(4):
        s0, y0 = samples[n][0]
        np.testing.assert_allclose(H[n] @ y0, s0, rtol=1e-9, atol=1e-12 * np.abs(s0).max())
        np.testing.assert_allclose(H[n], H[n].T, rtol=1e-9, atol=1e-12 * np.abs(H[n]).max())
        assert np.linalg.eigvalsh(H[n]).min() > 0
    np.testing.assert_array_equal(H[4], np.eye(d))
    np.testing.assert_array_equal(w[4], np.ones(d))


def test_underflowing_descent_product_keeps_the_history():
    """Next to a stationary point g^T p can underflow to 0 (here |g| = 1e-170): that
    is not an ascent direction, so the history (the mode's curvature estimate) is
    kept; an ascent direction (g^T p > 0) still clears it."""
    d, m = 3, 4
    prob = I.small_quadratic(d, 2, seed=3)
    P = M.Params(m=m, grad_mode=M.GRAD_ADJOINT)
    st = M.new_state(np.zeros((2, d)), m)
    A = np.diag([1.0, 2.0, 3.0])
    for n in range(2):
        for k, s in enumerate(np.eye(d)[:2]):
            st.S[n, k], st.Y[n, k], st.rho[n, k] = s, A @ s, 1.0 / (s @ A @ s)
        st.hlen[n] = 2
    st.x = np.asarray(prob.objective.arrays["center"], np.float64)[None].repeat(2, axis=0)
    G = np.array([1e-170, 0.0, 0.0])
    Pd = M.lbfgs_direction(G[None], st.S[:1], st.Y[:1], st.rho[:1], st.hlen[:1])
    assert np.einsum("nd,nd->n", G[None], Pd)[0] == 0.0          # the product underflows
    st.f = np.zeros(2)
    st.g = -np.stack([G, G])                                     # grad f = -grad F
    M.lbfgs_iterations(prob, st, P, 1, fresh_gradient=False)
    assert list(st.hlen) == [2, 2]
    # a pair with negative curvature makes p an ascent direction: the history is cleared
    # (the restart along -grad F then fails its search here, which leaves it empty)
    st2 = M.new_state(np.zeros((1, d)), m)
    s, y = np.array([1.0, 0.0, 0.0]), np.array([-1.0, 0.0, 0.0])
    st2.S[0, 0], st2.Y[0, 0], st2.rho[0, 0], st2.hlen[0] = s, y, 1.0 / (s @ y), 1
    st2.x = st.x[:1].copy()
    st2.g = np.array([[1.0, 0.0, 0.0]])
    st2.f = M.evaluate(prob, st2.x)
    M.lbfgs_iterations(prob, st2, P, 1, fresh_gradient=False)
    assert st2.hlen[0] == 0


@pytest.mark.parametrize("eps,kept", [(2e-10, True), (0.5e-10, False), (-0.5e-10, False), (-1.0, False)])
def test_curvature_pair_threshold(eps, kept):
    """The reading of the curvature skip: a pair is kept iff s^T y > 1e-10 |s| |y|,
    checked on both sides of the threshold and for slightly negative curvature."""
    P = M.Params(m=3)
    st = M.new_state(np.zeros((1, 2)), P.m)
    s = np.array([[1.0, 0.0]])
    y = np.array([[eps, 1.0]])                       # s^T y = eps, |s| |y| = sqrt(1 + eps^2)
    ok = M.push_pair(st, np.array([0]), s, y, P)
    assert bool(ok[0]) == kept and st.hlen[0] == int(kept)


def _conjugate_pairs(rng, B, d):
    S = []
    for v in rng.standard_normal((d, d)):                 # B-orthogonalise (Gram-Schmidt)
        for s in S:
            v = v - (s @ B @ v) / (s @ B @ s) * s
        S.append(v)
    return [(s, B @ s) for s in S[::-1]]


def test_refine_with_kept_history_takes_the_newton_step():
    """Final refinement (reading of the FP32 polish of tensor-core modes): a survivor of
    the quadratic f = -(x - c)^T A (x - c) whose kept history holds d A-conjugate pairs
    (y = 2 A s for F = -f) has H = (2A)^-1, so one refinement iteration is the Newton
    step and lands on c (alpha = 1 passes Armijo).  A cleared history would take a
    steepest-descent step instead; a non-survivor or a removed sample must not move."""
    d = 4
    rng = np.random.default_rng(21)
    prob = I.small_quadratic(d, 3, seed=5, cond=50.0)
    A = prob.objective.arrays["Q"].T @ np.diag(prob.objective.arrays["lam"]) @ prob.objective.arrays["Q"]
    c = prob.objective.arrays["center"]
    st = _state_with_pairs([_conjugate_pairs(rng, 2.0 * A, d)] * 3, d, d)
    st.x = c + rng.uniform(-1.0, 1.0, (3, d))
    x_before = st.x.copy()
    st.stuck = np.array([True, False, True])
    st.removed = np.array([False, False, True])
    st.stuck &= ~st.removed
    M.refine(prob, st, M.Params(m=d, grad_mode=M.GRAD_ADJOINT), 1)
    np.testing.assert_allclose(st.x[0], c, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(st.x[1:], x_before[1:])
    assert st.hlen[0] == d and st.hlen[1] == d


def test_refine_reaches_a_stationary_point_of_the_exact_objective():
    """Cycles on the tensor-core objective (BF16-rounded precision factors) stop at that
    objective's modes; refinement on the exact mixture moves each survivor to a point
    where the exact gradient vanishes (the definition of a mode), starting from the
    kept history of the lower-precision run."""
    from oracle import objectives as OB
    prob = I.small_full_mixture(6, 3, 40, seed=3, box=4.0)
    tprob = I.Problem(prob.d, prob.n, prob.lo, prob.hi, OB.tensor_core_objective(prob.objective), prob.x0,
                      prob.eps_grad, prob.sigma_mode)
    P = M.Params(m=6, grad_mode=M.GRAD_ADJOINT, n_conv=200, eps_grad=1e-6)
    st = M.new_state(prob.x0, P.m)
    M.lbfgs_iterations(tprob, st, P, 200)
    # the split input x_hi + x_lo (relative residual 2^-17) leaves a gradient floor near 1e-5
    st.stuck = np.abs(st.g).max(axis=1) < 1e-4
    assert st.stuck.sum() >= 5
    g_exact = np.abs(OB.grad(prob.objective, st.x[st.stuck])).max(axis=1)
    assert g_exact.max() > 1e-6                         # not yet modes of the exact objective
    M.refine(prob, st, P, 50)
    g_after = np.abs(OB.grad(prob.objective, st.x[st.stuck])).max(axis=1)
    assert g_after.max() < 1e-9
