"""Whole-cycle pins for the oracle (Algorithm 1, Propositions 1-2, Remark 1)."""
import numpy as np
import pytest

from oracle import method as M
from oracle import modes as MD
from paper_2606_26164_gb300 import inputs as I


def test_newton_modes_of_symmetric_mixture():
    """Four equal isotropic components at (+-3, +-3), sigma = 0.5: the modes sit at
    the means up to exp(-72) cross-talk and all pass the delta gate."""
    p = I.mixture4_d2()
    mx, mf, negH = MD.significant_modes(p)
    assert mx.shape == (4, 2)
    got = sorted(map(tuple, np.round(mx, 9)))
    assert got == sorted([(3.0, 3.0), (3.0, -3.0), (-3.0, 3.0), (-3.0, -3.0)])
    np.testing.assert_allclose(mf, np.log(0.25) - np.log(2 * np.pi * 0.25), rtol=1e-12)
    np.testing.assert_allclose(negH, np.broadcast_to(4.0 * np.eye(2), (4, 2, 2)), rtol=1e-9)


def test_delta_gate_drops_low_modes():
    obj = I.Objective(1, 1, {"weights": np.array([0.75, 0.2, 0.05]), "means": np.array([[0.0], [10.0], [20.0]]),
                             "sigmas": np.ones((3, 1))})
    p = I.Problem(1, 1, np.array([-5.0]), np.array([25.0]), obj, np.zeros((1, 1), np.float32), 1e-6, 1.0)
    mx, mf, _ = MD.significant_modes(p, delta=0.1)
    # log(0.2/0.75) = -1.32 passes the gate log 0.1 = -2.30; log(0.05/0.75) = -2.71 does not
    assert mx.shape[0] == 2


def test_single_mode_cycle_collapses():
    """Remark 1: a unimodal objective is solved by the first Phase 1 alone: all
    samples reach the maximum, all are stuck, and one survives deduplication."""
    p = I.small_quadratic(3, 64, seed=11, cond=4.0)
    P = M.Params(n_osc=1, n_conv=40, m=5, eps_grad=1e-8, grad_mode=M.GRAD_ADJOINT)
    st = M.new_state(p.x0, P.m)
    M.cycle(p, st, P)
    assert st.last_k_lost == 63
    fx, _ = M.modes_of(st)
    assert fx.shape[0] == 1
    np.testing.assert_allclose(fx[0], p.objective.arrays["center"], atol=1e-9)


def test_first_pass_coverage_probability():
    """Proposition 2: N i.i.d. uniform samples miss a mode with probability
    (1 - V_k/vol)^N after the first convergence phase.  In the symmetric
    4-mode square each basin is one quadrant (V_k/vol = 1/4), so with N = 4
    the (+3, +3) mode is missed with probability (3/4)^4."""
    p = I.mixture4_d2()
    trials, n = 600, 4
    rng = np.random.default_rng(17)
    x0 = rng.uniform(-6, 6, size=(trials * n, 2))
    P = M.Params(m=5, grad_mode=M.GRAD_ADJOINT)
    st = M.new_state(x0, P.m)
    M.lbfgs_iterations(p, st, P, 30)
    hit = (np.abs(st.x - np.array([3.0, 3.0])).max(axis=1) < 1e-3).reshape(trials, n).any(axis=1)
    miss = 1.0 - hit.mean()
    expect = 0.75 ** n
    assert abs(miss - expect) < 4 * np.sqrt(expect * (1 - expect) / trials)


def test_full_run_recovers_all_four_modes():
    p = I.mixture4_d2(n=256)
    P = M.Params(n_osc=3, m=5, eps_grad=1e-5, grad_mode=M.GRAD_FD64, seed=0)
    (fx, ff), st = M.run(p, P)
    mx, mf, negH = MD.significant_modes(p)
    frac, worst, _ = MD.recovery(fx, mx, negH)
    assert frac == 1.0 and worst < 1e-3
    assert fx.shape[0] == 4                                  # no spurious modes


def test_mahalanobis_recovery_metric():
    mx = np.array([[0.0, 0.0]])
    negH = np.array([np.diag([4.0, 1.0])])
    found = np.array([[4e-4, 0.0], [0.0, 2e-3]])
    frac, worst, best = MD.recovery(found, mx, negH)
    assert frac == 1.0 and abs(best[0] - 8e-4) < 1e-15


@pytest.mark.parametrize("noise", [0.0, 1.0])
def test_two_mode_d6_noise_workload_both_peaks(noise):
    """The Sec. 5.6 workload (d = 6, unit components at +-2 e_1): with exact
    gradients the evaluation noise enters only through the Armijo test and the
    quality gate, and both peaks are returned with nothing else."""
    prob = I.mixture2_d6(n=256, seed=0, noise_sigma=noise)
    P = M.Params(n_osc=3, m=10, eps_grad=prob.eps_grad, grad_mode=M.GRAD_ADJOINT, seed=0)
    (ox, of), _ = M.run(prob, P)
    mx, mf, negH = MD.significant_modes(prob)
    assert len(mx) == 2 and abs(abs(mx[0][0]) - 2.0) < 2e-3     # x = 2 tanh(2 x): 1.99865
    frac, worst, _ = MD.recovery(ox, mx, negH)
    assert frac == 1.0 and ox.shape[0] == 2
