"""A caller-supplied batched objective (CHISAO_OBJ_EXTERNAL): the objective is a
torch function of a batch of points that the library calls on its stream, and
the cycle runs Phases 1, 5 and 6 as per-sample kernels around those calls.

The torch functions below compute the workloads' objectives in binary32; the
oracle evaluates the same objectives in FP64, so the tolerances are those of
the built-in binary32 objectives' parity tests."""
import dataclasses
import math

import numpy as np
import pytest

import gpu_util as U
from oracle import method as M
from oracle import modes as MD
from oracle import objectives as OB
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _torch_fn(obj):
    """(f, exact gradient) of a built-in objective, written with torch ops."""
    import torch
    A = {k: torch.as_tensor(np.asarray(v), dtype=torch.float32, device="cuda") for k, v in obj.arrays.items()}
    if obj.kind == I.OBJ_QUADRATIC:
        Amat = A["Q"].T @ (A["lam"][:, None] * A["Q"])

        def fn(x):
            r = x - A["center"]
            u = r @ Amat
            return -(r * u).sum(dim=1), -2.0 * u
        return fn
    assert obj.kind == I.OBJ_MIXTURE_DIAG
    logc = torch.log(A["weights"]) - torch.log(A["sigmas"]).sum(dim=1) - 0.5 * obj.d * math.log(2 * math.pi)

    def fval(x):
        z = (x[:, None, :] - A["means"][None]) / A["sigmas"][None]
        return torch.logsumexp(logc[None] - 0.5 * (z * z).sum(dim=2), dim=1)
    return CH.autograd_objective(fval)


def _external(prob):
    ob = prob.objective
    ext = I.Objective(I.OBJ_EXTERNAL, ob.d, {}, fn=_torch_fn(ob))
    return dataclasses.replace(prob, objective=ext)


def _copy(st):
    return M.State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.__dict__.items()})


PROBS = {
    "mix_d5": lambda n: I.small_mixture(5, 7, n, seed=2),
    "quad_d7": lambda n: I.small_quadratic(7, n, seed=7),
    "mix_d16": lambda n: I.small_mixture(16, 32, n, seed=3, box=10.0),
}


@pytest.mark.parametrize("name", list(PROBS))
def test_external_objective_eval(name):
    prob = PROBS[name](333)
    model = U.open_ctx(_external(prob), M.Params(grad_mode=M.GRAD_ADJOINT))
    import torch
    X = torch.from_numpy(prob.x0).cuda()
    f, g = model.eval(0, X, CH.GRAD_ADJOINT)
    x64 = prob.x0.astype(np.float64)
    f_ref, g_ref = OB.value(prob.objective, x64), OB.grad(prob.objective, x64)
    np.testing.assert_allclose(f.cpu().numpy(), f_ref, rtol=1e-5, atol=1e-5 * np.abs(f_ref).max())
    err = U.rel_err_rows(g.cpu().numpy(), g_ref, floor=1e-3 * np.abs(g_ref).max())
    assert err.max() <= 1e-4, err.max()
    model.close()


@pytest.mark.parametrize("name", list(PROBS))
def test_external_objective_lbfgs_iteration(name):
    """One Phase-1 iteration around the external evaluator (direction, T_ls
    rounds of batched trial evaluations, acceptance, history push) against the
    oracle from the same binary32 state."""
    prob = PROBS[name](700)
    P = M.Params(m=6, grad_mode=M.GRAD_ADJOINT)
    st = M.new_state(prob.x0, P.m)
    M.lbfgs_iterations(prob, st, P, 3)
    st = U.rounded(st)
    st.f = M.evaluate(prob, st.x)
    st.g = M.gradient(prob, st.x, P)
    st = U.rounded(st)
    model = U.open_ctx(_external(prob), P)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_LBFGS, -1)
    got = U.read_state(model, prob, P.m)
    ref = _copy(st)
    M.lbfgs_iterations(prob, ref, P, 1, fresh_gradient=False)
    step = np.abs(ref.x - st.x).max(axis=1)
    err = np.abs(got.x - ref.x).max(axis=1)
    ok = err <= 1e-5 * step + 4e-7 * np.abs(st.x).max(axis=1)
    # binary32-vs-FP64 ties of the Armijo test may take the neighbouring trial
    assert (~ok).sum() <= 0.02 * prob.n, ((~ok).sum(), err[~ok][:5], step[~ok][:5])
    g_ref = OB.grad(prob.objective, got.x)
    gerr = U.rel_err_rows(got.g, g_ref, floor=1e-3 * np.abs(g_ref).max())
    assert np.quantile(gerr, 0.99) <= 1e-4
    assert np.all(got.hlen[ok] == ref.hlen[ok])
    model.close()


def test_external_objective_history_ring():
    """Several Phase-1 iterations in one call with a short memory (m = 3, five pushes
    onto two stored pairs): the pairs are kept in a ring during the phase and rotated
    back after it, so the history read back is the oracle's, newest first, slot by slot
    (s, y and rho of every sample whose path matched)."""
    prob = I.small_quadratic(7, 700, seed=8)
    P = M.Params(m=3, grad_mode=M.GRAD_ADJOINT)
    st = M.new_state(prob.x0, P.m)
    M.lbfgs_iterations(prob, st, P, 2)
    st = U.rounded(st)
    st.f = M.evaluate(prob, st.x)
    st.g = M.gradient(prob, st.x, P)
    st = U.rounded(st)
    model = U.open_ctx(_external(prob), P)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_LBFGS, -5)
    got = U.read_state(model, prob, P.m)
    ref = _copy(st)
    M.lbfgs_iterations(prob, ref, P, 5, fresh_gradient=False)
    step = np.abs(ref.x - st.x).max(axis=1)
    err = np.abs(got.x - ref.x).max(axis=1)
    ok = (err <= 1e-4 * step + 1e-6 * np.abs(st.x).max(axis=1)) & (got.hlen == ref.hlen)
    assert ok.sum() >= 0.9 * prob.n, ok.sum()
    assert np.all(ref.hlen[ok] == P.m)
    for k in range(P.m):
        for a, b in ((got.S[:, k], ref.S[:, k]), (got.Y[:, k], ref.Y[:, k])):
            scale = np.abs(b).max(axis=1) + 1e-30
            e = np.abs(a - b).max(axis=1) / scale
            assert np.all(e[ok] <= 1e-3), (k, np.sort(e[ok])[-5:])
        r = np.abs(got.rho[:, k] - ref.rho[:, k]) / np.abs(ref.rho[:, k])
        assert np.all(r[ok] <= 1e-3), (k, np.sort(r[ok])[-5:])
    model.close()


def test_external_objective_hlc_and_anti_single_steps():
    prob = PROBS["mix_d5"](901)
    rng = np.random.default_rng(5)
    for phase in ("hlc", "anti"):
        P = M.Params(n_cloud=1, n_anti=1, M=8, grad_mode=M.GRAD_ADJOINT, seed=7)
        st = M.new_state(prob.x0 * np.float32(0.7), P.m)
        st.stuck = rng.random(prob.n) < 0.3
        st = U.rounded(st)
        model = U.open_ctx(_external(prob), P)
        U.write_state(model, prob, st)
        ref = _copy(st)
        if phase == "hlc":
            model.run_phase(0, CH.PHASE_HLC, 2)
            M.hlc(prob, ref, P, cycle=2)
        else:
            model.run_phase(0, CH.PHASE_ANTI)
            M.anti_converge(prob, ref, P)
        got = U.read_state(model, prob, P.m)
        moved = np.abs(ref.x - st.x).max(axis=1)
        err = np.abs(got.x - ref.x).max(axis=1)
        tol = 1e-4 * moved + 2e-6 * np.abs(st.x).max(axis=1)
        assert np.all(err <= tol), (phase, (err / tol).max())
        np.testing.assert_array_equal(got.x[st.stuck], st.x[st.stuck])
        model.close()


def test_external_objective_cycles_recover_the_modes():
    """d = 2, four isotropic components: whole cycles around the torch evaluator
    return the four modes within 1e-3 sigma, as the built-in objective does."""
    prob = I.mixture4_d2(n=1024)
    P = M.Params(n_osc=3, m=5, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=0)
    model = U.open_ctx(_external(prob), P)
    for _ in range(P.n_osc):
        model.step()
    fx, ff = model.modes(0)
    mx, mf, negH = MD.significant_modes(prob)
    frac, worst, _ = MD.recovery(fx, mx, negH)
    assert frac == 1.0 and worst <= 1e-3 and fx.shape[0] == 4
    c = model.counters(0)
    assert c["cycles"] == 3 and c["evals"] > 0 and c["grads"] > 0
    model.close()


def test_external_objective_errors_are_reported():
    prob = PROBS["quad_d7"](64)

    def broken(x):
        raise ValueError("objective failed")
    ext = dataclasses.replace(prob, objective=I.Objective(I.OBJ_EXTERNAL, prob.d, {}, fn=broken))
    model = U.open_ctx(ext, M.Params(n_osc=2, grad_mode=M.GRAD_ADJOINT))
    with pytest.raises(CH.ChisaoError, match="objective failed"):
        model.step()
    model.close()
    # an external objective needs exact gradients
    with pytest.raises(CH.ChisaoError):
        U.open_ctx(_external(prob), M.Params(grad_mode=M.GRAD_FD64))


def test_external_objectives_in_one_context_match_separate_ones():
    """Two problems with external objectives in one context (each on its own branch
    stream, the evaluator called with that stream) give the states of two separate
    contexts bit for bit."""
    import torch
    probs = [_external(PROBS["quad_d7"](300)), _external(PROBS["mix_d5"](400))]
    P = M.Params(n_osc=3, m=6, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=4)
    U.ensure_built()
    # leave garbage in the allocator's cache, so the arenas below start dirty: nothing may
    # depend on memory the library has not written (e.g. gradient padding, d < dp here)
    junk = torch.full((64 << 20,), float("nan"), device="cuda")
    del junk
    together = CH.Chisao(probs, U.lib_params(P))
    for _ in range(2):
        together.step()
    for q in range(2):
        alone = CH.Chisao(probs[:q + 1], U.lib_params(P))
        for _ in range(2):
            alone.step()
        for fld in (CH.FIELD_X, CH.FIELD_F, CH.FIELD_STUCK):
            np.testing.assert_array_equal(alone.get(q, fld), together.get(q, fld))
        alone.close()
    assert together.autotune()["trials"] == 0             # evaluators need not be capture-safe
    together.close()
