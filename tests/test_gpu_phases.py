"""Parity of Phases 4-6 (reseeding, Hands Like Clouds, anti-convergence) with
the oracle from identical binary32 state and the same Philox streams.

Reseeding: the strategy, the parent / peak / column / sign indices (integer
Philox arithmetic on both sides) and therefore every child's ray are
identical; positions agree to binary32 rounding (1e-5 of the box width).
HLC and anti-convergence: positions agree to 1e-5 of the distance moved plus
binary32 rounding of the position; the scale estimates to 1e-6.
"""
import zlib

import numpy as np
import pytest

import gpu_util as U
from oracle import method as M
from oracle import objectives as OB
from oracle import philox as PX
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _reseed_case(case, d, N, rng):
    stuck = rng.random(N) < 0.6
    removed = stuck & (rng.random(N) < 0.4)
    gr = (0, 0, -1)
    if case in ("gr", "gr_off", "no_surv"):
        stuck = np.ones(N, bool)
        stuck[rng.choice(N, 3, replace=False)] = False          # 3 unfrozen: Golden Rooster
        removed = stuck & (rng.random(N) < 0.5)
        if case == "no_surv":
            removed = stuck.copy()
    if case == "none":
        removed[:] = False
    if case == "gr_off":
        gr = (1, 1, int((stuck & ~removed).sum()))               # no growth again -> disabled
    else:
        gr = (1, 0, -1)
    return stuck, removed, gr


@pytest.mark.parametrize("case,d", [("rm", 5), ("rm", 64), ("gr", 5), ("gr", 64), ("gr_off", 8),
                                    ("none", 5), ("no_surv", 3), ("rm_large", 7), ("gr_large", 3)])
def test_reseed(case, d):
    """The _large cases (N = 70001, 2188 mask words) run the ordered compactions over
    several 32-word rounds per warp with a ragged last word: the parents Repulse Monkey
    draws by position in the unfrozen list, and the peaks Golden Rooster takes by rank
    from the survivor list, come out right only if the lists are in index order."""
    rng = np.random.default_rng(zlib.crc32(f"{case}{d}".encode()))
    N = 70001 if case.endswith("_large") else 777
    case = case.replace("_large", "")
    prob = I.small_mixture(d, 3, N, seed=12)
    P = M.Params(seed=21)
    stuck, removed, gr = _reseed_case(case, d, N, rng)
    st = M.new_state(prob.x0, P.m)
    st.f = rng.normal(0, 1, N).astype(np.float32).astype(np.float64)
    st.hlen[:] = 2
    st = U.rounded(st)
    model = U.open_ctx(prob, P)
    st.stuck, st.removed = stuck, removed
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_LISTS)
    model.set_gr_state(0, *gr)
    model.run_phase(0, CH.PHASE_RESEED, 3)
    got = U.read_state(model, prob, P.m)
    ref = M.State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.__dict__.items()})
    ref.stuck = stuck & ~removed
    ref.gr_enabled, ref.gr_noprog, ref.gr_prev_surv = bool(gr[0]), gr[1], gr[2]
    M.reseed(prob, ref, P, cycle=3)
    c = model.counters(0)
    assert c["last_reseed"] == ref.last_reseed
    assert c["gr_enabled"] == int(ref.gr_enabled)
    width = (prob.hi - prob.lo).max()
    np.testing.assert_allclose(got.x, ref.x, rtol=0, atol=1e-5 * width)
    untouched = ~removed
    np.testing.assert_array_equal(got.x[untouched], st.x[untouched])
    assert np.all(got.hlen[removed] == 0) and np.all(got.hlen[untouched] == 2)
    model.close()


def _copy(st):
    return M.State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.__dict__.items()})


def _sensitivity(run, st, seed=0):
    """How far the oracle's own result moves when its input positions are
    perturbed at the binary32 rounding level (relative 2^-24): the part of a
    multi-step difference that input rounding alone explains."""
    pert = _copy(st)
    rng = np.random.default_rng(seed)
    pert.x = st.x * (1.0 + 2.0 ** -24 * rng.choice([-1.0, 1.0], size=st.x.shape))
    a, b = _copy(st), pert
    run(a)
    run(b)
    return np.abs(a.x - b.x).max(axis=1)


def _check_moves(got, ref, st, sens, rtol, extra=0.0):
    move = np.abs(ref.x - st.x).max(axis=1)
    err = np.abs(got.x - ref.x).max(axis=1)
    tol = rtol * move + 2e-6 * np.abs(st.x).max(axis=1) + 20.0 * sens + extra
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-30)).max()


U32 = 2.0 ** -24

# Problems of the smoothed-gradient and momentum parity tests.  The quadratic runs
# at 1, 4, 8 and 16 lanes per sample (d = 3, 12, 27, 64; condition up to 1e4, the
# benchmark's), through its own multi-point products in Hands Like Clouds; the
# full-covariance mixture through its binary32 row-walk products.
PHASE_PROBS = {
    "mix_d3": lambda n: I.small_mixture(3, 4, n, seed=13),
    "mix_d16": lambda n: I.small_mixture(16, 4, n, seed=13),
    "quad_d3": lambda n: I.small_quadratic(3, n, seed=41),
    "quad_d12": lambda n: I.small_quadratic(12, n, seed=42, cond=1e3),
    "quad_d27": lambda n: I.small_quadratic(27, n, seed=43, cond=1e4),
    "quad_d64": lambda n: I.small_quadratic(64, n, seed=44, cond=1e4),
    "full_d8": lambda n: I.small_full_mixture(8, 5, n, seed=45),
    "full_d33": lambda n: I.small_full_mixture(33, 6, n, seed=46),
}


def _grad_bound(prob, X, mode):
    """Per-row bound on |g_device - g_oracle|_inf at points X: the objective parity
    bound for exact gradients (1e-5 of the summed terms' magnitude plus the
    softmax's sensitivity to binary32 log-densities), 1e-6 of the terms for FD64
    (FP64 stencil on both sides, binary32 storage)."""
    from test_gpu_kernels import grad_term_scale, softmax_error_scale
    if mode == M.GRAD_ADJOINT:
        return 1e-5 * grad_term_scale(prob, X) + U32 * softmax_error_scale(prob, X)
    return 1e-6 * grad_term_scale(prob, X)


def _amplification(sens, st):
    """How much the oracle's multi-step map amplifies an input perturbation: its
    change under the relative 2^-24 perturbation over that perturbation's size."""
    return np.maximum(1.0, sens / (U32 * np.maximum(np.abs(st.x).max(axis=1), 1e-30)))


def _alpha_rel(prob, st, unf, mode):
    """Relative error bound of the step size 0.1 s / g_rms: the device forms g_rms from
    its own gradients, each within _grad_bound of the oracle's."""
    from oracle import objectives as OBJ
    g = OBJ.grad(prob.objective, st.x[unf])
    b = _grad_bound(prob, st.x[unf], mode)
    return float(np.sqrt(np.mean(b ** 2)) / max(np.sqrt(np.mean(g ** 2)), 1e-300))


HLC_CASES = ([(nm, mode, nc, 8) for nm in ("mix_d3", "mix_d16") for mode in (M.GRAD_ADJOINT, M.GRAD_FD64)
              for nc in (1, 3)]
             + [(nm, M.GRAD_ADJOINT, nc, Mk) for nm in ("quad_d3", "quad_d12", "quad_d27", "quad_d64")
                for nc in (1, 3) for Mk in (7, 8)]
             + [(nm, M.GRAD_FD64, 1, 8) for nm in ("quad_d12", "quad_d64")]
             # d <= 4 with finite differences: the perturbations run on separate lanes (k_hlc_wide),
             # M = 7 leaving one lane of each sample idle
             + [("quad_d3", M.GRAD_FD64, nc, Mk) for nc in (1, 3) for Mk in (7, 8)]
             + [(nm, mode, nc, 8) for nm in ("full_d8", "full_d33") for mode in (M.GRAD_ADJOINT, M.GRAD_FD64)
                for nc in (1, 3)])


@pytest.mark.parametrize("name,mode,n_cloud,Mk", HLC_CASES)
def test_hands_like_clouds(name, mode, n_cloud, Mk):
    """Phase 5 (Eq. 5) from identical binary32 state: M = 7 makes the quadratic run its
    four-point, two-point and single-point products in one step, M = 8 (the
    benchmark's) two four-point passes.  Positions within 1e-5 of the move, plus the
    gradient rounding bound carried through the step (alpha times the mean bound at
    the perturbed points, amplified as the oracle's own map amplifies input rounding
    over several steps), plus 20 times that input sensitivity."""
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    N = 901
    prob = PHASE_PROBS[name](N)
    P = M.Params(n_cloud=n_cloud, M=Mk, grad_mode=mode, seed=3)
    st = M.new_state(prob.x0, P.m)
    st.stuck = rng.random(N) < 0.3
    st.hlen[:] = 1
    st = U.rounded(st)
    model = U.open_ctx(prob, P)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_HLC, 2)
    got = U.read_state(model, prob, P.m)
    ref = _copy(st)
    sigma, alpha = M.hlc(prob, ref, P, cycle=2)
    unf = np.flatnonzero(~st.stuck)
    rel_a = _alpha_rel(prob, st, unf, mode)
    c = model.counters(0)
    assert c["sigma"] == pytest.approx(sigma, rel=1e-6)
    assert c["alpha_hlc"] == pytest.approx(alpha, rel=max(1e-5, 1.01 * rel_a))
    gb = np.zeros(N)
    for k in range(Mk):
        zk = PX.normal_rows(3, unf, prob.d, PX.TAG_HLC, 2, 0, 0, k)
        gb[unf] += _grad_bound(prob, st.x[unf] + sigma * zk, mode) / Mk
    gb *= alpha
    if n_cloud == 1:
        sens, extra = 0.0, gb
    else:
        sens = _sensitivity(lambda s: M.hlc(prob, s, P, cycle=2), st)
        extra = n_cloud * _amplification(sens, st) * gb
    _check_moves(got, ref, st, sens, 1e-5 + 1.01 * rel_a, extra)
    np.testing.assert_array_equal(got.x[st.stuck], st.x[st.stuck])
    assert np.all(got.hlen[~st.stuck] == 0) and np.all(got.hlen[st.stuck] == 1)
    model.close()


@pytest.mark.parametrize("mode", [M.GRAD_ADJOINT, M.GRAD_FD64])
@pytest.mark.parametrize("d", [3, 16])
def test_hands_like_clouds_value_only(mode, d):
    """The value-only smoothing variant, one step: the same Philox perturbations,
    the estimator (f(x + sigma z) - f(x)) z / sigma from binary32 (FD64 mode: FP64)
    values.  Besides 1e-5 of the move, the device's rounding of f (a few u of the
    magnitude of the values) enters through the division by sigma."""
    rng = np.random.default_rng(d + 7)
    N = 777
    prob = I.small_mixture(d, 4, N, seed=13)
    P = M.Params(n_cloud=1, M=8, grad_mode=mode, seed=3, hlc_value_only=1)
    st = M.new_state(prob.x0, P.m)
    st.stuck = rng.random(N) < 0.3
    st = U.rounded(st)
    model = U.open_ctx(prob, P)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_HLC, 2)
    got = U.read_state(model, prob, P.m)
    ref = _copy(st)
    sigma, alpha = M.hlc(prob, ref, P, cycle=2)
    c = model.counters(0)
    assert c["sigma"] == pytest.approx(sigma, rel=1e-6)
    unf = np.flatnonzero(~st.stuck)
    X = st.x[unf]
    fabs = np.abs(OB.value(prob.objective, X))
    zsum = np.zeros_like(X)
    for k in range(8):
        z = PX.normal_rows(3, unf, d, PX.TAG_HLC, 2, 0, 0, k)
        fabs = np.maximum(fabs, np.abs(OB.value(prob.objective, X + sigma * z)))
        zsum += np.abs(z)
    # binary32 values: each f carries ~ (d + 4) u |f| (the log-sum-exp and its terms),
    # and the perturbed point is rounded before the evaluation (|grad f| u |x|)
    u = 2.0 ** -24 if mode == M.GRAD_ADJOINT else 2.0 ** -50
    gscale = np.abs(OB.grad(prob.objective, X)).max(axis=1) * np.abs(X).max(axis=1) + 1.0
    ferr = 32 * (d + 4) * u * (fabs + 1.0) + 4 * 2.0 ** -24 * gscale
    bound = alpha * (2 * ferr / sigma)[:, None] * zsum / 8
    move = np.abs(ref.x[unf] - X).max(axis=1)
    err = np.abs(got.x[unf] - ref.x[unf])
    tol = 1e-5 * move[:, None] + bound + 2e-6 * np.abs(X)
    assert np.all(err <= tol), (err / tol).max()
    np.testing.assert_array_equal(got.x[st.stuck], st.x[st.stuck])
    model.close()


ANTI_CASES = ([(nm, mode, na) for nm in ("mix_d3", "mix_d16") for mode in (M.GRAD_ADJOINT, M.GRAD_FD64)
               for na in (1, 5)]
              + [(nm, M.GRAD_ADJOINT, na) for nm in ("quad_d3", "quad_d12", "quad_d27", "quad_d64") for na in (1, 5)]
              + [(nm, M.GRAD_FD64, 5) for nm in ("quad_d12", "quad_d64")]
              + [(nm, mode, na) for nm in ("full_d8", "full_d33") for mode in (M.GRAD_ADJOINT, M.GRAD_FD64)
                 for na in (1, 5)])


@pytest.mark.parametrize("name,mode,n_anti", ANTI_CASES)
def test_anti_convergence(name, mode, n_anti):
    """Phase 6 (Eq. 6) from identical binary32 state: positions within 1e-5 of the
    move plus the gradient rounding bound carried through the momentum recursion
    (step t sees sum_{s<=t} mu^(t-s) of the per-step bound, amplified as the
    oracle's own map amplifies input rounding), plus 20 times that sensitivity."""
    rng = np.random.default_rng(zlib.crc32(name.encode()) + 100)
    N = 1203
    prob = PHASE_PROBS[name](N)
    P = M.Params(n_anti=n_anti, mu=0.9, grad_mode=mode)
    st = M.new_state(prob.x0 * np.float32(0.8), P.m)
    st.stuck = rng.random(N) < 0.25
    st = U.rounded(st)
    model = U.open_ctx(prob, P)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_ANTI)
    got = U.read_state(model, prob, P.m)
    ref = _copy(st)
    alpha = M.anti_converge(prob, ref, P)
    unf = np.flatnonzero(~st.stuck)
    rel_a = _alpha_rel(prob, st, unf, mode)
    assert model.counters(0)["alpha_anti"] == pytest.approx(alpha, rel=max(1e-5, 1.01 * rel_a))
    gb = np.zeros(N)
    gb[unf] = alpha * _grad_bound(prob, st.x[unf], mode)
    carry = sum((1.0 - P.mu ** t) / (1.0 - P.mu) for t in range(1, n_anti + 1))
    if n_anti == 1:
        sens, extra = 0.0, gb
    else:
        sens = _sensitivity(lambda s: M.anti_converge(prob, s, P), st)
        extra = carry * _amplification(sens, st) * gb
    _check_moves(got, ref, st, sens, 1e-5 + 1.01 * rel_a, extra)
    np.testing.assert_array_equal(got.x[st.stuck], st.x[st.stuck])
    model.close()


# ----------------------------------------------------------------------- tensor-core mode
# The tensor-core path evaluates the mixture with BF16-rounded precision factors
# at the BF16-split input (oracle: objectives.tensor_core_objective); its
# gradients carry the error bound test_gpu_kernels.tc_error_bounds.

def _tc_problem(N, seed):
    prob = I.small_full_mixture(24, 10, N, seed=seed, box=6.0)
    tprob = I.Problem(prob.d, prob.n, prob.lo, prob.hi, OB.tensor_core_objective(prob.objective), prob.x0,
                      prob.eps_grad, prob.sigma_mode)
    return prob, tprob


def _tc_grad_bound(tprob, X):
    from test_gpu_kernels import tc_error_bounds
    return tc_error_bounds(tprob.objective, OB.bf16_split(X))[1].max(axis=1)


def test_tc_lbfgs_iteration():
    prob, tprob = _tc_problem(700, 31)
    P = M.Params(m=6, grad_mode=M.GRAD_ADJOINT)
    st = M.new_state(prob.x0, P.m)
    M.lbfgs_iterations(tprob, st, P, 3)
    st = U.rounded(st)
    st.f = M.evaluate(tprob, st.x)
    st.g = M.gradient(tprob, st.x, P)
    st = U.rounded(st)
    model = U.open_ctx(prob, P, grad_mode=CH.GRAD_ADJOINT_TC)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_LBFGS, -1)
    got = U.read_state(model, prob, P.m)
    ref = _copy(st)
    M.lbfgs_iterations(tprob, ref, P, 1, fresh_gradient=False)
    step = np.abs(ref.x - st.x).max(axis=1)
    err = np.abs(got.x - ref.x).max(axis=1)
    ok = err <= 1e-5 * step + 4e-7 * np.abs(st.x).max(axis=1)
    assert (~ok).sum() <= 0.02 * prob.n, ((~ok).sum(), err[~ok][:5], step[~ok][:5])
    gerr = np.abs(got.g - OB.grad(tprob.objective, got.x)).max(axis=1)
    assert np.all(gerr <= _tc_grad_bound(tprob, got.x))
    assert np.all(got.hlen[ok] == ref.hlen[ok])
    model.close()


def test_tc_hlc_and_anti_single_steps():
    prob, tprob = _tc_problem(901, 32)
    rng = np.random.default_rng(5)
    for phase in ("hlc", "anti"):
        P = M.Params(n_cloud=1, n_anti=1, M=8, grad_mode=M.GRAD_ADJOINT, seed=7)
        st = M.new_state(prob.x0 * np.float32(0.7), P.m)
        st.stuck = rng.random(prob.n) < 0.3
        st = U.rounded(st)
        model = U.open_ctx(prob, P, grad_mode=CH.GRAD_ADJOINT_TC)
        U.write_state(model, prob, st)
        ref = _copy(st)
        unf = np.flatnonzero(~st.stuck)
        # the step size alpha = 0.1 s / g_rms uses the tensor-core gradient at x: relative error <= rms(bound)/g_rms
        g_rms = np.sqrt(np.mean(OB.grad(tprob.objective, st.x[unf]) ** 2))
        rel_alpha = np.sqrt(np.mean(_tc_grad_bound(tprob, st.x[unf]) ** 2)) / g_rms
        if phase == "hlc":
            model.run_phase(0, CH.PHASE_HLC, 2)
            sigma, alpha = M.hlc(tprob, ref, P, cycle=2)
            bound = np.zeros(prob.n)
            for k in range(8):
                zk = PX.normal_rows(7, unf, prob.d, PX.TAG_HLC, 2, 0, 0, k)
                bound[unf] += _tc_grad_bound(tprob, st.x[unf] + sigma * zk) / 8.0
        else:
            model.run_phase(0, CH.PHASE_ANTI)
            alpha = M.anti_converge(tprob, ref, P)
            bound = _tc_grad_bound(tprob, st.x)
        got = U.read_state(model, prob, P.m)
        move = np.abs(ref.x - st.x).max(axis=1)
        err = np.abs(got.x - ref.x).max(axis=1)
        tol = 1.01 * alpha * bound + (1e-5 + 1.01 * rel_alpha) * move + 2e-6 * np.abs(st.x).max(axis=1)
        assert np.all(err <= tol), (phase, (err / tol).max())
        np.testing.assert_array_equal(got.x[st.stuck], st.x[st.stuck])
        model.close()


@pytest.mark.parametrize("method", [CH.SEED_UNIFORM, CH.SEED_CARRY_TIGER])
@pytest.mark.parametrize("d", [2, 7, 64])
def test_seeding(method, d):
    """Device populations against the oracle's: the same Philox words, so the same
    anchors and ray positions; binary32 coordinates within a few ulp of the box."""
    from oracle import seeding as SD
    prob = I.small_mixture(d, 2, 3001, seed=5)
    prob.lo = prob.lo - np.arange(d) * 0.5                 # an asymmetric box
    P = M.Params(seed=17)
    model = U.open_ctx(prob, P)
    model.seed(0, method)
    x = model.get(0, CH.FIELD_X)[:, :d].astype(np.float64)
    lo32, hi32 = prob.lo.astype(np.float32).astype(np.float64), prob.hi.astype(np.float32).astype(np.float64)
    f = SD.uniform if method == CH.SEED_UNIFORM else SD.carry_tiger
    ref = f(lo32, hi32, prob.n, seed=17)
    scale = np.abs(lo32) + np.abs(hi32)
    np.testing.assert_allclose(x, ref, rtol=0, atol=4 * 2.0 ** -24 * scale.max())
    assert np.all((x >= lo32) & (x <= hi32))
    if method == CH.SEED_CARRY_TIGER:
        E, _ = SD.carry_tiger_directions(d, prob.n, seed=17)
        c = (0.5 * (lo32 + hi32)).astype(np.float32).astype(np.float64)
        np.testing.assert_array_equal(x[E == 0], np.broadcast_to(c, x.shape)[E == 0])   # off-ray axes at the centre
    assert model.counters(0)["cycles"] == 0
    model.close()


def _history(rng, N, d, m, hlen):
    S = np.zeros((N, m, d))
    Y = np.zeros((N, m, d))
    for n in range(N):
        B = rng.standard_normal((d, d)) / np.sqrt(d)
        A = B @ B.T + 0.5 * np.eye(d)
        for k in range(hlen[n]):
            s = rng.standard_normal(d)
            S[n, k], Y[n, k] = s, A @ s
    return S, Y


@pytest.mark.parametrize("d,m,p_stuck", [(2, 5, 0.5), (5, 10, 0.3), (16, 10, 0.7), (64, 10, 0.2), (7, 4, 0.0)])
def test_laplace_widths(d, m, p_stuck):
    """Widths and inverse-Hessian rows of the survivors from their stored history
    (empty histories included: H = I) against the oracle on the same binary32
    pairs; survivors in sample-index order, none at all when nothing is stuck."""
    rng = np.random.default_rng(100 + d)
    N = 333
    prob = I.small_quadratic(d, N, seed=d)
    P = M.Params(m=m, grad_mode=M.GRAD_ADJOINT)
    model = U.open_ctx(prob, P)
    st = M.new_state(prob.x0, m)
    st.hlen = rng.integers(0, m + 1, size=N)
    st.S, st.Y = _history(rng, N, d, m, st.hlen)
    st = U.rounded(st)
    st.stuck = rng.random(N) < p_stuck
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_LISTS)
    w, H = model.widths(0, cov=True)
    idx = np.flatnonzero(st.stuck)
    assert w.shape == (idx.size, d) and H.shape == (idx.size, d, d)
    if idx.size == 0:
        model.close()
        return
    H_ref, w_ref = M.laplace_widths(st, idx)
    # H e_j in binary32: each row within 1e-5 of its norm (the direction test's bound)
    rows = H.reshape(-1, d).astype(np.float64)
    rows_ref = H_ref.reshape(-1, d)
    err = U.rel_err_rows(rows, rows_ref)
    assert err.max() <= 1e-5, err.max()
    # w^2 = H_jj within the same bound relative to |H e_j|
    scale = np.abs(H_ref).max(axis=2)
    assert np.all(np.abs(w.astype(np.float64) ** 2 - w_ref ** 2) <= 1e-5 * scale)
    empty = st.hlen[idx] == 0
    np.testing.assert_array_equal(w[empty], np.ones((empty.sum(), d), np.float32))
    w_only, none = model.widths(0)
    assert none is None
    np.testing.assert_array_equal(w_only, w)
    model.close()


def test_laplace_widths_after_cycles_match_the_mode_curvature():
    """d = 2, four isotropic components (sigma = 0.5): after the cycles every
    mode's width from its kept history is the Laplace width sqrt(diag(-Hess f)^-1)
    at the returned point to 1 %."""
    prob = I.mixture4_d2(n=1024)
    P = M.Params(n_osc=3, m=5, eps_grad=1e-4, grad_mode=M.GRAD_ADJOINT, seed=0)
    model = U.open_ctx(prob, P)
    for _ in range(P.n_osc):
        model.step()
    fx, _ = model.modes(0)
    w, _ = model.widths(0)
    assert fx.shape[0] == 4 and w.shape == (4, 2)
    for x, wr in zip(fx.astype(np.float64), w.astype(np.float64)):
        lap = np.sqrt(np.diag(np.linalg.inv(-OB.hessian(prob.objective, x))))
        np.testing.assert_allclose(wr, lap, rtol=1e-2)
    model.close()


def test_tc_cycle_independent_of_prior_memory_contents():
    """Tensor-core mode with d < dp (d = 21, dp = 32: padding coordinates in every row):
    whole cycles give the same bits whether the arena starts clean or holds NaNs left by
    earlier allocations — nothing reads memory the library has not written."""
    import torch
    prob = I.small_full_mixture(21, 6, 1500, seed=33, box=6.0)
    P = M.Params(n_osc=4, m=6, eps_grad=1e-2, grad_mode=M.GRAD_ADJOINT, seed=6)
    out = []
    for dirty in (False, True):
        if dirty:
            junk = torch.full((256 << 20,), float("nan"), device="cuda")
            del junk
        model = U.open_ctx(prob, P, grad_mode=CH.GRAD_ADJOINT_TC, use_graph=0)
        for _ in range(2):
            model.step()
        out.append([model.get(0, f).copy() for f in (CH.FIELD_X, CH.FIELD_G, CH.FIELD_F)])
        model.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
