"""Pins for the oracle's Phases 2-6 (freeze, dedup, reseed, HLC, anti-convergence)."""
import numpy as np
import pytest

from oracle import method as M
from oracle import objectives as OB
from oracle import philox as PX
from paper_2606_26164_gb300 import inputs as I


# --------------------------------------------------------------------- Phase 2 (Eq. 3)

def test_freeze_hand_case():
    f = np.array([0.0, -1.0, -2.5, -2.0, 0.0])
    g = np.array([[1e-7, 0.0], [0.0, -5e-7], [1e-8, 0.0], [2e-6, 0.0], [1e-6, 0.0]])
    stuck, fmax = M.freeze(f, g, 1e-6, 0.1)
    # thr = 0 + log 0.1 = -2.3026: sample 2 fails the quality gate, 3 and 4 the gradient gate
    assert fmax == 0.0
    assert list(stuck) == [True, True, False, False, False]


def test_freeze_binary32_threshold_rounding():
    """The FP32 decision uses thr = fl32(fl32(f_max) + fl32(log delta)); a value
    equal to that rounded threshold sticks, its predecessor does not."""
    f32 = np.array([10.0, 0.0, 0.0], dtype=np.float32)
    thr = np.float32(np.float32(10.0) + np.float32(np.log(0.1)))
    f32[1] = thr
    f32[2] = np.nextafter(thr, np.float32(-np.inf))
    g32 = np.zeros((3, 2), np.float32)
    stuck, _ = M.freeze(f32, g32, 1e-6, 0.1, dtype=np.float32)
    assert list(stuck) == [True, True, False]


def test_freeze_excludes_nonfinite_from_fmax():
    f = np.array([np.nan, -1.0, -1.5])
    stuck, fmax = M.freeze(f, np.zeros((3, 1)), 1.0, 0.1)
    assert fmax == -1.0 and list(stuck) == [False, True, True]


# --------------------------------------------------------------------- Phase 3 (Eq. 4)

def test_dedup_chain_literal_reading():
    """A ~ B and B ~ C but A !~ C, f_A > f_B > f_C: B is removed by A and C by B
    (B counts although it is itself removed)."""
    x = np.array([[0.0], [0.0008], [0.0016], [5.0]])
    f = np.array([3.0, 2.0, 1.0, 0.0])
    stuck = np.array([True, True, True, False])
    rem = M.dedup(x, f, stuck, 1e-3)
    assert list(rem) == [False, True, True, False]


def test_dedup_ties_keep_lower_index_and_ignore_unstuck():
    x = np.array([[1.0, 1.0], [1.0, 1.0005], [1.0, 1.0], [1.0, 1.0]])
    f = np.array([2.0, 2.0, 5.0, 2.0])
    stuck = np.array([True, True, False, True])
    rem = M.dedup(x, f, stuck, 1e-3)
    assert list(rem) == [False, True, False, True]


def test_dedup_strict_distance():
    x = np.array([[0.0], [0.5]])                        # |dx| = eps exactly: not a duplicate
    rem = M.dedup(x, np.array([1.0, 0.0]), np.array([True, True]), 0.5)
    assert not rem.any()


def test_dedup_invariants_random():
    rng = np.random.default_rng(3)
    x = np.round(rng.uniform(0, 0.02, size=(300, 2)), 4)
    f = np.round(rng.uniform(0, 1, size=300), 2)
    stuck = rng.random(300) < 0.8
    rem = M.dedup(x, f, stuck, 1e-3)
    surv = np.flatnonzero(stuck & ~rem)
    # survivors are pairwise at L-inf distance >= eps
    D = np.abs(x[surv][:, None] - x[surv][None]).max(axis=2)
    assert (D[~np.eye(surv.size, dtype=bool)] >= 1e-3).all()
    # every removed sample has a higher-ranked stuck neighbour within eps
    st_idx = np.flatnonzero(stuck)
    for j in np.flatnonzero(rem):
        d = np.abs(x[st_idx] - x[j]).max(axis=1)
        above = (f[st_idx] > f[j]) | ((f[st_idx] == f[j]) & (st_idx < j))
        assert ((d < 1e-3) & above).any()
    assert not rem[~stuck].any()


# --------------------------------------------------------------------- Phase 4 (Sec. 3.2.4)

@pytest.mark.parametrize("d", [2, 5, 16, 64])
def test_householder_qr_matches_library(d):
    G = np.random.default_rng(d).standard_normal((d, d))
    Q, R = M.householder_qr(G)
    q, r = np.linalg.qr(G)
    sgn = np.sign(np.diag(r))
    np.testing.assert_allclose(Q, q * sgn[None, :], atol=1e-12)
    np.testing.assert_allclose(Q @ R, G, atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(d), atol=1e-12)
    assert (np.diag(R) > 0).all() and np.allclose(np.tril(R, -1), 0.0, atol=1e-12)


def test_ray_exit_hand_cases():
    lo, hi = np.array([-1.0, -1.0]), np.array([1.0, 1.0])
    p = np.array([[0.0, 0.0], [0.5, 0.0], [1.0, 0.0]])
    u = np.array([[1.0, 0.0], [np.sqrt(0.5), -np.sqrt(0.5)], [1.0, 0.0]])
    np.testing.assert_allclose(M.ray_exit(p, u, lo, hi), [1.0, 0.5 / np.sqrt(0.5), 0.0])


def _reseed_setup(n_unfrozen, d=3, N=40):
    p = I.small_mixture(d, 3, N, seed=9)
    st = M.new_state(p.x0, 4)
    st.f = -np.arange(N, dtype=np.float64)
    st.stuck[:] = True
    st.stuck[N - n_unfrozen:] = False
    st.removed[:] = False
    st.removed[1:10] = True                             # 9 free slots, removed from the stuck set
    st.stuck &= ~st.removed
    st.hlen[:] = 3
    return p, st


def test_repulse_monkey_children_on_parent_rays():
    p, st = _reseed_setup(n_unfrozen=12)
    x_before = st.x.copy()
    P = M.Params(seed=11)
    M.reseed(p, st, P, cycle=2)
    assert st.last_reseed == M.RESEED_RM
    free = np.arange(1, 10)
    unfrozen = np.flatnonzero(~st.stuck)
    unfrozen = unfrozen[~np.isin(unfrozen, free)]
    w = PX.words(11, np.arange(9), 0, PX.TAG_RM, 2, 0, 0, 0)
    pick = ((w[:, 0].astype(np.uint64) * np.uint64(unfrozen.size)) >> np.uint64(32)).astype(int)
    parents = x_before[unfrozen[pick]]
    z = PX.normal_rows(11, np.arange(9), 3, PX.TAG_RM_DIR, 2, 0, 0, 0)
    u = z / np.linalg.norm(z, axis=1, keepdims=True)
    delta = st.x[free] - parents
    t = np.einsum("nd,nd->n", delta, u)
    np.testing.assert_allclose(delta, t[:, None] * u, atol=1e-12)            # on the ray
    assert (t >= 0).all() and (t <= M.ray_exit(parents, u, p.lo, p.hi) + 1e-12).all()
    assert (st.x >= p.lo).all() and (st.x <= p.hi).all()
    assert not st.stuck[free].any() and (st.hlen[free] == 0).all()


def test_golden_rooster_orthonormal_rays_round_robin():
    p, st = _reseed_setup(n_unfrozen=2, d=4)
    x_before = st.x.copy()
    P = M.Params(seed=5)
    M.reseed(p, st, P, cycle=1)
    assert st.last_reseed == M.RESEED_GR
    surv = np.flatnonzero(st.stuck)
    ranked = surv[np.lexsort((surv, -st.f[surv]))]
    Gm = PX.normal_rows(5, np.arange(4), 4, PX.TAG_GR_MAT, 1, 0, 0, 0)
    Q, _ = M.householder_qr(Gm)
    S = ranked.size
    for r, slot in enumerate(range(1, 10)):
        peak = x_before[ranked[r % S]]
        u = Q[:, (r // S) % 4] * (1.0 if (r // (S * 4)) % 2 == 0 else -1.0)
        delta = st.x[slot] - peak
        t = delta @ u
        np.testing.assert_allclose(delta, t * u, atol=1e-12)
        assert t >= -1e-15


def test_golden_rooster_disables_after_patience():
    P = M.Params(seed=1, gr_patience=2)
    modes = []
    st = None
    for gen in range(4):
        p, st2 = _reseed_setup(n_unfrozen=2, d=2)
        if st is not None:
            st2.gr_enabled, st2.gr_noprog, st2.gr_prev_surv = st.gr_enabled, st.gr_noprog, st.gr_prev_surv
        M.reseed(p, st2, P, cycle=gen + 1)
        modes.append(st2.last_reseed)
        st = st2
    # same survivor count every generation: GR, GR (1 no-progress), then disabled -> uniform
    assert modes == [M.RESEED_GR, M.RESEED_GR, M.RESEED_UNIFORM, M.RESEED_UNIFORM]
    assert not st.gr_enabled


def test_uniform_redraw_inside_box():
    p, st = _reseed_setup(n_unfrozen=2, d=3)
    st.gr_enabled = False
    M.reseed(p, st, M.Params(seed=2), cycle=1)
    assert st.last_reseed == M.RESEED_UNIFORM
    u = PX.uniform_rows(2, np.arange(9), 3, PX.TAG_UNIFORM, 1, 0, 0, 0)
    np.testing.assert_allclose(st.x[1:10], p.lo + u * (p.hi - p.lo), atol=1e-12)


# --------------------------------------------------------------------- Phases 5-6

def _quad_state(N=64, d=3, seed=3):
    p = I.small_quadratic(d, N, seed=seed, cond=4.0)
    p.lo, p.hi = np.full(d, -100.0), np.full(d, 100.0)
    st = M.new_state(p.x0, 4)
    return p, st


def test_population_scales_hand_case():
    obj = I.Objective(3, 2, {"center": np.zeros(2), "Q": np.eye(2), "lam": np.array([1.0, 1.0])})
    p = I.Problem(2, 3, np.full(2, -9.0), np.full(2, 9.0), obj, np.zeros((3, 2), np.float32), 1e-6, 1.0)
    st = M.new_state(np.array([[1.0, 0.0], [3.0, 2.0], [8.0, 8.0]]), 2)
    unf = np.array([True, True, False])
    P = M.Params(grad_mode=M.GRAD_ADJOINT)
    idx, G, sigma, alpha, s, g_rms = M.population_scales(p, st, P, unf)
    # var_x = 1, var_y = 1 -> s = 1; grad = -2x: (-2,0), (-6,-4) -> g_rms = sqrt(56/4)
    assert s == pytest.approx(1.0) and sigma == pytest.approx(0.1)
    assert g_rms == pytest.approx(np.sqrt(14.0))
    assert alpha == pytest.approx(0.1 / np.sqrt(14.0))


def test_hlc_step_algebra_and_unbiasedness():
    """Appendix B: for a quadratic, grad f(theta + sigma z) = grad f(theta) + sigma H z,
    so one HLC step is x + alpha (grad f(x) + sigma H zbar) with zbar the mean of
    the M perturbations, and sqrt(M) zbar ~ N(0, I) (chi-square check)."""
    p, st = _quad_state(N=400, d=3)
    P = M.Params(n_cloud=1, M=8, grad_mode=M.GRAD_ADJOINT, seed=4)
    x0 = st.x.copy()
    sigma, alpha = M.hlc(p, st, P, cycle=1)
    H = -2.0 * p.objective.arrays["Q"].T @ np.diag(p.objective.arrays["lam"]) @ p.objective.arrays["Q"]
    g0 = -2.0 * (x0 - p.objective.arrays["center"]) @ (p.objective.arrays["Q"].T @ np.diag(p.objective.arrays["lam"]) @ p.objective.arrays["Q"])
    zbar = np.mean([PX.normal_rows(4, np.arange(400), 3, PX.TAG_HLC, 1, 0, 0, k) for k in range(8)], axis=0)
    np.testing.assert_allclose(st.x, x0 + alpha * (g0 + sigma * zbar @ H.T), rtol=1e-10, atol=1e-10)
    chi2 = float((8.0 * zbar * zbar).sum())
    dof = zbar.size
    assert abs(chi2 - dof) < 5 * np.sqrt(2 * dof)


def test_hlc_value_only_estimator_algebra_and_unbiasedness():
    """The value-only smoothing variant on a quadratic f = -r^T A r (r = x - c):
    f(x + sigma z) - f(x) = -2 sigma z^T A r - sigma^2 z^T A z, so one step adds
    alpha (1/M) sum_k (-2 z_k^T A r - sigma z_k^T A z_k) z_k; and the estimator
    (f(x + sigma z) - f(x)) z / sigma has the gradient as its mean over z."""
    p, st = _quad_state(N=400, d=3)
    P = M.Params(n_cloud=1, M=8, grad_mode=M.GRAD_ADJOINT, seed=4, hlc_value_only=1)
    x0 = st.x.copy()
    sigma, alpha = M.hlc(p, st, P, cycle=1)
    A = p.objective.arrays["Q"].T @ np.diag(p.objective.arrays["lam"]) @ p.objective.arrays["Q"]
    r = x0 - p.objective.arrays["center"]
    acc = np.zeros_like(x0)
    for k in range(8):
        z = PX.normal_rows(4, np.arange(400), 3, PX.TAG_HLC, 1, 0, 0, k)
        w = -2.0 * np.einsum("ni,ij,nj->n", z, A, r) - sigma * np.einsum("ni,ij,nj->n", z, A, z)
        acc += w[:, None] * z
    np.testing.assert_allclose(st.x, np.clip(x0 + alpha * acc / 8, p.lo, p.hi), rtol=1e-9, atol=1e-9)
    # mean of the estimator at one point over many independent draws = grad f
    rng = np.random.default_rng(9)
    x = x0[:1]
    Z = rng.normal(size=(200000, 3))
    est = ((OB.value(p.objective, x + 0.3 * Z) - OB.value(p.objective, x)) / 0.3)[:, None] * Z
    g = OB.grad(p.objective, x)[0]
    se = est.std(axis=0) / np.sqrt(len(Z))
    assert np.all(np.abs(est.mean(axis=0) - g) < 5 * se)


def test_anti_convergence_momentum_algebra():
    """Eq. 6 with a linear f (constant gradient g): v1 = -a g, v2 = -a g (1 + mu)."""
    obj = I.Objective(3, 1, {"center": np.array([0.0]), "Q": np.eye(1), "lam": np.array([1e-12])})
    p = I.Problem(1, 6, np.array([-1e6]), np.array([1e6]), obj, np.zeros((6, 1), np.float32), 1e-6, 1.0)
    # f = -1e-12 x^2 is locally linear: use the analytic gradient and a fixed alpha
    st = M.new_state(np.linspace(1000.0, 1005.0, 6)[:, None], 2)
    P = M.Params(n_anti=2, mu=0.9, alpha=3.0, grad_mode=M.GRAD_ADJOINT)
    x0 = st.x.copy()
    g = -2e-12 * x0
    M.anti_converge(p, st, P)
    g1 = -2e-12 * (x0 - 3.0 * g)
    np.testing.assert_allclose(st.x, x0 - 3.0 * g + (0.9 * (-3.0 * g) - 3.0 * g1), rtol=1e-14)


def test_anti_convergence_zeroes_velocity_on_clamped_coordinates():
    obj = I.Objective(3, 2, {"center": np.array([0.0, 0.0]), "Q": np.eye(2), "lam": np.array([1.0, 1.0])})
    p = I.Problem(2, 1, np.array([-1.0, -1.0]), np.array([1.0, 1.0]), obj, np.zeros((1, 2), np.float32), 1e-6, 1.0)
    st = M.new_state(np.array([[0.9, 0.1]]), 2)
    P = M.Params(n_anti=2, mu=0.5, alpha=1.0, grad_mode=M.GRAD_ADJOINT)
    M.anti_converge(p, st, P)
    # step 1: g = (-1.8, -0.2), v = (1.8, 0.2), x = (2.7 -> 1.0 clamped, 0.3), v_x := 0
    # step 2: g = (-2, -0.6), v = (0 + 2, 0.1 + 0.6), x = (1.0 clamped, 1.0)
    np.testing.assert_allclose(st.x, [[1.0, 1.0]], atol=1e-12)


def test_carry_tiger_rays():
    """Carry Tiger (reading of Sec. 5.1): every sample on the segment from the box
    centre to a face centre, an edge midpoint or a vertex, classes cycling with the
    index; face centres round-robin; positions along the ray uniform in (0, 1)."""
    from oracle import seeding as SD
    d, n = 5, 6000
    lo, hi = np.full(d, -3.0), np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    X = SD.carry_tiger(lo, hi, n, seed=11)
    E, t = SD.carry_tiger_directions(d, n, seed=11)
    c, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    assert np.all((X >= lo) & (X <= hi))
    R = (X - c) / half                                  # = t e on every coordinate
    nz = (E != 0).sum(axis=1)
    cls = np.arange(n) % 3
    assert np.all(nz[cls == 0] == 1) and np.all(nz[cls == 1] == d - 1) and np.all(nz[cls == 2] == d)
    np.testing.assert_allclose(np.abs(R).max(axis=1), t, rtol=1e-12)
    np.testing.assert_allclose(R, t[:, None] * E, atol=1e-12)
    faces = [tuple(e) for e in E[cls == 0][:2 * d]]
    assert len(set(faces)) == 2 * d                      # the first 2d face samples cover every face
    from scipy import stats
    assert stats.kstest(t, "uniform").pvalue > 1e-4
    # vertex signs: each coordinate +-1 about equally often
    assert abs(E[cls == 2].mean()) < 4 / np.sqrt(E[cls == 2].size)


def test_uniform_seed_in_box():
    from oracle import seeding as SD
    lo, hi = np.array([-1.0, 0.0, 5.0]), np.array([1.0, 10.0, 6.0])
    X = SD.uniform(lo, hi, 4000, seed=3)
    assert np.all((X > lo) & (X < hi))
    from scipy import stats
    for a in range(3):
        assert stats.kstest((X[:, a] - lo[a]) / (hi[a] - lo[a]), "uniform").pvalue > 1e-4


def _exit_distance(p, u, lo, hi):
    """Distance from p along the unit direction u to the box boundary (independent of
    the oracle's helper): the smallest positive step that reaches a face."""
    with np.errstate(divide="ignore"):
        up = np.where(u > 0, (hi - p) / u, np.inf)
        dn = np.where(u < 0, (lo - p) / u, np.inf)
    return np.minimum(up, dn).min(axis=-1)


@pytest.mark.parametrize("n_unfrozen,mode", [(60, "rm"), (2, "gr")])
def test_reseed_children_uniform_along_their_rays(n_unfrozen, mode):
    """Sec. 3.2.4 places each child uniformly along its ray inside Theta: the child's
    distance from its parent (RM) or peak (GR) divided by the ray's exit distance is
    uniform on [0, 1] (Kolmogorov-Smirnov over 1500 children)."""
    from scipy import stats
    d, N, nfree = 3, 1600, 1500
    p = I.small_mixture(d, 3, N, seed=19)
    st = M.new_state(p.x0, 4)
    st.f = -np.arange(N, dtype=np.float64)
    st.stuck[:] = True
    st.stuck[N - n_unfrozen:] = False
    st.removed[:] = False
    st.removed[1:1 + nfree] = True
    st.stuck &= ~st.removed
    x_before = st.x.copy()
    P = M.Params(seed=23)
    M.reseed(p, st, P, cycle=1)
    assert st.last_reseed == (M.RESEED_RM if mode == "rm" else M.RESEED_GR)
    free = np.arange(1, 1 + nfree)
    if mode == "rm":
        unfrozen = np.flatnonzero(~st.stuck)
        unfrozen = unfrozen[~np.isin(unfrozen, free)]
        w = PX.words(23, np.arange(nfree), 0, PX.TAG_RM, 1, 0, 0, 0)
        pick = ((w[:, 0].astype(np.uint64) * np.uint64(unfrozen.size)) >> np.uint64(32)).astype(int)
        parents = x_before[unfrozen[pick]]
    else:
        surv = np.flatnonzero(st.stuck)
        ranked = surv[np.lexsort((surv, -st.f[surv]))]
        parents = x_before[ranked[np.arange(nfree) % ranked.size]]
    delta = st.x[free] - parents
    t = np.linalg.norm(delta, axis=1)
    keep = t > 0
    u = delta[keep] / t[keep, None]
    ratio = t[keep] / _exit_distance(parents[keep], u, p.lo, p.hi)
    assert keep.sum() > 0.99 * nfree and (ratio <= 1 + 1e-12).all()
    assert stats.kstest(ratio, "uniform").pvalue > 1e-3


# --------------------------------------------------------------------- boundaries of the readings

@pytest.mark.parametrize("n_unfrozen,mode", [(5, M.RESEED_RM), (4, M.RESEED_GR)])
def test_repulse_monkey_needs_at_least_five_unfrozen(n_unfrozen, mode):
    """Sec. 3.2.4 reading: Repulse Monkey when 5 or more samples are unfrozen,
    Golden Rooster below that -- the boundary case itself."""
    p, st = _reseed_setup(n_unfrozen=n_unfrozen)
    M.reseed(p, st, M.Params(seed=3), cycle=1)
    assert st.last_reseed == mode


def test_golden_rooster_sign_alternates_after_every_peak_and_axis():
    """With S survivors in d dimensions, slots r and r + S d use the same peak and
    the same column of Q with opposite signs: their children leave the peak in
    opposite directions along one line (S = 3, d = 2, 9 free slots)."""
    p, st = _reseed_setup(n_unfrozen=2, d=2, N=14)
    x_before = st.x.copy()
    surv = np.flatnonzero(st.stuck)
    S, d = surv.size, 2
    assert S * d < 9
    M.reseed(p, st, M.Params(seed=8), cycle=1)
    assert st.last_reseed == M.RESEED_GR
    ranked = surv[np.lexsort((surv, -st.f[surv]))]
    for r in range(9 - S * d):
        peak = x_before[ranked[r % S]]
        a = st.x[1 + r] - peak
        b = st.x[1 + r + S * d] - peak
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos == pytest.approx(-1.0, abs=1e-12), (r, cos)


def test_hlc_draws_fresh_perturbations_every_step():
    """Eq. 5 averages over new perturbations at every step.  On a quadratic each
    step is x + alpha (grad f(x) + sigma H zbar_t) (Appendix B), so the random
    parts alpha sigma H zbar_t of two consecutive steps are uncorrelated across
    samples when the draws are fresh (and identical when they are reused)."""
    N, d = 2000, 3
    p, st = _quad_state(N=N, d=d)
    A = p.objective.arrays["Q"].T @ np.diag(p.objective.arrays["lam"]) @ p.objective.arrays["Q"]
    c = p.objective.arrays["center"]

    def grad(x):
        return -2.0 * (x - c) @ A

    one = M.State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.__dict__.items()})
    x0 = st.x.copy()
    s1, a1 = M.hlc(p, one, M.Params(n_cloud=1, M=8, grad_mode=M.GRAD_ADJOINT, seed=4), cycle=1)
    s2, a2 = M.hlc(p, st, M.Params(n_cloud=2, M=8, grad_mode=M.GRAD_ADJOINT, seed=4), cycle=1)
    assert (s1, a1) == (s2, a2)
    x1, x2 = one.x, st.x
    r1 = (x1 - x0 - a1 * grad(x0)).ravel()
    r2 = (x2 - x1 - a2 * grad(x1)).ravel()
    assert np.abs(r1).max() > 0 and np.abs(r2).max() > 0
    corr = np.corrcoef(r1, r2)[0, 1]
    assert abs(corr) < 0.1, corr


def test_anti_convergence_velocity_zeroed_where_the_box_stopped_it():
    """Eq. 6 with the box: the velocity of a clamped coordinate is zeroed, so when
    the gradient there reverses the next step starts from rest.  1-D mixture of unit
    components at 5 and 14 (outside the box [-10, 10]), alpha = 2, mu = 0.9, from
    x = 7: step 1 overshoots past 10 and is clamped; at 10 the outside component
    dominates, and step 2 is -alpha f'(10) with no momentum term."""
    w = np.array([0.5, 0.5])
    mu_k = np.array([5.0, 14.0])
    obj = I.Objective(1, 1, {"weights": w, "means": mu_k[:, None], "sigmas": np.ones((2, 1))})
    p = I.Problem(1, 1, np.array([-10.0]), np.array([10.0]), obj, np.zeros((1, 1), np.float32), 1e-6, 1.0)
    st = M.new_state(np.array([[7.0]]), 2)
    M.anti_converge(p, st, M.Params(n_anti=2, mu=0.9, alpha=2.0, grad_mode=M.GRAD_ADJOINT))
    # f'(x) = sum_k r_k (mu_k - x), r the responsibilities (equal weights and widths)
    lc = -0.5 * (10.0 - mu_k) ** 2
    r = np.exp(lc - lc.max())
    r /= r.sum()
    fp10 = float(r @ (mu_k - 10.0))
    lc7 = -0.5 * (7.0 - mu_k) ** 2
    r7 = np.exp(lc7 - lc7.max())
    r7 /= r7.sum()
    assert 7.0 - 2.0 * float(r7 @ (mu_k - 7.0)) > 10.0      # step 1 leaves the box
    np.testing.assert_allclose(st.x[0, 0], 10.0 - 2.0 * fp10, rtol=1e-12)


def test_carry_tiger_enumeration_hand_case_d2():
    """The anchor enumeration of the Carry Tiger reading, by hand for d = 2: sample i
    has class i mod 3 and counter j = i div 3; face slots take face q = j mod 2d, axis
    q div 2, sign - for even q and + for odd q; edge slots leave axis j mod d free."""
    from oracle import seeding as SD
    E, _ = SD.carry_tiger_directions(2, 12, seed=5)
    faces = E[0::3]
    np.testing.assert_array_equal(faces, [[-1, 0], [1, 0], [0, -1], [0, 1]])
    edges = E[1::3]
    free = [0, 1, 0, 1]
    for e, a in zip(edges, free):
        assert e[a] == 0 and abs(e[1 - a]) == 1
    assert np.all(np.abs(E[2::3]) == 1)
