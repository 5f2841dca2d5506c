"""Pins for the oracle's Philox streams and objective families (CPU only)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import objectives as OB
from oracle import philox as PX
from paper_2606_26164_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt")) if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(t, 16) for t in r]
        out = PX.philox4x32_10(np.array(v[0:4]), np.array(v[4:6]))
        assert [int(o) for o in out] == v[6:10]


def test_uniform_endpoints_exact():
    u = PX.u01(np.array([0, 511, 512, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24
    assert u[2] == 3 * 2.0 ** -24
    assert u[3] == 1.0 - 2.0 ** -24
    # every value is exactly representable in binary32
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_normals_are_standard_gaussian():
    z = PX.normal_rows(7, np.arange(20000), 8, PX.TAG_HLC, 3, 1, 0, 5).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_stream_counters_separate():
    a = PX.words(1, np.arange(4), 0, PX.TAG_RM, 2, 0, 0, 0)
    b = PX.words(1, np.arange(4), 0, PX.TAG_RM, 3, 0, 0, 0)
    c = PX.words(1, np.arange(4), 0, PX.TAG_GR_T, 2, 0, 0, 0)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def _scipy_mixture_logpdf(obj, X):
    A = obj.arrays
    comps = []
    for k in range(A["weights"].shape[0]):
        if obj.kind == OB.OBJ_MIXTURE_DIAG:
            cov = np.diag(A["sigmas"][k] ** 2)
        else:
            cov = A["chol"][k] @ A["chol"][k].T
        comps.append(np.log(A["weights"][k]) + stats.multivariate_normal(A["means"][k], cov).logpdf(X))
    return np.logaddexp.reduce(np.stack(comps, axis=1), axis=1)


@pytest.mark.parametrize("kind", ["diag", "full"])
def test_mixture_value_matches_scipy(kind):
    p = I.small_mixture(5, 6, 40, seed=1) if kind == "diag" else I.small_full_mixture(5, 6, 40, seed=1)
    X = p.x0.astype(np.float64)
    np.testing.assert_allclose(OB.value(p.objective, X), _scipy_mixture_logpdf(p.objective, X), rtol=1e-12, atol=1e-10)


def test_quadratic_closed_form():
    p = I.small_quadratic(6, 10, seed=2)
    A = p.objective.arrays
    c = A["center"]
    assert OB.value(p.objective, c[None])[0] == 0.0
    np.testing.assert_array_equal(OB.grad(p.objective, c[None])[0], np.zeros(6))
    # with Q = I the form is -sum lam_i (x_i - c_i)^2
    obj = I.Objective(OB.OBJ_QUADRATIC, 3, {"center": np.array([1.0, -2.0, 0.5]), "Q": np.eye(3), "lam": np.array([1.0, 10.0, 100.0])})
    x = np.array([[2.0, -1.0, 0.0]])
    assert OB.value(obj, x)[0] == pytest.approx(-(1.0 + 10.0 + 100.0 * 0.25))
    np.testing.assert_allclose(OB.grad(obj, x)[0], [-2.0, -20.0, 100.0])


@pytest.mark.parametrize("maker", [lambda: I.small_mixture(4, 5, 12, seed=3),
                                   lambda: I.small_full_mixture(4, 5, 12, seed=3),
                                   lambda: I.small_quadratic(4, 12, seed=3)])
def test_analytic_gradient_and_fd_order(maker):
    """Central differences converge to the analytic gradient at O(h^2):
    halving h divides the truncation error by about four (Richardson)."""
    from oracle import method as M
    p = maker()
    X = p.x0.astype(np.float64) * 0.5
    g = OB.grad(p.objective, X)
    errs = []
    for h in (1e-2, 5e-3):
        P = M.Params(h=h, grad_mode=M.GRAD_FD64)
        errs.append(np.abs(M.fd_gradient(p, X, P) - g).max())
    scale = np.abs(g).max()
    if p.objective.kind == OB.OBJ_QUADRATIC:
        assert errs[0] < 1e-9 * scale                # exact for a quadratic up to rounding
    else:
        assert 3.0 < errs[0] / errs[1] < 5.0
    P = M.Params(h=1e-5, grad_mode=M.GRAD_FD64)
    np.testing.assert_allclose(M.fd_gradient(p, X, P), g, rtol=1e-6, atol=1e-7 * scale)


@pytest.mark.parametrize("maker", [lambda: I.small_mixture(3, 4, 4, seed=4),
                                   lambda: I.small_full_mixture(3, 4, 4, seed=4)])
def test_hessian_matches_gradient_differences(maker):
    p = maker()
    x = p.x0[0].astype(np.float64) * 0.3
    H = OB.hessian(p.objective, x)
    h = 1e-6
    Hn = np.stack([(OB.grad(p.objective, (x + h * e)[None])[0] - OB.grad(p.objective, (x - h * e)[None])[0]) / (2 * h)
                   for e in np.eye(3)], axis=1)
    np.testing.assert_allclose(H, Hn, rtol=1e-5, atol=1e-7 * np.abs(H).max())
    np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())


def test_point_noise_draws():
    """Sec. 5.6 noise: one N(0,1) draw per evaluation point, repeatable for the
    same point, independent across the FD stencil's neighbouring points."""
    rng = np.random.default_rng(3)
    X = rng.uniform(-5, 5, (20000, 3))
    z = PX.point_noise(0, 0, X)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    np.testing.assert_array_equal(z, PX.point_noise(0, 0, X.copy()))
    Xp = X.copy()
    Xp[:, 1] = np.nextafter(X[:, 1].astype(np.float32), np.float32(np.inf)).astype(np.float64)
    zp = PX.point_noise(0, 0, Xp)
    assert abs(np.corrcoef(z, zp)[0, 1]) < 0.05
    assert abs(np.corrcoef(z, PX.point_noise(1, 0, X))[0, 1]) < 0.05


def test_bf16_rounding_and_split():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    a = np.concatenate([rng.normal(0, 10, 5000), [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(OB.bf16_round(a), ref)
    assert OB.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0            # tie goes to even
    x = rng.uniform(-20, 20, 5000).astype(np.float32).astype(np.float64)
    assert np.all(np.abs(OB.bf16_split(x) - x) <= 2.0 ** -17 * np.abs(x))


def test_precision_factor_mixture_matches_cholesky_form():
    p = I.small_full_mixture(5, 4, 30, seed=12)
    A = p.objective.arrays
    W = np.stack([np.linalg.inv(L) for L in A["chol"]])
    pobj = I.Objective(OB.OBJ_MIXTURE_PREC, 5, {"weights": A["weights"], "means": A["means"], "linv": W})
    X = p.x0.astype(np.float64)
    np.testing.assert_allclose(OB.value(pobj, X), OB.value(p.objective, X), rtol=1e-12)
    np.testing.assert_allclose(OB.grad(pobj, X), OB.grad(p.objective, X), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(OB.hessian(pobj, X[0]), OB.hessian(p.objective, X[0]), rtol=1e-9, atol=1e-12)
    # the rounded factors keep every component's peak at its centre
    tco = OB.tensor_core_objective(p.objective, split=False)
    np.testing.assert_allclose(OB.grad(tco, A["means"][:1]), OB.grad(p.objective, A["means"][:1]), atol=1e-6)


def test_noisy_evaluation_adds_scaled_draw():
    from oracle import method as M
    p = I.small_mixture(3, 2, 50, seed=4, noise_sigma=0.5)
    X = p.x0.astype(np.float64)
    f = M.evaluate(p, X, seed=9)
    np.testing.assert_allclose(f - OB.value(p.objective, X), 0.5 * PX.point_noise(9, 0, X), rtol=1e-9, atol=1e-9)


def test_normals_of_one_block_are_independent():
    """The four normals of one Philox block come from two Box-Muller pairs on
    disjoint words, so the angle of (z0, z1) carries no information about the
    radius of (z2, z3) (and vice versa): rank correlations near zero.  A generator
    that reused a word across the pairs would make them functions of each other."""
    from scipy import stats
    z = PX.normal_rows(21, np.arange(20000), 4, PX.TAG_HLC, 1, 0, 0, 0)
    ang01 = np.mod(np.arctan2(z[:, 1], z[:, 0]), 2 * np.pi)
    ang23 = np.mod(np.arctan2(z[:, 3], z[:, 2]), 2 * np.pi)
    rad01 = z[:, 0] ** 2 + z[:, 1] ** 2
    rad23 = z[:, 2] ** 2 + z[:, 3] ** 2
    for a, b in ((ang01, rad23), (ang23, rad01), (ang01, ang23), (rad01, rad23)):
        assert abs(stats.spearmanr(a, b)[0]) < 0.05
