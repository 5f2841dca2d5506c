"""Pins for the Appendix D benchmark objectives of the oracle (CPU only): the
optima and values App. D states, closed-form special values, and the analytic
gradients and Hessians against differences of the values."""
import numpy as np
import pytest

from oracle import benchmarks as B

SMOOTH = [B.OBJ_RASTRIGIN, B.OBJ_ACKLEY, B.OBJ_SCHWEFEL, B.OBJ_STYBLINSKI_TANG, B.OBJ_MICHALEWICZ, B.OBJ_TRID,
          B.OBJ_BUKIN6]


def _points(kind, d, n, seed):
    lo, hi = B.box(kind, d)
    X = np.random.default_rng(seed).uniform(lo, hi, (n, d))
    if kind == B.OBJ_BUKIN6:                       # stay off the non-differentiable ridge and x = -10
        X = X[np.abs(X[:, 1] - 0.01 * X[:, 0] ** 2) > 0.05]
        X = X[np.abs(X[:, 0] + 10.0) > 0.05]
    return X


def test_rastrigin_and_ackley_global_maximum_at_origin():
    for d in (1, 3, 16):
        z = np.zeros((1, d))
        assert B.value(B.OBJ_RASTRIGIN, z)[0] == 0.0
        np.testing.assert_array_equal(B.grad(B.OBJ_RASTRIGIN, z)[0], np.zeros(d))
        assert abs(B.value(B.OBJ_ACKLEY, z)[0]) < 1e-14
        np.testing.assert_array_equal(B.grad(B.OBJ_ACKLEY, z)[0], np.zeros(d))
    # on the integer lattice cos(2 pi x) = 1: Rastrigin = -|x|^2, Ackley = a (exp(-b rms(x)) - 1)
    X = np.array([[1.0, -2.0, 3.0], [0.0, 0.0, -4.0]])
    np.testing.assert_allclose(B.value(B.OBJ_RASTRIGIN, X), -(X * X).sum(axis=1), atol=1e-12)
    rms = np.sqrt((X * X).mean(axis=1))
    np.testing.assert_allclose(B.value(B.OBJ_ACKLEY, X), 20.0 * (np.exp(-0.2 * rms) - 1.0), atol=1e-12)


def test_styblinski_tang_stationary_points():
    roots = np.sort(np.roots([4.0, 0.0, -32.0, 5.0]).real)      # d/dx (x^4 - 16 x^2 + 5 x) = 0
    lo_root, hi_root = roots[0], roots[2]
    for d in (2, 7):
        for r in (lo_root, hi_root):
            x = np.full((1, d), r)
            np.testing.assert_allclose(B.grad(B.OBJ_STYBLINSKI_TANG, x)[0], 0.0, atol=1e-12)
            assert np.all(np.linalg.eigvalsh(B.hessian(B.OBJ_STYBLINSKI_TANG, x[0])) < 0)
        fg = B.value(B.OBJ_STYBLINSKI_TANG, np.full((1, d), lo_root))[0]
        np.testing.assert_allclose(fg, -0.5 * d * (lo_root ** 4 - 16 * lo_root ** 2 + 5 * lo_root))
        assert fg > B.value(B.OBJ_STYBLINSKI_TANG, np.full((1, d), hi_root))[0]


def test_schwefel_near_the_stated_optimum():
    # App. D: the maximum is near x_i = 420.97, where f is close to 0 (the constant
    # 418.9829 is the per-coordinate maximum of x sin(sqrt|x|))
    s = np.sqrt(420.9687)
    for d in (1, 4):
        x = np.full((1, d), 420.9687)
        assert abs(B.value(B.OBJ_SCHWEFEL, x)[0]) < 1e-4 * d
        np.testing.assert_allclose(B.grad(B.OBJ_SCHWEFEL, x)[0], np.sin(s) + 0.5 * s * np.cos(s))
        assert np.all(np.abs(B.grad(B.OBJ_SCHWEFEL, x)[0]) < 1e-4)


def test_michalewicz_index_and_exponent():
    # coordinate i = 2 at x = pi/2: i x^2 / pi = pi/2, so its term is sin(pi/2) * 1 = 1;
    # coordinate 1 at x = 0 contributes sin(0) = 0
    assert abs(B.value(B.OBJ_MICHALEWICZ, np.array([[0.0, np.pi / 2]]))[0] - 1.0) < 1e-15
    # coordinate 1 at x = pi / sqrt 2: the same inner argument, term sin(pi / sqrt 2)
    x1 = np.pi / np.sqrt(2.0)
    np.testing.assert_allclose(B.value(B.OBJ_MICHALEWICZ, np.array([[x1]]))[0], np.sin(x1), rtol=1e-14)
    # the exponent 2m = 20 halves the term at an inner argument with sin^2 = 2^(-1/10)
    u = np.arcsin(2.0 ** (-1.0 / 20.0))
    x = np.sqrt(u * np.pi)
    np.testing.assert_allclose(B.value(B.OBJ_MICHALEWICZ, np.array([[x]]))[0], 0.5 * np.sin(x), rtol=1e-12)


def test_trid_stated_optimum():
    for d in (2, 6, 64):
        i = np.arange(1, d + 1, dtype=np.float64)
        xs = (i * (d + 1 - i))[None, :]
        np.testing.assert_array_equal(B.grad(B.OBJ_TRID, xs)[0], np.zeros(d))
        np.testing.assert_allclose(B.value(B.OBJ_TRID, xs)[0], d * (d + 4) * (d - 1) / 6.0, rtol=1e-14)
        assert np.all(np.linalg.eigvalsh(B.hessian(B.OBJ_TRID, xs[0])) < 0)


def test_bukin_stated_optimum_and_ridge():
    assert B.value(B.OBJ_BUKIN6, np.array([[-10.0, 1.0]]))[0] == 0.0
    x = np.linspace(-15.0, -5.0, 11)
    np.testing.assert_allclose(B.value(B.OBJ_BUKIN6, np.stack([x, 0.01 * x * x], axis=1)),
                               -0.01 * np.abs(x + 10.0), atol=1e-12)


@pytest.mark.parametrize("kind", SMOOTH)
def test_gradient_against_value_differences(kind):
    d = 2 if kind == B.OBJ_BUKIN6 else 6
    X = _points(kind, d, 40, seed=kind)
    g = B.grad(kind, X)
    scale = np.abs(X).max(axis=1, keepdims=True)
    errs = []
    for h in (1e-3, 5e-4):
        hh = h * np.maximum(scale, 1.0)
        G = np.stack([(B.value(kind, X + hh * e) - B.value(kind, X - hh * e)) / (2 * hh[:, 0]) for e in np.eye(d)],
                     axis=1)
        errs.append(np.abs(G - g).max())
    gs = np.abs(g).max() + 1.0
    # O(h^2) truncation: halving h divides the error by about four, or it is at rounding level
    assert errs[1] < 1e-7 * gs or 3.0 < errs[0] / errs[1] < 5.0, errs


@pytest.mark.parametrize("kind", [B.OBJ_RASTRIGIN, B.OBJ_SCHWEFEL, B.OBJ_STYBLINSKI_TANG, B.OBJ_MICHALEWICZ,
                                  B.OBJ_TRID])
def test_hessian_against_gradient_differences(kind):
    d = 5
    X = _points(kind, d, 6, seed=100 + kind)
    for x in X:
        H = B.hessian(kind, x)
        h = 1e-6 * max(1.0, np.abs(x).max())
        Hn = np.stack([(B.grad(kind, (x + h * e)[None])[0] - B.grad(kind, (x - h * e)[None])[0]) / (2 * h)
                       for e in np.eye(d)], axis=1)
        np.testing.assert_allclose(H, Hn, rtol=1e-5, atol=1e-6 * (np.abs(H).max() + 1.0))
