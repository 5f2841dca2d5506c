"""The Appendix D benchmark functions on the device against the oracle: value
and adjoint gradient at random points of each App. D domain (ragged tails over
several lanes) and at the stated optima, FD64 gradients, and whole cycles whose
returned points are local maxima of the function.

Tolerances bound the binary32 evaluation: every elementary operation and every
transcendental (a few ulp) errs by at most a small multiple of u = 2^-24 of its
own magnitude, so the error of a sum is ~u times the sum of the magnitudes of
its pieces (M below), plus the effect of the rounded arguments of sin, cos,
exp and sqrt, which the derivative with respect to the argument amplifies."""
import numpy as np
import pytest

import gpu_util as U
from oracle import benchmarks as B
from oracle import method as M
from oracle import modes as MD
from oracle import objectives as OB
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
TINY = 1e-35            # binary32 underflow (sin^20 of a small argument): far below every function's scale
NAMES = ["rastrigin", "ackley", "schwefel", "styblinski_tang", "michalewicz", "trid", "bukin6"]


def _torch_x(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def magnitudes(kind, X):
    """Per-point value magnitude Mf (n,) and per-coordinate gradient magnitude Mg (n, d)."""
    n, d = X.shape
    ax = np.abs(X)
    H = np.stack([np.diag(B.hessian(kind, x)) for x in X]) if kind != B.OBJ_BUKIN6 else np.zeros_like(X)
    g = np.abs(B.grad(kind, X))
    if kind == B.OBJ_RASTRIGIN:
        Mf = (X * X + 20.0).sum(axis=1)
        Mg = 2.0 * ax + 20.0 * np.pi + ax * np.abs(H)
    elif kind == B.OBJ_ACKLEY:
        r = np.sqrt((X * X).mean(axis=1))
        e1 = np.exp(-0.2 * r)
        e2 = np.exp(np.cos(2 * np.pi * X).mean(axis=1))
        Mf = 20.0 * e1 * (1.0 + 0.2 * (d + 4) * r) + e2 * (d + 4) + 40.0
        radial = np.where(r > 0, 4.0 * e1 / (d * np.where(r > 0, r, 1.0)), 0.0)
        Mg = (radial * (2.0 + 0.2 * r) * (d + 4))[:, None] * ax + (2 * np.pi / d) * (e2 * (d + 4))[:, None]
    elif kind == B.OBJ_SCHWEFEL:
        s = np.sqrt(ax)
        Mf = (ax * (1.0 + s)).sum(axis=1) + 419.0 * d
        Mg = 1.0 + s * (1.0 + s) + ax * np.abs(H)
    elif kind == B.OBJ_STYBLINSKI_TANG:
        Mf = (ax ** 4 + 16 * ax ** 2 + 5 * ax).sum(axis=1)
        Mg = 2.0 * ax ** 3 + 16.0 * ax + 2.5 + ax * np.abs(H)
    elif kind == B.OBJ_MICHALEWICZ:
        i = np.arange(1, d + 1)[None, :]
        u = i * X * X / np.pi
        s20, s19 = np.abs(np.sin(u)) ** 20, np.abs(np.sin(u)) ** 19
        Mf = (s20 + 60.0 * s19 * u + ax * s20).sum(axis=1)
        Mg = g + s20 + 40.0 * s19 * i * ax / np.pi * (1.0 + 3.0 * u) + ax * np.abs(H)
    elif kind == B.OBJ_TRID:
        prev = np.concatenate([np.zeros((n, 1)), ax[:, :-1]], axis=1)
        nxt = np.concatenate([ax[:, 1:], np.zeros((n, 1))], axis=1)
        Mf = ((ax + 1.0) ** 2 + ax * prev).sum(axis=1)
        Mg = 2.0 * (ax + 1.0) + prev + nxt
    else:                                                   # Bukin N.6
        x, y = X[:, 0], X[:, 1]
        w = np.abs(y - 0.01 * x * x)
        wm = np.abs(y) + 0.01 * x * x
        on = w == 0.0                                       # on the ridge the sqrt term and its gradient are 0
        ws = np.where(on, 1.0, w)
        Mf = np.where(on, 0.0, 100.0 * np.sqrt(ws) + 50.0 * wm / np.sqrt(ws)) + 0.2
        dw = np.where(on, 0.0, 50.0 / np.sqrt(ws))
        Mg = np.stack([dw * 0.02 * np.abs(x) * (2.0 + wm / ws) + 0.01, dw * (2.0 + wm / ws)], axis=1)
    return Mf, Mg


def _problem(name, d, n, seed):
    return I.benchmark(name, d, n, seed)


def _points(prob, seed):
    """Uniform points of the domain plus the stated optima where App. D gives them."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(prob.lo, prob.hi, (prob.n, prob.d)).astype(np.float32)
    kind, d = prob.objective.kind, prob.d
    special = []
    if kind in (B.OBJ_RASTRIGIN, B.OBJ_ACKLEY):
        special.append(np.zeros(d))
    if kind == B.OBJ_TRID:
        i = np.arange(1, d + 1)
        special.append(i * (d + 1.0 - i))
    if kind == B.OBJ_BUKIN6:
        special.append(np.array([-10.0, 1.0]))
        X = X[np.abs(X[:, 1] - 0.01 * X[:, 0].astype(np.float64) ** 2) > 1e-3]    # off the ridge
    if special:
        X = np.concatenate([X, np.array(special, dtype=np.float32)])
    return X


CASES = [(nm, d) for nm in NAMES if nm != "bukin6" for d in (5, 33, 64)] + [("bukin6", 2)]


@pytest.mark.parametrize("name,d", CASES)
def test_benchmark_value_and_adjoint(name, d):
    prob = _problem(name, d, 301, seed=d)
    model = U.open_ctx(prob, M.Params(grad_mode=M.GRAD_ADJOINT))
    X = _points(prob, seed=d + 1)
    f, g = model.eval(0, _torch_x(X), CH.GRAD_ADJOINT)
    f, g = f.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    X64 = X.astype(np.float64)
    kind = prob.objective.kind
    f_ref, g_ref = B.value(kind, X64), B.grad(kind, X64)
    Mf, Mg = magnitudes(kind, X64)
    tol_f = 32 * U32 * (Mf + np.abs(f_ref)) + TINY
    rows = np.ones(len(X64), bool)
    if kind == B.OBJ_BUKIN6:
        # near the ridge the rounding of w = y - x^2/100 (a few u (|y| + x^2/100)) passes
        # through the square root unlinearised: |sqrt a - sqrt b| <= sqrt|a - b|; the
        # gradient is unbounded there, so it is compared off the ridge only
        x, y = X64[:, 0], X64[:, 1]
        tol_f = tol_f + 100.0 * np.sqrt(8 * U32 * (np.abs(y) + 0.01 * x * x))
        rows = np.abs(y - 0.01 * x * x) > 1e-3
    assert np.all(np.abs(f - f_ref) <= tol_f), (np.abs(f - f_ref) / tol_f).max()
    tol_g = 32 * U32 * (Mg + np.abs(g_ref)) + TINY
    assert np.all(np.abs(g - g_ref)[rows] <= tol_g[rows]), (np.abs(g - g_ref)[rows] / tol_g[rows]).max()
    if kind in (B.OBJ_RASTRIGIN, B.OBJ_ACKLEY):
        np.testing.assert_array_equal(g[-1], np.zeros(d))          # the zero subgradient at the optimum
    model.close()


@pytest.mark.parametrize("name,d", [("rastrigin", 7), ("styblinski_tang", 16), ("michalewicz", 5), ("trid", 9),
                                    ("schwefel", 4), ("ackley", 6)])
def test_benchmark_fd64_gradient(name, d):
    prob = _problem(name, d, 203, seed=40 + d)
    P = M.Params(grad_mode=M.GRAD_FD64, h=1e-5)
    model = U.open_ctx(prob, P)
    X = _points(prob, seed=41 + d)[:200]
    f, g = model.eval(0, _torch_x(X), CH.GRAD_FD64)
    g = g.cpu().numpy().astype(np.float64)
    g_ref = M.fd_gradient(prob, X.astype(np.float64), P)
    err = U.rel_err_rows(g, g_ref, floor=1e-3 * np.abs(g_ref).max())
    assert err.max() <= 1e-6, err.max()
    model.close()


def _local_maxima(prob, fx, tol=1e-3):
    """Each returned point is within tol local sigmas of the local maximum Newton's
    method reaches from it (the Hessian there negative definite)."""
    for x in fx:
        xs, ok = MD.newton_max(prob.objective, x.astype(np.float64))
        H = -OB.hessian(prob.objective, xs)
        assert np.linalg.eigvalsh(H).min() > 0
        assert MD.mahalanobis(x[None].astype(np.float64), xs, H)[0] <= tol


# eps_grad bounds the local-sigma error by ~sqrt(d) eps / sqrt(lambda_min) of -H at the mode:
# Trid's smallest curvature (2 - 2 cos(pi / 9) = 0.12 at d = 8) needs 1e-4 for 1e-3 sigmas
@pytest.mark.parametrize("name,d,n,n_osc,eps,global_x", [
    ("rastrigin", 4, 8192, 4, 1e-3, lambda d: np.zeros(d)),
    ("styblinski_tang", 6, 8192, 3, 1e-3, lambda d: np.full(d, np.sort(np.roots([4.0, 0.0, -32.0, 5.0]).real)[0])),
    ("trid", 8, 2048, 2, 1e-4, lambda d: np.arange(1, d + 1) * (d + 1.0 - np.arange(1, d + 1))),
])
def test_benchmark_cycles_find_the_global_maximum(name, d, n, n_osc, eps, global_x):
    """Whole cycles with exact gradients: every returned point is a local maximum
    and the global maximum App. D states is among them."""
    prob = I.benchmark(name, d, n, seed=7, eps_grad=eps)
    P = M.Params(n_osc=n_osc, m=10, eps_grad=prob.eps_grad, grad_mode=M.GRAD_ADJOINT, seed=11)
    model = U.open_ctx(prob, P)
    for _ in range(n_osc):
        model.step()
    fx, ff = model.modes(0)
    assert fx.shape[0] >= 1
    _local_maxima(prob, fx)
    xg = global_x(d)
    Hg = -OB.hessian(prob.objective, xg)
    assert MD.mahalanobis(fx.astype(np.float64), xg, Hg).min() <= 1e-3
    model.close()
