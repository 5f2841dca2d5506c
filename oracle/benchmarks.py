"""Benchmark objectives of Appendix D in FP64 (oracle side; test infrastructure).

Each function is the negated (maximisation) form of App. D, vectorised over the
rows of X (n, d); coordinates are indexed i = 1..d in the formulas below.

* Rastrigin:  f = -sum_i (x_i^2 - A cos(2 pi x_i) + A),  A = 10
* Ackley:     f = a exp(-b sqrt(S / d)) + exp(C / d) - a - e,
              S = sum x_i^2, C = sum cos(c x_i), a = 20, b = 0.2, c = 2 pi
* Schwefel:   f = sum_i x_i sin(sqrt|x_i|) - 418.9829 d
* Styblinski-Tang: f = -(1/2) sum_i (x_i^4 - 16 x_i^2 + 5 x_i)
* Michalewicz: f = sum_i sin(x_i) sin(i x_i^2 / pi)^(2m),  m = 10
* Trid:       f = -sum_i (x_i - 1)^2 + sum_{i>=2} x_i x_{i-1}
* Bukin N.6:  f = -100 sqrt|y - x^2 / 100| - |x + 10| / 100   (d = 2, (x, y))

Gradients are the analytic ones.  Where a function is not differentiable the
gradient takes the value of the zero subgradient term: Ackley's first term at
x = 0 (its radial derivative has no limit there), Bukin's ridge term where
y = x^2 / 100 and its |x + 10| term at x = -10.  The Hessian is analytic for the
separable functions and Trid, and the symmetrised central difference of the
analytic gradient for Ackley and Bukin N.6 (mode checks only).
"""
from __future__ import annotations

import numpy as np

OBJ_RASTRIGIN = 10
OBJ_ACKLEY = 11
OBJ_SCHWEFEL = 12
OBJ_STYBLINSKI_TANG = 13
OBJ_MICHALEWICZ = 14
OBJ_TRID = 15
OBJ_BUKIN6 = 16
BENCH_KINDS = (OBJ_RASTRIGIN, OBJ_ACKLEY, OBJ_SCHWEFEL, OBJ_STYBLINSKI_TANG, OBJ_MICHALEWICZ, OBJ_TRID,
               OBJ_BUKIN6)

RASTRIGIN_A = 10.0
ACKLEY_A, ACKLEY_B, ACKLEY_C = 20.0, 0.2, 2.0 * np.pi
SCHWEFEL_C = 418.9829
MICHALEWICZ_M = 10


def box(kind, d):
    """The App. D domain Theta (lo, hi)."""
    if kind == OBJ_RASTRIGIN:
        return np.full(d, -5.12), np.full(d, 5.12)
    if kind == OBJ_ACKLEY:
        return np.full(d, -32.768), np.full(d, 32.768)
    if kind == OBJ_SCHWEFEL:
        return np.full(d, -500.0), np.full(d, 500.0)
    if kind == OBJ_STYBLINSKI_TANG:
        return np.full(d, -5.0), np.full(d, 5.0)
    if kind == OBJ_MICHALEWICZ:
        return np.zeros(d), np.full(d, np.pi)
    if kind == OBJ_TRID:
        return np.full(d, -float(d * d)), np.full(d, float(d * d))
    if kind == OBJ_BUKIN6:
        assert d == 2
        return np.array([-15.0, -3.0]), np.array([-5.0, 3.0])
    raise ValueError(kind)


def _idx(d):
    return np.arange(1, d + 1, dtype=np.float64)


def value(kind, X):
    X = np.asarray(X, dtype=np.float64)
    d = X.shape[1]
    if kind == OBJ_RASTRIGIN:
        return -(X * X - RASTRIGIN_A * np.cos(2.0 * np.pi * X) + RASTRIGIN_A).sum(axis=1)
    if kind == OBJ_ACKLEY:
        S, C = (X * X).sum(axis=1), np.cos(ACKLEY_C * X).sum(axis=1)
        return ACKLEY_A * np.exp(-ACKLEY_B * np.sqrt(S / d)) + np.exp(C / d) - ACKLEY_A - np.e
    if kind == OBJ_SCHWEFEL:
        return (X * np.sin(np.sqrt(np.abs(X)))).sum(axis=1) - SCHWEFEL_C * d
    if kind == OBJ_STYBLINSKI_TANG:
        return -0.5 * (X ** 4 - 16.0 * X ** 2 + 5.0 * X).sum(axis=1)
    if kind == OBJ_MICHALEWICZ:
        U = _idx(d)[None, :] * X * X / np.pi
        return (np.sin(X) * np.sin(U) ** (2 * MICHALEWICZ_M)).sum(axis=1)
    if kind == OBJ_TRID:
        return -((X - 1.0) ** 2).sum(axis=1) + (X[:, 1:] * X[:, :-1]).sum(axis=1)
    if kind == OBJ_BUKIN6:
        x, y = X[:, 0], X[:, 1]
        return -100.0 * np.sqrt(np.abs(y - 0.01 * x * x)) - 0.01 * np.abs(x + 10.0)
    raise ValueError(kind)


def grad(kind, X):
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    if kind == OBJ_RASTRIGIN:
        return -(2.0 * X + 2.0 * np.pi * RASTRIGIN_A * np.sin(2.0 * np.pi * X))
    if kind == OBJ_ACKLEY:
        S, C = (X * X).sum(axis=1), np.cos(ACKLEY_C * X).sum(axis=1)
        r = np.sqrt(S / d)
        safe = np.where(r > 0.0, r, 1.0)
        radial = np.where(r > 0.0, -ACKLEY_A * ACKLEY_B * np.exp(-ACKLEY_B * r) / (d * safe), 0.0)
        return radial[:, None] * X - (ACKLEY_C / d) * np.exp(C / d)[:, None] * np.sin(ACKLEY_C * X)
    if kind == OBJ_SCHWEFEL:
        s = np.sqrt(np.abs(X))
        return np.sin(s) + 0.5 * s * np.cos(s)
    if kind == OBJ_STYBLINSKI_TANG:
        return -0.5 * (4.0 * X ** 3 - 32.0 * X + 5.0)
    if kind == OBJ_MICHALEWICZ:
        i = _idx(d)[None, :]
        U = i * X * X / np.pi
        su, cu = np.sin(U), np.cos(U)
        m2 = 2 * MICHALEWICZ_M
        return np.cos(X) * su ** m2 + np.sin(X) * m2 * su ** (m2 - 1) * cu * (2.0 * i * X / np.pi)
    if kind == OBJ_TRID:
        G = -2.0 * (X - 1.0)
        G[:, 1:] += X[:, :-1]
        G[:, :-1] += X[:, 1:]
        return G
    if kind == OBJ_BUKIN6:
        x, y = X[:, 0], X[:, 1]
        w = y - 0.01 * x * x
        aw = np.abs(w)
        dw = np.where(aw > 0.0, -50.0 * np.sign(w) / np.sqrt(np.where(aw > 0.0, aw, 1.0)), 0.0)   # d f / d w
        return np.stack([dw * (-0.02 * x) - 0.01 * np.sign(x + 10.0), dw], axis=1)
    raise ValueError(kind)


def hessian(kind, x):
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[0]
    if kind == OBJ_RASTRIGIN:
        return np.diag(-(2.0 + 4.0 * np.pi ** 2 * RASTRIGIN_A * np.cos(2.0 * np.pi * x)))
    if kind == OBJ_SCHWEFEL:
        s = np.sqrt(np.abs(x))
        safe = np.where(s > 0.0, s, 1.0)
        h = np.where(s > 0.0, np.sign(x) * (0.75 * np.cos(s) / safe - 0.25 * np.sin(s)), 0.0)
        return np.diag(h)
    if kind == OBJ_STYBLINSKI_TANG:
        return np.diag(-0.5 * (12.0 * x ** 2 - 32.0))
    if kind == OBJ_TRID:
        H = -2.0 * np.eye(d)
        H[np.arange(1, d), np.arange(d - 1)] = 1.0
        H[np.arange(d - 1), np.arange(1, d)] = 1.0
        return H
    if kind == OBJ_MICHALEWICZ:
        i = _idx(d)
        U = i * x * x / np.pi
        su, cu = np.sin(U), np.cos(U)
        du = 2.0 * i * x / np.pi
        m2 = 2 * MICHALEWICZ_M
        p = su ** m2                                     # sin^20 u and its derivatives in x
        dp = m2 * su ** (m2 - 1) * cu * du
        ddp = (m2 * (m2 - 1) * su ** (m2 - 2) * cu * cu * du * du - m2 * su ** m2 * du * du
               + m2 * su ** (m2 - 1) * cu * (2.0 * i / np.pi))
        return np.diag(-np.sin(x) * p + 2.0 * np.cos(x) * dp + np.sin(x) * ddp)
    # Ackley and Bukin N.6: central differences of the analytic gradient
    h = 1e-6 * max(1.0, float(np.abs(x).max()))
    H = np.stack([(grad(kind, (x + h * e)[None])[0] - grad(kind, (x - h * e)[None])[0]) / (2 * h)
                  for e in np.eye(d)], axis=1)
    return 0.5 * (H + H.T)
