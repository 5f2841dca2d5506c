"""Objective families in FP64 (oracle side): value, analytic gradient, Hessian.

* Gaussian mixture log-density (Appendix D "Gaussian mixture", generalised to
  per-component weights and diagonal or full covariances):
      f(x) = log sum_k w_k N(x; mu_k, Sigma_k)
  computed as a log-sum-exp over the component log-densities.
* Rotated quadratic f(x) = -(x-c)^T Q^T Lambda Q (x-c) (a log-concave target
  with the single mode c, the setting of Proposition 1).
* The benchmark functions of Appendix D (``oracle.benchmarks``).

The optional additive noise of Section 5.6 (f~ = f + eps, eps ~ N(0, s^2)) is
applied by ``method.evaluate``, which knows the evaluation's stream position.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import benchmarks as BENCH

OBJ_MIXTURE_DIAG = 1
OBJ_MIXTURE_FULL = 2
OBJ_QUADRATIC = 3
OBJ_MIXTURE_PREC = 4      # mixture given by precision factors W_k (Sigma_k^-1 = W_k^T W_k)
OBJ_MIXTURE_PREC_SPLIT = 5   # the same, evaluated at the BF16-split input x_hi + x_lo

LOG2PI = np.log(2.0 * np.pi)


def bf16_round(a):
    """Round to bfloat16 (round to nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return (u.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def bf16_split(X):
    """x_hi + x_lo with x_hi = bf16(x), x_lo = bf16(x - x_hi) (x taken in binary32)."""
    x32 = np.asarray(X, dtype=np.float32).astype(np.float64)
    hi = bf16_round(x32)
    return hi + bf16_round(x32 - hi)


def tensor_core_objective(obj, split=True):
    """The full-covariance mixture with each precision factor L_k^-1 rounded to
    bfloat16 (its modes stay at the component centres); with ``split`` it is
    evaluated at the BF16-split input -- the objective the BF16 tensor-core path
    evaluates, value and gradient."""
    from paper_2606_26164_gb300.inputs import Objective
    A = obj.arrays
    W = np.stack([bf16_round(np.linalg.inv(L)) for L in A["chol"]])
    kind = OBJ_MIXTURE_PREC_SPLIT if split else OBJ_MIXTURE_PREC
    return Objective(kind, obj.d, {"weights": A["weights"], "means": A["means"], "linv": W})


def _component_logdens(obj, X):
    """log w_k + log N(x; mu_k, Sigma_k) for all samples and components -> (N, K),
    plus the per-component score a_k(x) = grad_x log N_k(x) -> (N, K, d)."""
    A = obj.arrays
    w, mu = A["weights"], A["means"]
    K, d = mu.shape
    if obj.kind == OBJ_MIXTURE_PREC_SPLIT:
        X = bf16_split(X)
    R = X[:, None, :] - mu[None, :, :]                     # (N, K, d)
    if obj.kind == OBJ_MIXTURE_DIAG:
        sig = A["sigmas"]
        Z = R / sig[None]
        logdet = np.log(sig).sum(axis=1)                   # log |Sigma_k|^(1/2)
        score = -R / (sig[None] ** 2)
    elif obj.kind in (OBJ_MIXTURE_PREC, OBJ_MIXTURE_PREC_SPLIT):
        W = A["linv"]
        Rk = R.transpose(1, 0, 2)                          # (K, N, d)
        Zk = np.matmul(Rk, W.transpose(0, 2, 1))           # rows z = W_k (x - mu_k)
        Z = Zk.transpose(1, 0, 2)
        score = -np.matmul(Zk, W).transpose(1, 0, 2)       # rows -W_k^T z_k
        logdet = -np.log(np.abs(np.einsum("kii->ki", W))).sum(axis=1)
    else:
        L = A["chol"]
        Z = np.empty_like(R)
        score = np.empty_like(R)
        for k in range(K):
            zk = solve_triangular(L[k], R[:, k, :].T, lower=True)          # L^-1 (x - mu)
            Z[:, k, :] = zk.T
            score[:, k, :] = -solve_triangular(L[k], zk, lower=True, trans="T").T   # -Sigma^-1 (x-mu)
        logdet = np.log(np.abs(np.einsum("kii->ki", L))).sum(axis=1)
    lc = np.log(w)[None, :] - 0.5 * np.einsum("nkd,nkd->nk", Z, Z) - logdet[None, :] - 0.5 * d * LOG2PI
    return lc, score


def _lse(lc):
    m = lc.max(axis=1, keepdims=True)
    return (m + np.log(np.exp(lc - m).sum(axis=1, keepdims=True)))[:, 0]


def value(obj, X):
    X = np.asarray(X, dtype=np.float64)
    if obj.kind in BENCH.BENCH_KINDS:
        return BENCH.value(obj.kind, X)
    if obj.kind == OBJ_QUADRATIC:
        A = obj.arrays
        Z = (X - A["center"][None, :]) @ A["Q"].T
        return -(Z * Z * A["lam"][None, :]).sum(axis=1)
    lc, _ = _component_logdens(obj, X)
    return _lse(lc)


def grad(obj, X):
    """Analytic gradient of f (the exact gradient the adjoint path computes)."""
    X = np.asarray(X, dtype=np.float64)
    if obj.kind in BENCH.BENCH_KINDS:
        return BENCH.grad(obj.kind, X)
    if obj.kind == OBJ_QUADRATIC:
        A = obj.arrays
        Q, lam = A["Q"], A["lam"]
        Z = (X - A["center"][None, :]) @ Q.T
        return -2.0 * (Z * lam[None, :]) @ Q
    lc, score = _component_logdens(obj, X)
    r = np.exp(lc - _lse(lc)[:, None])                      # responsibilities
    return np.einsum("nk,nkd->nd", r, score)


def _precisions(obj):
    """Sigma_k^-1 for every component (computed once per objective)."""
    cache = obj.__dict__.setdefault("_oracle_cache", {})
    if "prec" not in cache:
        A = obj.arrays
        if obj.kind == OBJ_MIXTURE_DIAG:
            cache["prec"] = np.stack([np.diag(1.0 / s ** 2) for s in A["sigmas"]])
        elif obj.kind in (OBJ_MIXTURE_PREC, OBJ_MIXTURE_PREC_SPLIT):
            cache["prec"] = np.einsum("kji,kjl->kil", A["linv"], A["linv"])
        else:
            P = []
            for L in A["chol"]:
                Linv = np.linalg.inv(L)
                P.append(Linv.T @ Linv)
            cache["prec"] = np.stack(P)
    return cache["prec"]


def hessian(obj, x):
    """Hessian of f at one point x (d,), for the Newton mode finder:
    sum_k r_k (a_k a_k^T - Sigma_k^-1) - gbar gbar^T."""
    if obj.kind in BENCH.BENCH_KINDS:
        return BENCH.hessian(obj.kind, x)
    x = np.asarray(x, dtype=np.float64)[None, :]
    if obj.kind == OBJ_QUADRATIC:
        A = obj.arrays
        Q, lam = A["Q"], A["lam"]
        return -2.0 * Q.T @ np.diag(lam) @ Q
    lc, score = _component_logdens(obj, x)
    r = np.exp(lc - _lse(lc)[:, None])[0]
    a = score[0]                                            # (K, d)
    prec = _precisions(obj)
    H = np.einsum("k,kij->ij", r, -prec) + np.einsum("k,ki,kj->ij", r, a, a)
    gbar = r @ a
    return H - np.outer(gbar, gbar)
