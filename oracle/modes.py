"""Ground-truth significant-mode sets (Eq. 1) -- oracle side, test infrastructure.

M* = { theta : grad f = 0, Hessian negative definite, f(theta) >= f_max + log delta }.

* Rotated quadratic: the single mode is the centre c (closed form).
* Gaussian mixtures: damped Newton's method in FP64 from every component
  mean; the distinct fixed points with a negative-definite Hessian that pass
  the delta gate are the significant modes.  For well-separated components each
  mode lies near one mean, so starting from every mean reaches all of them.

A returned point x matches mode theta* when its distance in units of the mode's
own local standard deviation, the Mahalanobis distance
sqrt((x - theta*)^T (-Hessian(theta*)) (x - theta*)), is at most 1e-3: for an
isotropic mode of width sigma this is |x - theta*|_2 <= 1e-3 sigma.
"""
from __future__ import annotations

import numpy as np

from . import objectives as OB


def newton_max(obj, x0, iters=200, tol=1e-13):
    x = np.array(x0, dtype=np.float64)
    f = OB.value(obj, x[None])[0]
    for _ in range(iters):
        g = OB.grad(obj, x[None])[0]
        if np.abs(g).max() < tol * max(1.0, abs(f)):
            break
        H = OB.hessian(obj, x)
        w = np.linalg.eigvalsh(H)
        step = -np.linalg.solve(H, g) if w.max() < 0 else g / max(1.0, np.abs(w).max())
        a = 1.0
        while a > 1e-12:
            xn = x + a * step
            fn = OB.value(obj, xn[None])[0]
            if fn >= f:
                break
            a *= 0.5
        if a <= 1e-12:
            break
        x, f = xn, fn
    return x, f


def significant_modes(prob, delta=0.1):
    """Returns (modes (K*, d), f values (K*,), -Hessian at each mode (K*, d, d))."""
    obj = prob.objective
    if obj.kind == OB.OBJ_QUADRATIC:
        c = obj.arrays["center"].copy()
        return c[None, :], np.array([0.0]), -OB.hessian(obj, c)[None]
    cands = []
    for mu in obj.arrays["means"]:
        x, f = newton_max(obj, mu)
        H = OB.hessian(obj, x)
        ev = np.linalg.eigvalsh(H)
        if ev.max() >= 0:
            continue
        if any(np.abs(x - c[0]).max() < 1e-6 for c in cands):
            continue
        cands.append((x, f, -H))
    fmax = max(c[1] for c in cands)
    keep = [c for c in cands if c[1] >= fmax + np.log(delta)]
    keep.sort(key=lambda c: -c[1])
    return (np.array([c[0] for c in keep]), np.array([c[1] for c in keep]),
            np.array([c[2] for c in keep]))


def mahalanobis(found_x, mode_x, neg_hess):
    """Distance of each found point from one mode in units of its local sigma."""
    D = np.asarray(found_x, dtype=np.float64) - mode_x[None, :]
    return np.sqrt(np.maximum(np.einsum("nd,de,ne->n", D, neg_hess, D), 0.0))


def recovery(found_x, modes_x, neg_hess, rel=1e-3):
    """(fraction of true modes matched within ``rel`` local sigmas, worst
    Mahalanobis error over the matched modes, best error per mode)."""
    found_x = np.asarray(found_x, dtype=np.float64).reshape(-1, modes_x.shape[1])
    best = np.full(modes_x.shape[0], np.inf)
    for k, (m, H) in enumerate(zip(modes_x, neg_hess)):
        if found_x.shape[0]:
            best[k] = mahalanobis(found_x, m, H).min()
    hit = best <= rel
    worst = float(best[hit].max()) if hit.any() else float("nan")
    return float(hit.mean()) if best.size else 0.0, worst, best
