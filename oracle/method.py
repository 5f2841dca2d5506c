"""The ChiSao oscillation cycle in FP64 -- oracle (test infrastructure only).

Algorithm 1 (Section 3.4), phase by phase, vectorised over the sample index
(every phase acts on each sample independently except for the population
reductions, which Section 3.5 also treats as batched operations):

    for k = 1..n_osc:
        stuck <- False                                   Phase 1, Sec. 3.2.1
        x, grad f(x) <- L-BFGS_batch(x, n_conv)          Eq. 2
        f_max <- max_i f(x_i)
        stuck_i <- |grad f(x_i)|_inf < eps_grad and
                   f(x_i) >= f_max + log(delta)          Phase 2, Eq. 3
        x, K_lost <- deduplicate(x, stuck, eps_dup)      Phase 3, Eq. 4
        if k < n_osc:
            reseed (Repulse Monkey / Golden Rooster)     Phase 4, Sec. 3.2.4
            Hands Like Clouds on unfrozen samples        Phase 5, Eq. 5
            anti-convergence on unfrozen samples         Phase 6, Eq. 6
    return {x_i : stuck_i}

Where the paper leaves a detail open the code follows one stated reading
(line search, history lifetime, step sizes, tie-breaks, ray rules); each is
noted at the function that implements it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from . import objectives as OB
from . import philox as PX

GRAD_FD64 = 0     # central differences, h absolute, FP64 stencil and values
GRAD_FD32 = 1     # central differences, h_j = h_rel * max(1, |x_j|)
GRAD_ADJOINT = 2  # exact analytic gradient

RESEED_NONE, RESEED_RM, RESEED_GR, RESEED_UNIFORM = 0, 1, 2, 3


@dataclasses.dataclass
class Params:
    """Hyperparameters of Table 1 plus the readings that fix unstated details."""
    n_osc: int = 3
    n_conv: int = 0            # 0 -> max(10, ceil(3 log2 d))  (Sec. 3.2.1)
    n_anti: int = 5
    n_cloud: int = 3
    M: int = 8                 # perturbations per smoothed gradient (K in Eq. 5)
    m: int = 10                # L-BFGS memory
    T_ls: int = 20             # backtracking trials
    eps_grad: float = 1e-6
    eps_dup: float = 1e-3
    delta: float = 0.1
    mu: float = 0.9
    alpha: float = 0.0         # <= 0: auto
    sigma: float = 0.0         # <= 0: auto, c_sigma * std(unfrozen x)
    c_sigma: float = 0.1
    alpha_scale: float = 0.1   # auto step: alpha = alpha_scale * s / g_rms
    h: float = 1e-5            # FD64 absolute step
    h_rel: float = 2.0 ** (-23.0 / 3.0)   # FD32 relative step (cube root of binary32 eps)
    c1: float = 1e-4           # Armijo constant
    curv_eps: float = 1e-10    # curvature-pair acceptance s^T y > curv_eps |s||y|
    grad_mode: int = GRAD_FD64
    seed: int = 0
    rm_min_unfrozen: int = 5   # Repulse Monkey needs >= 5 unfrozen samples
    gr_patience: int = 2       # Golden Rooster disables after 2 generations without new peaks
    hlc_value_only: int = 0    # 1: Phase 5 with the value-only smoothing estimator (a variant)

    def n_conv_for(self, d: int) -> int:
        if self.n_conv > 0:
            return self.n_conv
        return max(10, int(math.ceil(3.0 * math.log2(d)))) if d > 1 else 10


@dataclasses.dataclass
class State:
    x: np.ndarray              # (N, d)
    f: np.ndarray              # (N,)
    g: np.ndarray              # (N, d) gradient of f
    S: np.ndarray              # (N, m, d) L-BFGS s pairs, slot 0 = newest
    Y: np.ndarray              # (N, m, d) y pairs (of F = -f)
    rho: np.ndarray            # (N, m) 1 / s^T y
    hlen: np.ndarray           # (N,) number of stored pairs
    stuck: np.ndarray          # (N,) bool
    removed: np.ndarray        # (N,) bool, removed by the last deduplication
    cycle: int = 0             # completed cycles
    gr_enabled: bool = True
    gr_noprog: int = 0
    gr_prev_surv: int = -1
    evals: int = 0             # objective evaluations performed
    grads: int = 0             # gradient evaluations performed
    ls_fail: int = 0
    last_k_lost: int = 0
    last_reseed: int = RESEED_NONE
    last_fmax: float = float("nan")


def new_state(x0, m: int) -> State:
    x = np.asarray(x0, dtype=np.float64).copy()
    N, d = x.shape
    return State(x=x, f=np.zeros(N), g=np.zeros((N, d)), S=np.zeros((N, m, d)), Y=np.zeros((N, m, d)),
                 rho=np.zeros((N, m)), hlen=np.zeros(N, dtype=np.int64), stuck=np.zeros(N, bool),
                 removed=np.zeros(N, bool))


# ----------------------------------------------------------------------------------------------
# objective access (Sec. 3.1: gradients from differences of values, or exact where available)
# ----------------------------------------------------------------------------------------------

def _pidx(prob) -> int:
    """Index of the problem within a batched context (0 for a lone problem)."""
    return int(getattr(prob, "index", 0))


def evaluate(prob, X, st: Optional[State] = None, seed: int = 0, prob_index: int = 0):
    """f at the rows of X, plus the additive N(0, sigma_noise^2) evaluation noise
    of Sec. 5.6 when the objective has some.  Reading (the paper does not say
    how the noise is drawn): each evaluation point gets its own draw, keyed by
    the point's binary32 coordinates (philox.point_noise), so repeated
    evaluations of one point see the same value.  Parity with the paper's noise
    table is unpinned."""
    if st is not None:
        st.evals += X.shape[0]
    f = OB.value(prob.objective, X)
    s = getattr(prob.objective, "noise_sigma", 0.0)
    if s:
        f = f + s * PX.point_noise(seed, prob_index, X)
    return f


def fd_steps(X, P: Params):
    """Per-coordinate FD steps: absolute h (FD64) or h_rel * max(1, |x_j|) (FD32)."""
    if P.grad_mode == GRAD_FD32:
        return P.h_rel * np.maximum(1.0, np.abs(X))
    return np.full_like(X, P.h)


def fd_gradient(prob, X, P: Params, st: Optional[State] = None):
    """Central differences g_j = (f(x + h_j e_j) - f(x - h_j e_j)) / ((x_j + h_j) - (x_j - h_j)),
    the difference of the two stencil coordinates as the denominator."""
    X = np.asarray(X, dtype=np.float64)
    H = fd_steps(X, P)
    N, d = X.shape
    G = np.empty((N, d))
    for j in range(d):
        Xp = X.copy()
        Xm = X.copy()
        Xp[:, j] = X[:, j] + H[:, j]
        Xm[:, j] = X[:, j] - H[:, j]
        G[:, j] = (evaluate(prob, Xp, st, P.seed, _pidx(prob)) -
                   evaluate(prob, Xm, st, P.seed, _pidx(prob))) / (Xp[:, j] - Xm[:, j])
    return G


def gradient(prob, X, P: Params, st: Optional[State] = None):
    if st is not None:
        st.grads += X.shape[0]
    if P.grad_mode == GRAD_ADJOINT:
        return OB.grad(prob.objective, X)
    return fd_gradient(prob, X, P, st)


# ----------------------------------------------------------------------------------------------
# Phase 1: batched L-BFGS (Sec. 3.2.1, Eq. 2), maximising f = minimising F = -f
# ----------------------------------------------------------------------------------------------

def lbfgs_direction(G, S, Y, rho, hlen):
    """Two-loop recursion (Nocedal & Wright, Algorithm 7.4) for p = -H grad F.

    H_0 = gamma I with gamma = s^T y / y^T y of the newest pair (gamma = 1 with
    an empty history).  Slot 0 holds the newest pair.
    """
    N, m, d = S.shape
    q = np.array(G, dtype=np.float64, copy=True)
    a = np.zeros((N, m))
    for i in range(m):                                   # newest -> oldest
        act = hlen > i
        ai = rho[:, i] * np.einsum("nd,nd->n", S[:, i], q)
        ai = np.where(act, ai, 0.0)
        a[:, i] = ai
        q = q - ai[:, None] * Y[:, i]
    sy = np.einsum("nd,nd->n", S[:, 0], Y[:, 0])
    yy = np.einsum("nd,nd->n", Y[:, 0], Y[:, 0])
    gamma = np.where(hlen > 0, sy / np.where(yy > 0, yy, 1.0), 1.0)
    r = gamma[:, None] * q
    for i in reversed(range(m)):                         # oldest -> newest
        act = hlen > i
        b = rho[:, i] * np.einsum("nd,nd->n", Y[:, i], r)
        r = r + np.where(act, a[:, i] - b, 0.0)[:, None] * S[:, i]
    return -r


def line_search(prob, X, F, G, Pd, alpha0, P: Params, st: Optional[State] = None, active=None):
    """Backtracking Armijo search on F = -f over alpha = alpha0 * 2^-t, t < T_ls.

    Trial points are projected onto the box, x_t = clip(x + alpha p), and the
    sufficient-decrease test is F(x_t) <= F(x) + c1 * grad F^T (x_t - x).  The
    first passing trial is the largest passing alpha.  Returns
    (accepted, x_new, F_new, trials).
    """
    N, d = X.shape
    lo, hi = prob.lo, prob.hi
    if active is None:
        active = np.ones(N, bool)
    acc = np.zeros(N, bool)
    Xn = X.copy()
    Fn = F.copy()
    trials = np.zeros(N, dtype=np.int64)
    for t in range(P.T_ls):
        todo = active & ~acc
        if not todo.any():
            break
        idx = np.flatnonzero(todo)
        a = alpha0[idx] * 2.0 ** (-t)
        Xt = np.clip(X[idx] + a[:, None] * Pd[idx], lo, hi)
        Ft = -evaluate(prob, Xt, st, P.seed, _pidx(prob))
        trials[idx] += 1
        ok = Ft <= F[idx] + P.c1 * np.einsum("nd,nd->n", G[idx], Xt - X[idx])
        sel = idx[ok]
        acc[sel] = True
        Xn[sel] = Xt[ok]
        Fn[sel] = Ft[ok]
    return acc, Xn, Fn, trials


def push_pair(st: State, idx, s, y, P: Params):
    """Store (s, y) as the newest pair when it has curvature s^T y > curv_eps |s| |y|
    and rho = 1 / s^T y is finite in the state precision (a subnormal s^T y, reached
    when the coordinates converge to 0, would store an infinite rho)."""
    sy = np.einsum("nd,nd->n", s, y)
    nrm = np.sqrt(np.einsum("nd,nd->n", s, s) * np.einsum("nd,nd->n", y, y))
    ok = (sy > P.curv_eps * nrm) & (sy >= 1.0 / np.finfo(np.float64).max)
    j = idx[ok]
    if j.size:
        st.S[j] = np.roll(st.S[j], 1, axis=1)
        st.Y[j] = np.roll(st.Y[j], 1, axis=1)
        st.rho[j] = np.roll(st.rho[j], 1, axis=1)
        st.S[j, 0] = s[ok]
        st.Y[j, 0] = y[ok]
        st.rho[j, 0] = 1.0 / sy[ok]
        st.hlen[j] = np.minimum(st.hlen[j] + 1, st.S.shape[1])
    return ok


def lbfgs_iterations(prob, st: State, P: Params, n_iter: int, fresh_gradient: bool = True):
    """n_iter L-BFGS iterations on every sample (direction, line search, new
    gradient, history update).  With ``fresh_gradient`` the gradient and value
    at the starting points are evaluated first (start of Phase 1)."""
    X = st.x
    N, d = X.shape
    if fresh_gradient:
        st.f = evaluate(prob, X, st, P.seed, _pidx(prob))
        st.g = gradient(prob, X, P, st)
    F = -st.f
    G = -st.g
    for _ in range(n_iter):
        gnorm = np.abs(G).max(axis=1)
        with np.errstate(divide="ignore", over="ignore"):
            inv_g = np.where(gnorm > 0, 1.0 / np.where(gnorm > 0, gnorm, 1.0), 1.0)
        moving = gnorm > 0.0
        Pd = lbfgs_direction(G, st.S, st.Y, st.rho, st.hlen)
        alpha0 = np.where(st.hlen > 0, 1.0, np.minimum(1.0, inv_g))
        gp = np.einsum("nd,nd->n", G, Pd)
        # restart when p is an ascent direction or not finite; g^T p = 0 (a product that
        # underflows next to a stationary point) keeps the history, the mode's curvature
        bad = moving & ~(gp <= 0.0)
        if bad.any():
            st.hlen[bad] = 0
            Pd[bad] = -G[bad]
            alpha0[bad] = np.minimum(1.0, inv_g[bad])
        acc, Xn, Fn, _ = line_search(prob, X, F, G, Pd, alpha0, P, st, active=moving)
        failed = moving & ~acc
        if failed.any():
            st.hlen[failed] = 0
            st.ls_fail += int(failed.sum())
        idx = np.flatnonzero(acc)
        if idx.size:
            Gn = -gradient(prob, Xn[idx], P, st)
            push_pair(st, idx, Xn[idx] - X[idx], Gn - G[idx], P)
            X[idx] = Xn[idx]
            F[idx] = Fn[idx]
            G[idx] = Gn
    st.x = X
    st.f = -F
    st.g = -G


# ----------------------------------------------------------------------------------------------
# Phase 2: stick detection (Eq. 3)
# ----------------------------------------------------------------------------------------------

def fmax_of(f):
    fin = np.isfinite(f)
    return float(f[fin].max()) if fin.any() else float("-inf")


def freeze(f, g, eps_grad, delta, dtype=np.float64):
    """stuck_i = (|g_i|_inf < eps_grad) and (f_i >= f_max + log delta).

    ``dtype`` is the precision the comparisons are taken in: float32 inputs
    with dtype=float32 reproduce the binary32 decision of the GPU bit for bit
    (threshold thr = fl(f_max + fl(log delta)))."""
    f = np.asarray(f, dtype=dtype)
    g = np.asarray(g, dtype=dtype)
    fmax = dtype(fmax_of(f))
    thr = dtype(fmax + dtype(np.log(delta)))
    gmax = np.abs(g).max(axis=1)
    stuck = (gmax < dtype(eps_grad)) & (f >= thr)
    return stuck, float(fmax)


# ----------------------------------------------------------------------------------------------
# Phase 3: L-infinity deduplication (Eq. 4, Appendix A)
# ----------------------------------------------------------------------------------------------

def dedup(x, f, stuck, eps_dup, dtype=np.float64, chunk=64):
    """Remove stuck x_j when some other stuck x_i lies within L-inf distance
    eps_dup and ranks above it.  Ranking is the strict total order (f desc,
    index asc), so of two equal-valued neighbours the lower index survives; i
    is tested whether or not i is itself removed (the literal, order-free
    reading of Eq. 4).  Returns the removed mask."""
    N = x.shape[0]
    idx = np.flatnonzero(stuck)
    xs = np.asarray(x, dtype=dtype)[idx]
    fs = np.asarray(f, dtype=dtype)[idx]
    eps = dtype(eps_dup)
    removed = np.zeros(N, bool)
    S = idx.size
    for j0 in range(0, S, chunk):
        j1 = min(S, j0 + chunk)
        D = np.abs(xs[None, :, :] - xs[j0:j1, None, :]).max(axis=2)          # (cj, S)
        close = D < eps
        above = (fs[None, :] > fs[j0:j1, None]) | ((fs[None, :] == fs[j0:j1, None]) &
                                                   (idx[None, :] < idx[j0:j1, None]))
        removed[idx[j0:j1]] = (close & above).any(axis=1)
    return removed


# ----------------------------------------------------------------------------------------------
# Phase 4: reseeding (Sec. 3.2.4)
# ----------------------------------------------------------------------------------------------

def householder_qr(A):
    """Householder QR (Golub & Van Loan, Algorithm 5.2.1) with Q formed
    explicitly, normalised so that diag(R) > 0 (which makes Q unique)."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    Q = np.eye(n)
    for j in range(n - 1):
        x = A[j:, j]
        alpha = np.linalg.norm(x)
        if alpha == 0.0:
            continue
        v = x.copy()
        v[0] += math.copysign(alpha, x[0])
        v /= np.linalg.norm(v)
        A[j:, :] -= 2.0 * np.outer(v, v @ A[j:, :])
        Q[:, j:] -= 2.0 * np.outer(Q[:, j:] @ v, v)
    sgn = np.where(np.diag(A) < 0.0, -1.0, 1.0)
    return Q * sgn[None, :], sgn[:, None] * A


def ray_exit(p, u, lo, hi):
    """Largest t >= 0 with p + t u inside the box (per row)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        tp = np.where(u > 0, (hi[None, :] - p) / u, np.inf)
        tn = np.where(u < 0, (lo[None, :] - p) / u, np.inf)
    t = np.minimum(tp, tn).min(axis=1)
    return np.maximum(np.where(np.isfinite(t), t, 0.0), 0.0)


def reseed(prob, st: State, P: Params, cycle: int, prob_index: int = 0):
    """Fill the K_lost slots removed by deduplication.

    * Repulse Monkey (>= 5 unfrozen): for free slot r (in index order) the
      parent is unfrozen[floor(w0 U / 2^32)] (unfrozen samples in index order),
      the direction a normalised Gaussian, the child uniform on the ray inside
      the box: parent + u(w1) t_exit u.
    * Golden Rooster (< 5 unfrozen): one Gaussian d x d matrix per generation,
      Q from its Householder QR; survivors ranked (f desc, index asc); slot r
      uses peak r mod S, column floor(r/S) mod d, sign + when floor(r/(S d)) is
      even, and a uniform position on that ray inside the box.  GR disables
      itself after ``gr_patience`` successive generations whose survivor count
      did not grow; it then (and with no survivor) redraws uniformly in the box.
    Reseeded samples are unstuck and start with an empty L-BFGS history.
    """
    d = prob.d
    free = np.flatnonzero(st.removed)
    K = free.size
    st.last_k_lost = int(K)
    st.last_reseed = RESEED_NONE
    if K == 0:
        return
    unfrozen = np.flatnonzero(~st.stuck & ~st.removed)
    U = unfrozen.size
    surv = np.flatnonzero(st.stuck & ~st.removed)
    S = surv.size
    r = np.arange(K)
    mode = RESEED_UNIFORM
    if U >= P.rm_min_unfrozen:
        mode = RESEED_RM
    elif st.gr_enabled and S > 0:
        if st.gr_prev_surv >= 0:
            st.gr_noprog = 0 if S > st.gr_prev_surv else st.gr_noprog + 1
        if st.gr_noprog >= P.gr_patience:
            st.gr_enabled = False
        else:
            mode = RESEED_GR
            st.gr_prev_surv = S
    seed = P.seed
    if mode == RESEED_RM:
        w = PX.words(seed, r, 0, PX.TAG_RM, cycle, 0, prob_index, 0)
        pick = (w[:, 0].astype(np.uint64) * np.uint64(U)) >> np.uint64(32)
        parent = st.x[unfrozen[pick.astype(np.int64)]]
        z = PX.normal_rows(seed, r, d, PX.TAG_RM_DIR, cycle, 0, prob_index, 0)
        u = z / np.linalg.norm(z, axis=1, keepdims=True)
        t = PX.u01(w[:, 1]) * ray_exit(parent, u, prob.lo, prob.hi)
        child = np.clip(parent + t[:, None] * u, prob.lo, prob.hi)
    elif mode == RESEED_GR:
        Gm = PX.normal_rows(seed, np.arange(d), d, PX.TAG_GR_MAT, cycle, 0, prob_index, 0)
        Q, _ = householder_qr(Gm)
        order = np.lexsort((surv, -st.f[surv]))          # f descending, index ascending
        ranked = surv[order]
        peak = st.x[ranked[r % S]]
        col = (r // S) % d
        sgn = np.where(((r // (S * d)) % 2) == 0, 1.0, -1.0)
        u = sgn[:, None] * Q[:, col].T
        w = PX.words(seed, r, 0, PX.TAG_GR_T, cycle, 0, prob_index, 0)
        t = PX.u01(w[:, 0]) * ray_exit(peak, u, prob.lo, prob.hi)
        child = np.clip(peak + t[:, None] * u, prob.lo, prob.hi)
    else:
        uu = PX.uniform_rows(seed, r, d, PX.TAG_UNIFORM, cycle, 0, prob_index, 0)
        child = prob.lo[None, :] + uu * (prob.hi - prob.lo)[None, :]
    st.x[free] = child
    st.stuck[free] = False
    st.hlen[free] = 0
    st.last_reseed = mode


# ----------------------------------------------------------------------------------------------
# Phases 5 and 6: Hands Like Clouds (Eq. 5) and anti-convergence (Eq. 6)
# ----------------------------------------------------------------------------------------------

def population_scales(prob, st: State, P: Params, unfrozen):
    """Scale estimates over the unfrozen samples at a phase start.

    s     = sqrt(mean_j var_j), the per-coordinate population variance
            (divide by the count) pooled over coordinates;
    sigma = c_sigma * s (Sec. 3.2.5) unless supplied;
    g_rms = RMS of all gradient components at the current points;
    alpha = alpha_scale * s / max(g_rms, 1e-30) unless supplied.
    The gradient at the current points is returned for reuse."""
    idx = np.flatnonzero(unfrozen)
    X = st.x[idx]
    G = gradient(prob, X, P, st)
    U = idx.size
    mean = X.mean(axis=0)
    var = ((X - mean[None, :]) ** 2).mean(axis=0)
    s = math.sqrt(var.mean())
    g_rms = math.sqrt(float((G * G).sum()) / (U * prob.d))
    sigma = P.sigma if P.sigma > 0 else P.c_sigma * s
    alpha = P.alpha if P.alpha > 0 else P.alpha_scale * s / max(g_rms, 1e-30)
    return idx, G, sigma, alpha, s, g_rms


def hlc(prob, st: State, P: Params, cycle: int, prob_index: int = 0):
    """n_cloud ascent steps x <- clip(x + alpha_h * (1/M) sum_k grad f(x + sigma z_k))
    on unfrozen samples, z_k from the TAG_HLC stream (c0 = sample index,
    step = cloud step, k = perturbation).  The step alpha_h follows the same
    auto rule as the anti-convergence step, evaluated at the phase start.
    With P.hlc_value_only the gradients are replaced by the value-only
    Gaussian-smoothing estimator (f(x + sigma z_k) - f(x)) z_k / sigma (a
    variant of Eq. 5 built from M + 1 evaluations)."""
    unfrozen = ~st.stuck
    if not unfrozen.any() or P.n_cloud == 0:
        return None
    idx, _, sigma, alpha, s, g_rms = population_scales(prob, st, P, unfrozen)
    X = st.x[idx]
    d = prob.d
    for t in range(P.n_cloud):
        acc = np.zeros_like(X)
        f0 = evaluate(prob, X, st, P.seed, prob_index) if P.hlc_value_only else None
        for k in range(P.M):
            z = PX.normal_rows(P.seed, idx, d, PX.TAG_HLC, cycle, t, prob_index, k)
            if P.hlc_value_only:
                # Gaussian-smoothing estimator from values only: (f(x + sigma z) - f(x)) z / sigma
                acc += ((evaluate(prob, X + sigma * z, st, P.seed, prob_index) - f0) / sigma)[:, None] * z
            else:
                acc += gradient(prob, X + sigma * z, P, st)
        X = np.clip(X + alpha * (acc / P.M), prob.lo, prob.hi)
    st.x[idx] = X
    st.hlen[idx] = 0
    return sigma, alpha


def anti_converge(prob, st: State, P: Params):
    """n_anti momentum descent steps v <- mu v - alpha grad f(x), x <- x + v
    (Eq. 6) on unfrozen samples with v_0 = 0; x is projected onto the box and
    v is zeroed on the coordinates the projection changed."""
    unfrozen = ~st.stuck
    if not unfrozen.any() or P.n_anti == 0:
        return None
    idx, G, _, alpha, _, _ = population_scales(prob, st, P, unfrozen)
    X = st.x[idx]
    V = np.zeros_like(X)
    for t in range(P.n_anti):
        if t > 0:
            G = gradient(prob, X, P, st)
        V = P.mu * V - alpha * G
        Xn = X + V
        Xc = np.clip(Xn, prob.lo, prob.hi)
        V = np.where(Xc != Xn, 0.0, V)
        X = Xc
    st.x[idx] = X
    st.hlen[idx] = 0
    return alpha


# ----------------------------------------------------------------------------------------------
# one oscillation cycle and the driver (Algorithm 1)
# ----------------------------------------------------------------------------------------------

def cycle(prob, st: State, P: Params, prob_index: int = 0, last: Optional[bool] = None):
    k = st.cycle + 1                                      # 1-based cycle number
    if last is None:
        last = k >= P.n_osc
    st.stuck[:] = False                                   # Phase 1: release all
    st.removed[:] = False
    lbfgs_iterations(prob, st, P, P.n_conv_for(prob.d))
    st.stuck, st.last_fmax = freeze(st.f, st.g, P.eps_grad, P.delta)        # Phase 2
    st.removed = dedup(st.x, st.f, st.stuck, P.eps_dup)                      # Phase 3
    st.stuck &= ~st.removed
    st.last_k_lost = int(st.removed.sum())
    if not last:
        reseed(prob, st, P, k, prob_index)                                   # Phase 4
        hlc(prob, st, P, k, prob_index)                                      # Phase 5
        anti_converge(prob, st, P)                                           # Phase 6
    st.cycle = k
    return st


def refine(prob, st: State, P: Params, n_refine: int):
    """Final refinement of the returned modes when the cycles ran on a lower-precision
    objective (the tensor-core mixture of BF16-rounded factors).  The paper has no such
    step; its reading: after the last cycle's Phase 3, each survivor (stuck and not
    removed) takes n_refine more Phase 1 iterations (Sec. 3.2.1, Eq. 2) on `prob`'s
    exact objective, starting from a fresh value and gradient at its point and keeping
    its L-BFGS history (Sec. 3.2.3 preserves it).  No other sample changes, and no stick
    test or deduplication follows: the refined survivors are the mode set."""
    idx = np.flatnonzero(st.stuck & ~st.removed)
    if n_refine <= 0 or idx.size == 0:
        return st
    sub = State(x=st.x[idx].copy(), f=st.f[idx].copy(), g=st.g[idx].copy(), S=st.S[idx].copy(),
                Y=st.Y[idx].copy(), rho=st.rho[idx].copy(), hlen=st.hlen[idx].copy(),
                stuck=np.ones(idx.size, bool), removed=np.zeros(idx.size, bool))
    lbfgs_iterations(prob, sub, P, n_refine, fresh_gradient=True)
    st.x[idx], st.f[idx], st.g[idx] = sub.x, sub.f, sub.g
    st.S[idx], st.Y[idx], st.rho[idx], st.hlen[idx] = sub.S, sub.Y, sub.rho, sub.hlen
    st.evals += sub.evals
    st.grads += sub.grads
    st.ls_fail += sub.ls_fail
    return st


def run(prob, P: Params, prob_index: int = 0):
    st = new_state(prob.x0, P.m)
    for _ in range(P.n_osc):
        cycle(prob, st, P, prob_index)
    return modes_of(st), st


def modes_of(st: State):
    idx = np.flatnonzero(st.stuck)
    return st.x[idx].copy(), st.f[idx].copy()


def laplace_widths(st: State, idx):
    """Laplace widths of the samples idx (normally the survivors) from their kept
    L-BFGS history.  Sec. 3.2.3 keeps a surviving sample's inverse-Hessian estimate
    so that its width can be estimated; the paper gives no formula, so this is a
    reading: the estimate is the matrix H that the two-loop recursion applies
    (H_0 = gamma I with gamma of the newest pair), and under the Laplace
    approximation of f = log p at the mode the covariance is H, the inverse of the
    Hessian of F = -f.  Column j of H is H e_j = -lbfgs_direction(e_j); the width
    along coordinate j is sqrt(H_jj).  Returns (H (k, d, d), widths (k, d)).
    """
    idx = np.asarray(idx, dtype=np.int64)
    k, d = idx.size, st.x.shape[1]
    H = np.empty((k, d, d))
    for j in range(d):
        E = np.zeros((k, d))
        E[:, j] = 1.0
        H[:, :, j] = -lbfgs_direction(E, st.S[idx], st.Y[idx], st.rho[idx], st.hlen[idx])
    w = np.sqrt(np.maximum(np.diagonal(H, axis1=1, axis2=2), 0.0))
    return H, w
