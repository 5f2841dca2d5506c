"""Seeded synthetic workloads for the ChiSao population step.

This module only draws problem data (objective parameters, domain boxes and
initial populations) from seeded NumPy generators.  It contains none of the
method's arithmetic: the random numbers the method itself draws (reseeding
rays, Golden Rooster matrices, smoothing perturbations) come from counter-based
Philox streams that the CUDA library and the CPU oracle each implement.

Workloads (problem statement in Section 3.1; objectives below):

* ``mixture4_d2``   -- d=2, 4-component isotropic Gaussian mixture, means at
  (+-3, +-3), sigma=0.5, equal weights; N=1024 uniform in [-6, 6]^2.
* ``mixture32_d16`` -- d=16, K=32 diagonal mixture, means uniform in
  [-10, 10]^16 redrawn until pairwise separation >= 6 * max sigma, per-axis
  sigma log-uniform in [0.3, 1], Dirichlet(1) weights; N=16384.
* ``quadratic_d64`` -- d=64 rotated ill-conditioned quadratic
  f(x) = -(x-c)^T Q^T Lambda Q (x-c), Q orthogonal from the QR of a Gaussian
  matrix, Lambda geometric from 1 to 1e4, c uniform in [-5, 5]^64; N=65536.
* ``mixture256_d64`` -- d=64, K=256 full-covariance mixture, Cholesky factors
  lower-triangular (diagonal log-uniform [0.3, 1], strictly-lower N(0, 0.05^2),
  redrawn until cond_2 <= 100), means uniform in [-20, 20]^64, equal weights;
  N=65536.
* ``batched512``    -- 512 independent diagonal mixtures, d from
  {2,4,8,16,32,64}, N log-uniform in [256, 16384], K log-uniform integer in
  [4, 128], sigma uniform in [0.3, 1], means uniform in [-10, 10]^d, equal
  weights.
* ``benchmark(name, d, n)`` -- the Appendix D benchmark functions (Rastrigin,
  Ackley, Schwefel, Styblinski-Tang, Michalewicz, Trid, Bukin N.6) on their
  App. D domains, population uniform in the domain; ``rastrigin_d64`` etc.
  name the d = 64, N = 65536 cases.

The Gaussian-mixture family follows the mixture definition of Appendix D
(log of a weighted sum of Gaussian densities); the noise model of Section 5.6
adds N(0, sigma_noise^2) to every evaluation.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, List, Optional

import numpy as np

# Objective kinds (shared numbering with include/chisao.h).
OBJ_MIXTURE_DIAG = 1
OBJ_MIXTURE_FULL = 2
OBJ_QUADRATIC = 3
OBJ_EXTERNAL = 20        # a caller-supplied batched evaluator (Objective.fn)
# Appendix D benchmark functions (no parameters beyond d)
BENCHMARK_KINDS = {"rastrigin": 10, "ackley": 11, "schwefel": 12, "styblinski_tang": 13, "michalewicz": 14,
                   "trid": 15, "bukin6": 16}


@dataclasses.dataclass
class Objective:
    kind: int
    d: int
    # Mixtures: weights (K,), means (K, d); diag: sigmas (K, d);
    # full: chol (K, d, d) lower-triangular with Sigma_k = L_k L_k^T.
    # Quadratic: center (d,), Q (d, d) orthogonal, lam (d,).
    arrays: Dict[str, np.ndarray]
    noise_sigma: float = 0.0
    # OBJ_EXTERNAL: fn(x) -> (f, g) on CUDA float32 tensors x [k, d], f [k], g [k, d]
    # (g the exact gradient of f), run on the context's stream
    fn: Optional[Callable] = None

    @property
    def n_comp(self) -> int:
        return int(self.arrays["weights"].shape[0]) if "weights" in self.arrays else 0


@dataclasses.dataclass
class Problem:
    d: int
    n: int
    lo: np.ndarray          # (d,) float64 lower corner of the box Theta
    hi: np.ndarray          # (d,) float64 upper corner
    objective: Objective
    x0: np.ndarray          # (n, d) float32 initial population, uniform in Theta
    eps_grad: float         # stick threshold used with this problem
    sigma_mode: float       # 1/sqrt(lambda_max(-Hessian)) at the modes, for the 1e-3*sigma metric


def _uniform_box(rng, n, lo, hi):
    u = rng.random((n, lo.shape[0]))
    return (lo + u * (hi - lo)).astype(np.float32)


def mixture4_d2(n: int = 1024, seed: int = 0) -> Problem:
    d = 2
    means = np.array([[3.0, 3.0], [3.0, -3.0], [-3.0, 3.0], [-3.0, -3.0]])
    sig = np.full((4, d), 0.5)
    obj = Objective(OBJ_MIXTURE_DIAG, d, {"weights": np.full(4, 0.25), "means": means, "sigmas": sig})
    lo, hi = np.full(d, -6.0), np.full(d, 6.0)
    rng = np.random.default_rng(1000 + seed)
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-3, sigma_mode=0.5)


def mixture2_d6(n: int = 2048, seed: int = 0, noise_sigma: float = 0.0) -> Problem:
    """The noise-robustness workload of Sec. 5.6: two equally weighted unit-variance
    isotropic components at +2 e_1 and -2 e_1 in d = 6 (peaks four sigma apart).
    The box [-6, 6]^6 and the population size are this workload's choices (the paper
    states neither)."""
    d = 6
    means = np.zeros((2, d))
    means[0, 0], means[1, 0] = 2.0, -2.0
    obj = Objective(OBJ_MIXTURE_DIAG, d, {"weights": np.full(2, 0.5), "means": means, "sigmas": np.ones((2, d))},
                    noise_sigma)
    lo, hi = np.full(d, -6.0), np.full(d, 6.0)
    rng = np.random.default_rng(6000 + seed)
    # eps_grad 1e-4: a stuck point then lies within ~1e-4 of its peak (the local sigma is 1), so
    # the 1e-3 sigma recovery test and the 1e-3 dedup radius are not borderline
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-4, sigma_mode=1.0)


# the noise levels of the Sec. 5.6 table
NOISE_LEVELS = (1e-3, 1e-2, 0.05, 0.1, 0.2, 0.5, 1.0)


def _separated_means(rng, K, d, box, sig_max, sep):
    means = np.empty((K, d))
    for k in range(K):
        for _ in range(100000):
            cand = rng.uniform(-box, box, size=d)
            ok = all(np.linalg.norm(cand - means[l]) >= sep * max(sig_max[k], sig_max[l]) for l in range(k))
            if ok:
                break
        means[k] = cand
    return means


def mixture32_d16(n: int = 16384, seed: int = 0, noise_sigma: float = 0.0) -> Problem:
    d, K = 16, 32
    rng = np.random.default_rng(2000 + seed)
    sig = np.exp(rng.uniform(np.log(0.3), np.log(1.0), size=(K, d)))
    means = _separated_means(rng, K, d, 10.0, sig.max(axis=1), 6.0)
    e = -np.log(rng.random(K))                      # Dirichlet(1) = normalised Exp(1)
    w = e / e.sum()
    obj = Objective(OBJ_MIXTURE_DIAG, d, {"weights": w, "means": means, "sigmas": sig}, noise_sigma)
    lo, hi = np.full(d, -10.0), np.full(d, 10.0)
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-3,
                   sigma_mode=float(sig.min()))


def random_orthogonal(rng, d) -> np.ndarray:
    g = rng.standard_normal((d, d))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def quadratic_d64(n: int = 65536, seed: int = 0, d: int = 64) -> Problem:
    rng = np.random.default_rng(3000 + seed)
    Q = random_orthogonal(rng, d)
    lam = 10.0 ** (4.0 * np.arange(d) / max(d - 1, 1))
    c = rng.uniform(-5.0, 5.0, size=d).astype(np.float32).astype(np.float64)
    obj = Objective(OBJ_QUADRATIC, d, {"center": c, "Q": Q, "lam": lam})
    lo, hi = np.full(d, -10.0), np.full(d, 10.0)
    # -Hessian = 2 Q^T Lambda Q, largest eigenvalue 2*lam_max.  eps_grad 0.05 lies above the
    # gradient noise that binary32 positions leave near c (2 lam_max ulp(x) ~ 0.02 per coordinate)
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=0.05,
                   sigma_mode=float(1.0 / np.sqrt(2.0 * lam.max())))


def random_cholesky(rng, d, cond_max=100.0) -> np.ndarray:
    while True:
        L = np.tril(rng.normal(0.0, 0.05, size=(d, d)), -1)
        L[np.diag_indices(d)] = np.exp(rng.uniform(np.log(0.3), 0.0, size=d))
        s = np.linalg.svd(L, compute_uv=False)
        if s[0] / s[-1] <= cond_max:
            return L


def mixture256_d64(n: int = 65536, seed: int = 0, K: int = 256, d: int = 64) -> Problem:
    rng = np.random.default_rng(4000 + seed)
    chol = np.stack([random_cholesky(rng, d) for _ in range(K)])
    means = rng.uniform(-20.0, 20.0, size=(K, d))
    obj = Objective(OBJ_MIXTURE_FULL, d, {"weights": np.full(K, 1.0 / K), "means": means, "chol": chol})
    lo, hi = np.full(d, -20.0), np.full(d, 20.0)
    smin = min(float(np.linalg.svd(L, compute_uv=False)[-1]) for L in chol)
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-2, sigma_mode=smin)


def batched512(n_problems: int = 512, seed: int = 0, n_scale: float = 1.0) -> List[Problem]:
    rng = np.random.default_rng(5000 + seed)
    probs = []
    for _ in range(n_problems):
        d = int(rng.choice([2, 4, 8, 16, 32, 64]))
        n = int(np.exp(rng.uniform(np.log(256), np.log(16384))) * n_scale)
        n = max(n, 8)
        K = int(np.floor(np.exp(rng.uniform(np.log(4), np.log(129)))))
        K = min(max(K, 4), 128)
        sig = rng.uniform(0.3, 1.0, size=(K, d))
        means = rng.uniform(-10.0, 10.0, size=(K, d))
        obj = Objective(OBJ_MIXTURE_DIAG, d, {"weights": np.full(K, 1.0 / K), "means": means, "sigmas": sig})
        lo, hi = np.full(d, -10.0), np.full(d, 10.0)
        probs.append(Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-3,
                             sigma_mode=float(sig.min())))
    return probs


def small_mixture(d: int, K: int, n: int, seed: int, box: float = 6.0, noise_sigma: float = 0.0) -> Problem:
    """A small diagonal mixture for parity tests (several tiles and a ragged tail)."""
    rng = np.random.default_rng(6000 + seed)
    sig = np.exp(rng.uniform(np.log(0.4), np.log(1.0), size=(K, d)))
    means = rng.uniform(-0.7 * box, 0.7 * box, size=(K, d))
    e = -np.log(rng.random(K))
    obj = Objective(OBJ_MIXTURE_DIAG, d, {"weights": e / e.sum(), "means": means, "sigmas": sig}, noise_sigma)
    lo, hi = np.full(d, -box), np.full(d, box)
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-3, sigma_mode=float(sig.min()))


def small_quadratic(d: int, n: int, seed: int, cond: float = 1e2) -> Problem:
    rng = np.random.default_rng(7000 + seed)
    Q = random_orthogonal(rng, d)
    lam = cond ** (np.arange(d) / max(d - 1, 1))
    c = rng.uniform(-3.0, 3.0, size=d).astype(np.float32).astype(np.float64)
    obj = Objective(OBJ_QUADRATIC, d, {"center": c, "Q": Q, "lam": lam})
    lo, hi = np.full(d, -8.0), np.full(d, 8.0)
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-2,
                   sigma_mode=float(1.0 / np.sqrt(2.0 * lam.max())))


def small_full_mixture(d: int, K: int, n: int, seed: int, box: float = 8.0) -> Problem:
    rng = np.random.default_rng(8000 + seed)
    chol = np.stack([random_cholesky(rng, d) for _ in range(K)])
    means = rng.uniform(-0.7 * box, 0.7 * box, size=(K, d))
    obj = Objective(OBJ_MIXTURE_FULL, d, {"weights": np.full(K, 1.0 / K), "means": means, "chol": chol})
    lo, hi = np.full(d, -box), np.full(d, box)
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=1e-2, sigma_mode=0.3)


def benchmark_box(name: str, d: int):
    """The domain Theta each benchmark function is stated on in Appendix D."""
    half = {"rastrigin": 5.12, "ackley": 32.768, "schwefel": 500.0, "styblinski_tang": 5.0,
            "trid": float(d * d)}
    if name in half:
        return np.full(d, -half[name]), np.full(d, half[name])
    if name == "michalewicz":
        return np.zeros(d), np.full(d, np.pi)
    if name == "bukin6":
        if d != 2:
            raise ValueError("Bukin N.6 is two-dimensional")
        return np.array([-15.0, -3.0]), np.array([-5.0, 3.0])
    raise KeyError(name)


def benchmark(name: str, d: int = 64, n: int = 65536, seed: int = 0, eps_grad: float = 1e-3) -> Problem:
    """An Appendix D benchmark function on its domain, population uniform in it."""
    rng = np.random.default_rng(9000 + seed)
    lo, hi = benchmark_box(name, d)
    obj = Objective(BENCHMARK_KINDS[name], d, {})
    return Problem(d, n, lo, hi, obj, _uniform_box(rng, n, lo, hi), eps_grad=eps_grad, sigma_mode=1.0)


WORKLOADS = {
    "mixture4_d2": mixture4_d2,
    "mixture32_d16": mixture32_d16,
    "quadratic_d64": quadratic_d64,
    "mixture256_d64": mixture256_d64,
    "mixture2_d6": mixture2_d6,
}
for _name in BENCHMARK_KINDS:
    if _name != "bukin6":
        WORKLOADS[_name + "_d64"] = (lambda nm: (lambda seed=0, n=65536: benchmark(nm, 64, n, seed)))(_name)


