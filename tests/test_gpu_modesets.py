"""Mode sets against the oracle on all five workloads (Algorithm 1's return value).

The CUDA path and the FP64 oracle run the same inputs, Philox seed and parameters
-- a slice of the rows, or a fixed random choice of problems, where the full size
is too slow for the oracle -- and the two returned sets are compared both ways:
every oracle mode within 1e-3 of its local sigma of some GPU mode, and every GPU
mode within 1e-3 local sigma of some oracle mode.  The local sigma is the
Mahalanobis distance under -Hess f at the oracle's point (the recovery metric of
the significant modes, Eq. 1).  Each case also scores both sets against the
significant modes (Newton from every component mean, FP64) and prints a MODESET
line (run with -s): set sizes, both-way matches, worst errors, recovery fractions.

The two sides follow different roundings (binary32 against FP64), so a sample that
sits on a decision boundary (an Armijo tie, |grad f| at eps_grad) can take another
branch, and the reseeding after it then draws other children: the trajectories
need not stay identical, but the sets of modes they return must.
"""
import numpy as np
import pytest

import gpu_util as U
from oracle import method as M
from oracle import modes as MD
from oracle import objectives as OB
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _local_metric(prob, x):
    """-Hess f at x, with negative curvature clipped (a returned point need not be a
    strict maximum of every direction to rounding)."""
    H = -OB.hessian(prob.objective, x)
    w, V = np.linalg.eigh(0.5 * (H + H.T))
    return (V * np.maximum(w, 0.0)) @ V.T


def _dist(a, b, H):
    r = a - b
    return float(np.sqrt(max(r @ H @ r, 0.0)))


def compare_sets(prob, xo, xg, rel=1e-3):
    """(oracle modes matched by a GPU mode, GPU modes matched by an oracle mode, worst
    matched distances both ways, recovery fraction of each side)."""
    xo = np.asarray(xo, np.float64).reshape(-1, prob.d)
    xg = np.asarray(xg, np.float64).reshape(-1, prob.d)
    Hs = [_local_metric(prob, a) for a in xo]
    D = np.array([[_dist(a, b, H) for b in xg] for a, H in zip(xo, Hs)]).reshape(xo.shape[0], xg.shape[0])
    o_hit = D.min(axis=1) <= rel if xg.shape[0] else np.zeros(xo.shape[0], bool)
    g_hit = D.min(axis=0) <= rel if xo.shape[0] else np.zeros(xg.shape[0], bool)
    mx, _, negH = MD.significant_modes(prob)
    fo, wo, _ = MD.recovery(xo, mx, negH)
    fg, wg, _ = MD.recovery(xg, mx, negH)
    worst_o = float(D.min(axis=1)[o_hit].max()) if o_hit.any() else 0.0
    worst_g = float(D.min(axis=0)[g_hit].max()) if g_hit.any() else 0.0
    return {"n_oracle": xo.shape[0], "n_gpu": xg.shape[0], "oracle_matched": int(o_hit.sum()),
            "gpu_matched": int(g_hit.sum()), "worst_oracle_to_gpu": worst_o, "worst_gpu_to_oracle": worst_g,
            "recovery_oracle": fo, "recovery_gpu": fg, "significant": int(mx.shape[0]),
            "worst_recovery_gpu": wg}


def _report(name, r):
    print(f"\nMODESET {name}: oracle {r['n_oracle']} gpu {r['n_gpu']} | oracle->gpu {r['oracle_matched']}/"
          f"{r['n_oracle']} (worst {r['worst_oracle_to_gpu']:.2e}) gpu->oracle {r['gpu_matched']}/{r['n_gpu']} "
          f"(worst {r['worst_gpu_to_oracle']:.2e}) | significant {r['significant']} recovered oracle "
          f"{r['recovery_oracle']:.3f} gpu {r['recovery_gpu']:.3f}")


def _gpu_modes(probs, P, **over):
    model = CH.Chisao(probs, U.lib_params(P, **over))
    for _ in range(P.n_osc):
        model.step()
    out = [model.modes(q)[0] for q in range(len(probs))]
    model.close()
    return out


def _assert_same_set(r):
    assert r["oracle_matched"] == r["n_oracle"] and r["gpu_matched"] == r["n_gpu"], r
    assert r["recovery_gpu"] == r["recovery_oracle"], r


def test_modeset_mixture4_d2():
    """d = 2, K = 4, N = 1024, FD64 at h = 1e-5, m = 5, 50 cycles (the plain method)."""
    U.ensure_built()
    prob = I.mixture4_d2()
    P = M.Params(n_osc=50, m=5, eps_grad=1e-5, grad_mode=M.GRAD_FD64, seed=0)
    (xg,) = _gpu_modes([prob], P)
    (xo, _), _ = M.run(prob, P)
    r = compare_sets(prob, xo, xg)
    _report("mixture4_d2 FD64 50 cycles", r)
    _assert_same_set(r)
    assert r["recovery_gpu"] == 1.0


def test_modeset_mixture32_d16():
    """d = 16, K = 32, the first 4096 samples of the workload, exact gradients,
    n_conv = 40, 4 cycles."""
    U.ensure_built()
    prob = I.mixture32_d16(n=4096)
    P = M.Params(n_osc=4, n_conv=40, m=10, eps_grad=1e-4, grad_mode=M.GRAD_ADJOINT, seed=2)
    (xg,) = _gpu_modes([prob], P)
    (xo, _), _ = M.run(prob, P)
    r = compare_sets(prob, xo, xg)
    _report("mixture32_d16 N 4096 n_conv 40 4 cycles", r)
    _assert_same_set(r)


def test_modeset_quadratic_d64():
    """d = 64 rotated quadratic (condition 1e4), rows 0..511 of the workload, one cycle
    of n_conv = 2500 (enough for Prop. 1)."""
    U.ensure_built()
    full = I.quadratic_d64()
    prob = I.Problem(64, 512, full.lo, full.hi, full.objective, full.x0[:512], full.eps_grad, full.sigma_mode)
    P = M.Params(n_osc=1, n_conv=2500, m=10, eps_grad=1e-2, grad_mode=M.GRAD_ADJOINT, seed=3)
    (xg,) = _gpu_modes([prob], P)
    (xo, _), _ = M.run(prob, P)
    r = compare_sets(prob, xo, xg)
    _report("quadratic_d64 512 rows n_conv 2500", r)
    _assert_same_set(r)
    assert r["recovery_gpu"] == 1.0


def test_modeset_mixture256_d64_fp32():
    """d = 64, K = 256 full covariance, the first 512 samples of the workload, the FP32
    adjoint path (exact objective), n_conv = 100, 2 cycles."""
    U.ensure_built()
    prob = I.mixture256_d64(n=512)
    P = M.Params(n_osc=2, n_conv=100, m=10, eps_grad=1e-2, grad_mode=M.GRAD_ADJOINT, seed=4)
    (xg,) = _gpu_modes([prob], P)
    (xo, _), _ = M.run(prob, P)
    r = compare_sets(prob, xo, xg)
    _report("mixture256_d64 512 rows FP32 adjoint", r)
    _assert_same_set(r)


def test_modeset_mixture256_d64_tensor_cores():
    """The same rows and schedule on the BF16 tensor-core objective (oracle: the same
    BF16-rounded mixture at the split input, in FP64), then the final FP32 refinement on
    the exact objective (oracle: the same iterations in FP64).  The device's gradient
    weights are rounded to BF16 (relative error up to 2^-8, the bound of the objective's
    parity test) where the oracle's are exact, so over 100 L-BFGS iterations a sample can
    end in another local maximum on one side than on the other: every mode the device
    returns must be one the oracle returns, the oracle's set may hold a few more (at
    least 70 % of it matched), and both recover the same significant modes."""
    U.ensure_built()
    prob = I.mixture256_d64(n=512)
    tprob = I.Problem(prob.d, prob.n, prob.lo, prob.hi, OB.tensor_core_objective(prob.objective), prob.x0,
                      prob.eps_grad, prob.sigma_mode)
    P = M.Params(n_osc=2, n_conv=100, m=10, eps_grad=1e-2, grad_mode=M.GRAD_ADJOINT, seed=4)
    (xg,) = _gpu_modes([prob], P, grad_mode=CH.GRAD_ADJOINT_TC, n_refine=10)
    st = M.new_state(tprob.x0, P.m)
    for _ in range(P.n_osc):
        M.cycle(tprob, st, P)
    M.refine(prob, st, P, 10)
    xo, _ = M.modes_of(st)
    r = compare_sets(prob, xo, xg)
    _report("mixture256_d64 512 rows tensor cores + refinement", r)
    assert r["gpu_matched"] == r["n_gpu"] and r["oracle_matched"] >= 0.7 * r["n_oracle"], r
    assert r["recovery_gpu"] == r["recovery_oracle"], r


def test_modeset_batched_problems():
    """16 problems of the 512-problem workload (a fixed random choice), in one context
    with the same problem indices on both sides, exact gradients, 3 cycles."""
    U.ensure_built()
    allp = I.batched512()
    pick = np.sort(np.random.default_rng(0).choice(len(allp), 16, replace=False))
    probs = [allp[i] for i in pick]
    P = M.Params(n_osc=3, m=10, eps_grad=1e-4, grad_mode=M.GRAD_ADJOINT, seed=5)
    outs = _gpu_modes(probs, P)
    tot = {"n_oracle": 0, "n_gpu": 0, "oracle_matched": 0, "gpu_matched": 0}
    rec_o, rec_g, worst = [], [], 0.0
    for q, (prob, xg) in enumerate(zip(probs, outs)):
        st = M.new_state(prob.x0, P.m)
        for _ in range(P.n_osc):
            M.cycle(prob, st, P, prob_index=q)
        xo, _ = M.modes_of(st)
        r = compare_sets(prob, xo, xg)
        for k in tot:
            tot[k] += r[k]
        rec_o.append(r["recovery_oracle"])
        rec_g.append(r["recovery_gpu"])
        worst = max(worst, r["worst_oracle_to_gpu"], r["worst_gpu_to_oracle"])
        print(f"\n  problem {pick[q]} d {prob.d} N {prob.n} K {prob.objective.n_comp}: oracle {r['n_oracle']} "
              f"gpu {r['n_gpu']} matched {r['oracle_matched']}/{r['gpu_matched']} recovery "
              f"{r['recovery_oracle']:.3f}/{r['recovery_gpu']:.3f}")
    print(f"\nMODESET batched (16 problems): oracle {tot['n_oracle']} gpu {tot['n_gpu']} | oracle->gpu "
          f"{tot['oracle_matched']} gpu->oracle {tot['gpu_matched']} worst {worst:.2e} | mean recovery oracle "
          f"{np.mean(rec_o):.3f} gpu {np.mean(rec_g):.3f}")
    # binary32 against FP64 decisions at a threshold (|grad f| at eps_grad, an Armijo tie)
    # can send one sample down another branch and change the reseeding after it
    assert tot["oracle_matched"] >= 0.99 * tot["n_oracle"] and tot["gpu_matched"] >= 0.99 * tot["n_gpu"], tot
    assert abs(np.mean(rec_o) - np.mean(rec_g)) <= 0.01
