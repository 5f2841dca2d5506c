"""Per-kernel parity of the CUDA path against the FP64 oracle, from identical
state, through the C ABI.  Sizes span several thread blocks and a ragged tail.

Tolerances (binary32 state and arithmetic against an FP64 reference):
  * values and exact gradients: 1e-5 relative (per-sample inf-norm);
  * FD64 gradients (FP64 stencil on both sides, FP32 storage): 1e-6 relative;
  * FD32 gradients: the central-difference rounding bound
    |err_j| <= 64 u32 (|f| + 1) / h_j  (u32 = 2^-24) plus 1e-5 relative;
  * masks and indices: bit-exact, the oracle taking the same binary32 decisions.
"""
import zlib

import numpy as np
import pytest

import gpu_util as U
from oracle import method as M
from oracle import objectives as OB
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PROBS = {
    "mix_d2": lambda n: I.small_mixture(2, 4, n, seed=1),
    "mix_d5": lambda n: I.small_mixture(5, 7, n, seed=2),
    "mix_d16": lambda n: I.small_mixture(16, 32, n, seed=3, box=10.0),
    "mix_d64": lambda n: I.small_mixture(64, 8, n, seed=4),
    "full_d3": lambda n: I.small_full_mixture(3, 5, n, seed=5),
    "full_d33": lambda n: I.small_full_mixture(33, 6, n, seed=6),
    "quad_d7": lambda n: I.small_quadratic(7, n, seed=7),
    "quad_d64": lambda n: I.small_quadratic(64, n, seed=8, cond=1e4),
    # the symmetric block product at every lane count: 1, 4 and 8 lanes per sample
    "quad_d3": lambda n: I.small_quadratic(3, n, seed=9),
    "quad_d12": lambda n: I.small_quadratic(12, n, seed=10, cond=1e3),
    "quad_d27": lambda n: I.small_quadratic(27, n, seed=11, cond=1e3),
}
U32 = 2.0 ** -24


def _torch_x(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def grad_term_scale(prob, X):
    """Per-sample magnitude of the terms the gradient sums, with every
    difference x - mu counted as |x - mu| + |mu| because the device holds the
    centres rounded to binary32: sum_k r_k |P_k| (|x - mu_k| + |mu_k|) for
    mixtures (|P_k| = |L^-T| |L^-1|, diagonal 1/sigma^2), 2 |A| (|x - c| + |c|)
    for the quadratic (inf-norm over coordinates).  A binary32 evaluation of a
    sum has error ~u times this, not times |sum|."""
    obj = prob.objective
    if obj.kind == OB.OBJ_QUADRATIC:
        A = obj.arrays["Q"].T @ np.diag(obj.arrays["lam"]) @ obj.arrays["Q"]
        c = obj.arrays["center"]
        return (2.0 * (np.abs(X - c) + np.abs(c)) @ np.abs(A)).max(axis=1)
    lc, _ = OB._component_logdens(obj, X)
    r = np.exp(lc - OB._lse(lc)[:, None])
    A = obj.arrays
    out = np.zeros(X.shape)
    for k in range(A["weights"].shape[0]):
        mag = np.abs(X - A["means"][k]) + np.abs(A["means"][k])
        if obj.kind == OB.OBJ_MIXTURE_DIAG:
            out += r[:, k:k + 1] * mag / A["sigmas"][k] ** 2
        else:
            Linv = np.abs(np.linalg.inv(A["chol"][k]))
            out += r[:, k:k + 1] * (mag @ (Linv.T @ Linv))
    return out.max(axis=1)


def value_term_scale(prob, X):
    """For the quadratic, the magnitude of the terms its value sums,
    |x - c|^T |A| |x - c| (the centre is binary32-exact): a binary32 evaluation has
    error ~u times this, which near the centre of an ill-conditioned quadratic is far
    above u |f|."""
    obj = prob.objective
    A = obj.arrays["Q"].T @ np.diag(obj.arrays["lam"]) @ obj.arrays["Q"]
    R = np.abs(X - obj.arrays["center"])
    return np.einsum("nd,de,ne->n", R, np.abs(A), R)


def softmax_error_scale(prob, X):
    """For mixtures, sum_k r_k E_k |s_k - g| (inf-norm over coordinates), where
    E_k bounds |delta lc_k| / u32 for a binary32 evaluation of the component's
    log-density: the d-term quadratic form q_k = |z_k|^2 carries an error
    <= (d + 2) u32 (q_k + 2 sum_i |z_i| (|L^-1| |x - mu|)_i), and every error in
    lc_k moves the responsibilities by r_k (delta lc_k - sum_l r_l delta lc_l).
    Zero for the quadratic (no softmax)."""
    obj = prob.objective
    if obj.kind == OB.OBJ_QUADRATIC:
        return np.zeros(X.shape[0])
    A = obj.arrays
    lc, score = OB._component_logdens(obj, X)
    r = np.exp(lc - OB._lse(lc)[:, None])
    g = np.einsum("nk,nkd->nd", r, score)
    R = X[:, None, :] - A["means"][None]
    Rm = np.abs(R) + np.abs(A["means"])[None]          # binary32 centres: |x - mu| + |mu|
    d = X.shape[1]
    if obj.kind == OB.OBJ_MIXTURE_DIAG:
        q = ((R / A["sigmas"][None]) ** 2).sum(axis=2)
        qm = (np.abs(R) * Rm / A["sigmas"][None] ** 2).sum(axis=2)
        E = (d + 2) * (1.5 * q + 2.0 * qm)
    else:
        E = np.empty(lc.shape)
        for k in range(A["weights"].shape[0]):
            Linv = np.linalg.inv(A["chol"][k])
            z = R[:, k, :] @ Linv.T
            mag = Rm[:, k, :] @ np.abs(Linv).T
            E[:, k] = (d + 2) * ((z * z).sum(axis=1) + 2.0 * (np.abs(z) * mag).sum(axis=1))
    E = E + np.abs(lc) + 1.0
    return np.einsum("nk,nkd->nd", r * E, np.abs(score - g[:, None, :])).max(axis=1)


def assert_grad_close(g, g_ref, scale, rtol, cond=None):
    """|g - g_ref|_inf <= rtol * (term magnitude) + u32 * (softmax conditioning)."""
    tol = rtol * scale + (U32 * cond if cond is not None else 0.0)
    err = np.abs(g - g_ref).max(axis=1) / tol
    assert err.max() <= 1.0, (err.max(), np.argmax(err))


@pytest.mark.parametrize("name", sorted(PROBS))
def test_objective_value_and_adjoint(name):
    prob = PROBS[name](1037)
    model = U.open_ctx(prob, M.Params(grad_mode=M.GRAD_ADJOINT))
    x = prob.x0 * np.float32(0.6)
    f, g = model.eval(0, _torch_x(x), CH.GRAD_ADJOINT)
    f, g = f.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    x64 = x.astype(np.float64)
    f_ref, g_ref = OB.value(prob.objective, x64), OB.grad(prob.objective, x64)
    assert np.all(np.abs(f - f_ref) <= 1e-5 * (np.abs(f_ref) + 1.0)), np.abs(f - f_ref).max()
    assert_grad_close(g, g_ref, grad_term_scale(prob, x64), 1e-5, softmax_error_scale(prob, x64))
    model.close()


@pytest.mark.parametrize("name", ["mix_d5", "mix_d64", "full_d33", "quad_d7", "quad_d64"])
def test_autograd_objective(name):
    """ChisaoObjective (the torch.autograd.Function over the device objective; exact
    gradients as the analytic alternative to finite differences, Sec. 3.1): forward is
    the objective value, and torch.autograd.grad of sum_i w_i f(x_i) is w_i times the
    oracle's analytic gradient, element by element within the objective parity bound
    (scaled by |w_i|) plus the rounding of the product; the same through a
    non-contiguous input; and torch.autograd.gradcheck against central differences of
    forward on a small case (binary32: step 1e-3, tolerance 1e-2 plus the rounding of
    the differenced values)."""
    import torch
    prob = PROBS[name](301)
    model = U.open_ctx(prob, M.Params(grad_mode=M.GRAD_ADJOINT))
    x = prob.x0 * np.float32(0.6)
    x64 = x.astype(np.float64)
    w = np.random.default_rng(3).normal(size=prob.n).astype(np.float32)
    f_ref, g_ref = OB.value(prob.objective, x64), OB.grad(prob.objective, x64)
    bound = (np.abs(w).astype(np.float64) * (1e-5 * grad_term_scale(prob, x64) + U32 * softmax_error_scale(prob, x64))
             + U32 * np.abs(w[:, None] * g_ref).max(axis=1))
    wt = torch.from_numpy(w).cuda()
    base = torch.zeros(prob.n, 2 * prob.d, dtype=torch.float32, device="cuda")
    for contiguous in (True, False):
        if contiguous:
            xt = _torch_x(x).requires_grad_(True)
        else:
            base[:, ::2] = _torch_x(x)
            xt = base[:, ::2].detach().requires_grad_(True)      # stride 2 along the coordinates
            assert not xt.is_contiguous()
        f = CH.ChisaoObjective.apply(model, 0, xt)
        assert f.shape == (prob.n,) and f.requires_grad
        fv = f.detach().cpu().numpy().astype(np.float64)
        assert np.all(np.abs(fv - f_ref) <= 1e-5 * (np.abs(f_ref) + 1.0))
        (gx,) = torch.autograd.grad((wt * f).sum(), xt)
        assert gx.shape == xt.shape
        err = np.abs(gx.cpu().numpy().astype(np.float64) - w[:, None] * g_ref).max(axis=1)
        assert np.all(err <= bound), (err / bound).max()
    # central differences of binary32 values carry ~ u |f| / eps of rounding per entry
    small = _torch_x(x[:6]).requires_grad_(True)
    fmax = float(np.abs(f_ref[:6]).max())
    assert torch.autograd.gradcheck(lambda t: CH.ChisaoObjective.apply(model, 0, t), (small,), eps=1e-3,
                                    atol=1e-2 + 8 * U32 * fmax / 1e-3, rtol=1e-2)
    model.close()


@pytest.mark.parametrize("name", ["mix_d2", "mix_d5", "mix_d16", "full_d3", "quad_d7", "quad_d64"])
def test_fd64_gradient(name):
    prob = PROBS[name](517)
    P = M.Params(grad_mode=M.GRAD_FD64, h=1e-5)
    model = U.open_ctx(prob, P)
    x = prob.x0 * np.float32(0.6)
    f, g = model.eval(0, _torch_x(x), CH.GRAD_FD64)
    g = g.cpu().numpy().astype(np.float64)
    g_ref = M.fd_gradient(prob, x.astype(np.float64), P)
    err = U.rel_err_rows(g, g_ref, floor=1e-3 * np.abs(g_ref).max())
    assert err.max() <= 1e-6, err.max()
    model.close()


@pytest.mark.parametrize("name", ["mix_d2", "mix_d16", "quad_d7", "quad_d27"])
def test_fd32_gradient(name):
    prob = PROBS[name](517)
    P = M.Params(grad_mode=M.GRAD_FD32)
    model = U.open_ctx(prob, P)
    x = prob.x0 * np.float32(0.6)
    f, g = model.eval(0, _torch_x(x), CH.GRAD_FD32)
    g = g.cpu().numpy().astype(np.float64)
    x64 = x.astype(np.float64)
    g_ref = M.fd_gradient(prob, x64, P)
    fa = np.abs(OB.value(prob.objective, x64))[:, None]
    hj = P.h_rel * np.maximum(1.0, np.abs(x64))
    tol = 64 * U32 * (fa + 1.0) / hj + 1e-5 * np.abs(g_ref)
    assert np.all(np.abs(g - g_ref) <= tol)
    model.close()


def _random_history(rng, N, d, m, hlen):
    S = np.zeros((N, m, d))
    Y = np.zeros((N, m, d))
    for n in range(N):
        B = rng.standard_normal((d, d)) / np.sqrt(d)
        A = B @ B.T + 0.5 * np.eye(d)
        for k in range(hlen[n]):
            s = rng.standard_normal(d)
            S[n, k] = s
            Y[n, k] = A @ s
    return S, Y


@pytest.mark.parametrize("d,m", [(2, 5), (5, 10), (16, 10), (64, 10)])
def test_lbfgs_direction(d, m):
    rng = np.random.default_rng(d)
    N = 333
    prob = I.small_quadratic(d, N, seed=d)
    P = M.Params(m=m, grad_mode=M.GRAD_ADJOINT)
    model = U.open_ctx(prob, P)
    st = M.new_state(prob.x0, m)
    st.hlen = rng.integers(0, m + 1, size=N)
    st.S, st.Y = _random_history(rng, N, d, m, st.hlen)
    st.g = rng.standard_normal((N, d))
    st = U.rounded(st)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_DIRECTION)
    p_gpu = model.get(0, CH.FIELD_G)[:, :d]
    p_ref = M.lbfgs_direction(-st.g, st.S, st.Y, st.rho, st.hlen)
    err = U.rel_err_rows(p_gpu, p_ref)
    assert err.max() <= 1e-5, err.max()
    model.close()


def _armijo_margin(prob, st, P, Pd, alpha):
    """F(x) + c1 gradF^T (x_t - x) - F(x_t) at x_t = clip(x + alpha p), FP64."""
    Xt = np.clip(st.x + alpha[:, None] * Pd, prob.lo, prob.hi)
    Ft = -OB.value(prob.objective, Xt)
    F = -st.f
    return F + P.c1 * np.einsum("nd,nd->n", -st.g, Xt - st.x) - Ft, np.abs(F) + np.abs(Ft)


@pytest.mark.parametrize("mode", [M.GRAD_ADJOINT, M.GRAD_FD64, M.GRAD_FD32])
@pytest.mark.parametrize("name", ["mix_d5", "mix_d16", "mix_d64", "quad_d7", "quad_d12", "quad_d64", "full_d3"])
def test_lbfgs_iteration(name, mode):
    """One Phase-1 iteration (direction, Armijo search, new gradient, history
    push) from the same binary32 state on both sides."""
    prob = PROBS[name](700)
    P = M.Params(m=6, grad_mode=mode)
    # a realistic mid-run state: a few FP64 iterations, then rounded to binary32
    st = M.new_state(prob.x0, P.m)
    M.lbfgs_iterations(prob, st, M.Params(m=6, grad_mode=M.GRAD_ADJOINT), 3)
    st = U.rounded(st)
    st.f = M.evaluate(prob, st.x)
    st.g = M.gradient(prob, st.x, P)
    st = U.rounded(st)
    model = U.open_ctx(prob, P)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_LBFGS, -1)
    got = U.read_state(model, prob, P.m)
    ref = M.State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.__dict__.items()})
    Pd = M.lbfgs_direction(-st.g, st.S, st.Y, st.rho, st.hlen)
    M.lbfgs_iterations(prob, ref, P, 1, fresh_gradient=False)
    step = np.abs(ref.x - st.x).max(axis=1)
    xerr = np.abs(got.x - ref.x).max(axis=1)
    scale = np.abs(st.x).max(axis=1)
    ok = xerr <= 1e-5 * step + 4e-7 * scale
    # rows that differ must be binary32-vs-FP64 ties of the Armijo test: the
    # step the device took is a power-of-two multiple of the oracle's, and the
    # oracle's margin at the device's step is within rounding of zero
    bad = np.flatnonzero(~ok)
    assert bad.size <= 0.02 * prob.n, (bad.size, xerr[bad][:5], step[bad][:5])
    for i in bad:
        dg = got.x[i] - st.x[i]
        dr = ref.x[i] - st.x[i]
        j = np.argmax(np.abs(dr))
        ratio = dg[j] / dr[j] if dr[j] != 0 else np.inf
        assert np.isfinite(ratio) and abs(np.log2(abs(ratio)) - round(np.log2(abs(ratio)))) < 1e-3
    # the new gradient, compared at the point the device reached
    xg = got.x
    if mode == M.GRAD_ADJOINT:
        assert_grad_close(got.g, OB.grad(prob.objective, xg), grad_term_scale(prob, xg), 1e-5,
                          softmax_error_scale(prob, xg))
    elif mode == M.GRAD_FD64:
        assert_grad_close(got.g, M.fd_gradient(prob, xg, P), grad_term_scale(prob, xg), 1e-5)
    else:
        fa = np.abs(OB.value(prob.objective, xg))[:, None]
        tol = 64 * U32 * (fa + 1.0) / (P.h_rel * np.maximum(1.0, np.abs(xg))) + 1e-5 * grad_term_scale(prob, xg)[:, None]
        assert np.all(np.abs(got.g - M.fd_gradient(prob, xg, P)) <= tol)
    assert np.all(got.hlen[ok] == ref.hlen[ok])
    live = ok & (ref.hlen > 0)
    serr = U.rel_err_rows(got.S[live, 0], ref.S[live, 0])
    assert np.quantile(serr, 0.99) <= 1e-4
    # s^T y of the new pair, from the device's own binary32 s and y: exact
    # products summed in double-single must round to the FP64 value
    lg = got.hlen > 0
    sy = np.einsum("nd,nd->n", got.S[lg, 0], got.Y[lg, 0])
    np.testing.assert_allclose(got.rho[lg, 0], 1.0 / sy, rtol=3 * U32)
    model.close()


# ----------------------------------------------------------------------- Phase 2

def test_freeze_mask_bit_exact():
    rng = np.random.default_rng(5)
    N, d = 4133, 5
    prob = I.small_mixture(d, 3, N, seed=9)
    P = M.Params(eps_grad=1e-3, delta=0.1)
    model = U.open_ctx(prob, P)
    f = rng.normal(-3.0, 1.5, N).astype(np.float32)
    f[7] = 2.0                                           # f_max
    thr = np.float32(np.float32(2.0) + np.float32(np.log(0.1)))
    f[100:140] = thr                                     # exactly at the threshold
    f[140:180] = np.nextafter(thr, np.float32(-10))
    g = rng.uniform(-2e-3, 2e-3, (N, d)).astype(np.float32)
    g[200:260, 1] = np.float32(1e-3)                    # exactly eps: not < eps
    g[260:300, 2] = np.nextafter(np.float32(1e-3), np.float32(0))
    g[300, 0] = np.nan
    f[301] = np.nan
    st = M.new_state(prob.x0, P.m)
    st.f, st.g = f.astype(np.float64), g.astype(np.float64)
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_FREEZE)
    got = CH.unpack_bits(model.get(0, CH.FIELD_STUCK), N)
    ref, fmax = M.freeze(f, g, P.eps_grad, P.delta, dtype=np.float32)
    np.testing.assert_array_equal(got, ref)
    assert model.counters(0)["f_max"] == np.float32(fmax)
    model.close()


# ----------------------------------------------------------------------- Phase 3

@pytest.mark.parametrize("d", [2, 7, 64])
def test_dedup_bit_exact(d):
    rng = np.random.default_rng(d)
    N = 3001
    prob = I.small_mixture(d, 3, N, seed=10)
    P = M.Params(eps_dup=1e-3)
    model = U.open_ctx(prob, P)
    centers = rng.uniform(-3, 3, (12, d))
    x = centers[rng.integers(0, 12, N)] + rng.uniform(-1.2e-3, 1.2e-3, (N, d))
    x = x.astype(np.float32)
    f = np.round(rng.normal(0, 1, N), 1).astype(np.float32)   # many ties
    stuck = rng.random(N) < 0.7
    st = M.new_state(x, P.m)
    st.f = f.astype(np.float64)
    st.stuck = stuck
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_DEDUP)
    rem = CH.unpack_bits(model.get(0, CH.FIELD_REMOVED), N)
    stuck_after = CH.unpack_bits(model.get(0, CH.FIELD_STUCK), N)
    ref = M.dedup(x, f, stuck, P.eps_dup, dtype=np.float32)
    np.testing.assert_array_equal(rem, ref)
    np.testing.assert_array_equal(stuck_after, stuck & ~ref)
    assert model.counters(0)["k_lost"] == ref.sum()
    model.close()


@pytest.mark.parametrize("case", ["one_axis", "two_axes", "flat_axes", "boundaries"])
def test_dedup_hash_geometry(case):
    """Candidate generation by spatial hashing on the most-spread coordinates:
    the same mask as the pairwise definition when fewer than three coordinates
    vary, when the stuck set is constant along most axes, and for pairs that
    straddle cell boundaries by less than eps in every coordinate."""
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    d = {"one_axis": 1, "two_axes": 2, "flat_axes": 6, "boundaries": 4}[case]
    N = 2049
    prob = I.small_mixture(d, 2, N, seed=12)
    P = M.Params(eps_dup=1e-3)
    model = U.open_ctx(prob, P)
    if case == "boundaries":
        base = rng.uniform(-2, 2, (N // 2 + 1, d))
        # partners within eps along every coordinate (|offset| from 0.5 eps to just under eps), or just over
        off = rng.choice([-1.0, 1.0], (N // 2 + 1, d)) * rng.uniform(0.5e-3, 0.999e-3, (N // 2 + 1, d))
        off[::3, 0] = 1.001e-3
        x = np.concatenate([base, base + off])[:N]
    else:
        x = np.tile(rng.uniform(-3, 3, (1, d)), (N, 1))
        vary = {"one_axis": [0], "two_axes": [0, 1], "flat_axes": [4]}[case]
        for a in vary:
            x[:, a] = rng.uniform(-3, 3, 40)[rng.integers(0, 40, N)] + rng.uniform(-1.5e-3, 1.5e-3, N)
    x = x.astype(np.float32)
    f = np.round(rng.normal(0, 1, N), 1).astype(np.float32)
    stuck = rng.random(N) < 0.8
    st = M.new_state(x, P.m)
    st.f = f.astype(np.float64)
    st.stuck = stuck
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_DEDUP)
    rem = CH.unpack_bits(model.get(0, CH.FIELD_REMOVED), N)
    ref = M.dedup(x, f, stuck, P.eps_dup, dtype=np.float32)
    assert ref.sum() > 0 and (stuck & ~ref).sum() > 1
    np.testing.assert_array_equal(rem, ref)
    model.close()


@pytest.mark.parametrize("d,N", [(2, 1 << 20), (16, 1 << 18)])
def test_dedup_dense_cluster(d, N):
    """Every stuck sample converged into one cluster (offsets below eps/2 in every
    coordinate, f nearly tied): only the top-ranked sample (highest f, then lowest
    index) survives.  The cluster's top decides each member in one test, so this
    runs in a single short pass rather than a scan of the cluster per sample."""
    rng = np.random.default_rng(d)
    prob = I.small_mixture(d, 2, N, seed=13)
    P = M.Params(eps_dup=1e-3)
    model = U.open_ctx(prob, P)
    x = (rng.uniform(-1, 1, (1, d)) + rng.uniform(-4.9e-4, 4.9e-4, (N, d))).astype(np.float32)
    f = (-1.0 + np.round(rng.normal(0, 1e-6, N), 7)).astype(np.float32)      # many exact ties
    dp, mm = model.layout(0)
    xp = np.zeros((N, dp), np.float32)
    xp[:, :d] = x
    model.set(0, CH.FIELD_X, xp)
    model.set(0, CH.FIELD_F, f)
    model.set(0, CH.FIELD_STUCK, CH.pack_bits(np.ones(N, bool)))
    model.set(0, CH.FIELD_REMOVED, CH.pack_bits(np.zeros(N, bool)))
    model.run_phase(0, CH.PHASE_DEDUP)
    rem = CH.unpack_bits(model.get(0, CH.FIELD_REMOVED), N)
    top = np.lexsort((np.arange(N), -f.astype(np.float64)))[0]             # f desc, index asc
    assert (~rem).sum() == 1 and not rem[top]
    model.close()


def test_dedup_edge_cases():
    prob = I.small_mixture(3, 2, 33, seed=11)
    P = M.Params(eps_dup=1e-3)
    model = U.open_ctx(prob, P)
    x = np.zeros((33, 3), np.float32)
    st = M.new_state(x, P.m)
    st.f = np.zeros(33)
    for stuck in (np.zeros(33, bool), np.ones(33, bool)):     # nothing stuck / all identical and tied
        st.stuck = stuck
        U.write_state(model, prob, st)
        model.run_phase(0, CH.PHASE_DEDUP)
        rem = CH.unpack_bits(model.get(0, CH.FIELD_REMOVED), 33)
        np.testing.assert_array_equal(rem, M.dedup(x, st.f.astype(np.float32), stuck, 1e-3, np.float32))
    assert rem.sum() == 32 and not rem[0]
    model.close()


@pytest.mark.parametrize("sigma", [0.1, 1.0])
def test_noisy_objective(sigma):
    """Values carry sigma * N(0,1) keyed by the point (same draw as the oracle's);
    FD64 differences of the noisy values match the oracle's to binary32 noise
    rounding; the adjoint gradient is the noise-free one."""
    prob = I.small_mixture(16, 8, 700, seed=15, box=8.0, noise_sigma=sigma)
    P = M.Params(grad_mode=M.GRAD_FD64, seed=77)
    model = U.open_ctx(prob, P)
    x = prob.x0 * np.float32(0.6)
    x64 = x.astype(np.float64)
    f, g = model.eval(0, _torch_x(x), CH.GRAD_FD64)
    f_ref = M.evaluate(prob, x64, seed=77)
    assert np.all(np.abs(f.cpu().numpy() - f_ref) <= 1e-5 * (np.abs(f_ref) + 1.0) + 1e-6 * sigma)
    g_ref = M.fd_gradient(prob, x64, P)
    err = np.abs(g.cpu().numpy() - g_ref).max(axis=1) / (np.abs(g_ref).max(axis=1) + 1.0)
    assert err.max() <= 1e-5
    fa, ga = model.eval(0, _torch_x(x), CH.GRAD_ADJOINT)
    assert_grad_close(ga.cpu().numpy(), OB.grad(prob.objective, x64), grad_term_scale(prob, x64), 1e-5,
                      softmax_error_scale(prob, x64))
    model.close()


def tc_error_bounds(tco, Xs):
    """Absolute error bounds of the tensor-core evaluation of f and grad f at the
    split inputs Xs, against the FP64 evaluation of the same rounded objective:
    z = W x' - W mu accumulates in FP32 the 128 exact BF16 products and the three
    BF16 terms of the binary32 -W mu (|dz| <= 134 u (|W||x'| + |W||mu|)); q, lc,
    f follow; the gradient
    adds the BF16 rounding of y = r z (2^-9 relative), the FP32 accumulation of
    K d products, and the responsibilities' sensitivity to the lc errors."""
    A = tco.arrays
    W, mu = A["linv"], A["means"]
    K, d = mu.shape
    Wa = np.abs(W)
    R = Xs[:, None, :] - mu[None]
    Z = np.einsum("kij,nkj->nki", W, R)
    lc, score = OB._component_logdens(tco, Xs)
    r = np.exp(lc - OB._lse(lc)[:, None])
    f = OB._lse(lc)
    dz = 134 * U32 * (np.einsum("kij,nj->nki", Wa, np.abs(Xs)) + np.einsum("kij,kj->ki", Wa, np.abs(mu))[None])
    q = (Z * Z).sum(axis=2)
    E = (np.abs(Z) * dz).sum(axis=2) + 0.5 * (d + 2) * U32 * q + U32 * (np.abs(lc) + 1.0)
    tol_f = (r * E).sum(axis=1) + 4 * U32 * (np.abs(f) + 1.0)
    Wz = np.einsum("kji,nkj->nki", Wa, np.abs(Z))
    Wdz = np.einsum("kji,nkj->nki", Wa, dz)
    g = np.einsum("nk,nkd->nd", r, score)
    tol_g = (np.einsum("nk,nkd->nd", r, (2.0 ** -8 + 4 * K * d * U32) * Wz + Wdz)
             + np.einsum("nk,nkd->nd", r * E, np.abs(score - g[:, None, :])))
    return tol_f, tol_g


@pytest.mark.parametrize("which", ["k256_d64", "k6_d33"])
def test_tensor_core_mixture_objective(which):
    """tcgen05 BF16 evaluation (value and adjoint gradient) of the full-covariance
    mixture = the FP64 value and gradient of the mixture with BF16-rounded
    precision factors at the BF16-split input, within FP32 accumulation and the
    BF16 rounding of the gradient weights; far from and near the modes."""
    prob = (I.mixture256_d64(n=1031) if which == "k256_d64" else I.small_full_mixture(33, 6, 1031, seed=16))
    model = U.open_ctx(prob, M.Params(grad_mode=M.GRAD_ADJOINT))
    rng = np.random.default_rng(11)
    mu = prob.objective.arrays["means"]
    near = (mu[rng.integers(0, mu.shape[0], 500)] + rng.normal(0, 0.05, (500, prob.d))).astype(np.float32)
    x = np.concatenate([prob.x0[:531] * np.float32(0.7), near]).astype(np.float32)
    f, g = model.eval(0, _torch_x(x), CH.GRAD_ADJOINT_TC)
    f, g = f.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    assert model.counters(0) is not None
    tco = OB.tensor_core_objective(prob.objective)          # evaluated at the BF16-split input
    Xs = OB.bf16_split(x)
    f_ref, g_ref = OB.value(tco, x.astype(np.float64)), OB.grad(tco, x.astype(np.float64))
    tol_f, tol_g = tc_error_bounds(tco, Xs)
    assert np.all(np.abs(f - f_ref) <= tol_f), (np.abs(f - f_ref) / tol_f).max()
    assert np.all(np.abs(g - g_ref) <= tol_g), (np.abs(g - g_ref) / tol_g).max()
    # value-only launch agrees with the value of the value+gradient launch
    fv, _ = model.eval(0, _torch_x(x), CH.GRAD_ADJOINT_TC, want_grad=False)
    np.testing.assert_array_equal(fv.cpu().numpy(), f.astype(np.float32))
    model.close()


def _tc_split(tiles, ngroups, grid, nsm, split_max=16, units_max=256):
    """The component split the tensor-core kernel chooses for a launch of `tiles`
    128-point tiles: as many CTAs per tile as still fit one wave (none past it)."""
    sp = min(nsm // tiles, grid // tiles, units_max // tiles, ngroups, split_max)
    return sp if sp >= 2 else 1


def test_tensor_core_component_split():
    """A tile's component groups divided among several CTAs and merged (a launch of a few
    tiles) gives the objective within the same bounds as whole tiles (a launch of one tile
    per multiprocessor): both against the FP64 evaluation of the rounded objective, and
    against each other within the sum of their bounds."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    n_big = 128 * nsm
    prob = I.mixture256_d64(n=n_big)
    ng = (prob.objective.arrays["means"].shape[0] + 1) // 2
    assert _tc_split(nsm, ng, 1 << 30, nsm) == 1
    assert _tc_split(8, ng, 1 << 30, nsm) > 1
    model = U.open_ctx(prob, M.Params(grad_mode=M.GRAD_ADJOINT))
    rng = np.random.default_rng(12)
    mu = prob.objective.arrays["means"]
    x = (prob.x0 * np.float32(0.7)).astype(np.float32)
    sel = rng.choice(n_big, 1000, replace=False)
    x[sel[:500]] = (mu[rng.integers(0, mu.shape[0], 500)] + rng.normal(0, 0.05, (500, prob.d))).astype(np.float32)
    f1, g1 = model.eval(0, _torch_x(x), CH.GRAD_ADJOINT_TC)          # whole tiles
    xs = x[sel]
    f2, g2 = model.eval(0, _torch_x(xs), CH.GRAD_ADJOINT_TC)         # 8 tiles, split
    f1 = f1.cpu().numpy().astype(np.float64)[sel]
    g1 = g1.cpu().numpy().astype(np.float64)[sel]
    f2, g2 = f2.cpu().numpy().astype(np.float64), g2.cpu().numpy().astype(np.float64)
    tco = OB.tensor_core_objective(prob.objective)
    f_ref, g_ref = OB.value(tco, xs.astype(np.float64)), OB.grad(tco, xs.astype(np.float64))
    tol_f, tol_g = tc_error_bounds(tco, OB.bf16_split(xs))
    for f, g in ((f1, g1), (f2, g2)):
        assert np.all(np.abs(f - f_ref) <= tol_f), (np.abs(f - f_ref) / tol_f).max()
        assert np.all(np.abs(g - g_ref) <= tol_g), (np.abs(g - g_ref) / tol_g).max()
    assert np.all(np.abs(f1 - f2) <= 2 * tol_f) and np.all(np.abs(g1 - g2) <= 2 * tol_g)
    fv, _ = model.eval(0, _torch_x(xs), CH.GRAD_ADJOINT_TC, want_grad=False)
    np.testing.assert_array_equal(fv.cpu().numpy(), f2.astype(np.float32))
    model.close()


def test_mma_rate_measurement():
    """The tensor core's rate for the objective's MMA shape (M = 128, K = 16): one issuer
    is slower per MMA than four together, and every figure is a plausible clock count."""
    one = CH.measure_mma_rate(64, 1, 0)
    four = CH.measure_mma_rate(64, 4, 2)
    assert 8.0 < four < one < 2000.0, (one, four)
