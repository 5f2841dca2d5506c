"""End-to-end parity of whole oscillation cycles (Algorithm 1) through the C ABI:
recovered mode sets against the ground-truth modes of Eq. 1 (Newton from every
mean) and against the oracle's own run, plus properties that hold at the full
workload sizes in the launch configuration the benchmark times."""
import numpy as np
import pytest

import gpu_util as U
from oracle import method as M
from oracle import modes as MD
from oracle import objectives as OB
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(model, n):
    for _ in range(n):
        model.step()
    return model.modes(0)


def test_mixture4_d2_plain_method_recovers_all_modes():
    """d=2, 4 isotropic components, N=1024, central FD at h=1e-5 (FP64
    stencil), m=5, 50 cycles, Philox seed 0: all four modes, no spurious."""
    prob = I.mixture4_d2()
    P = M.Params(n_osc=50, m=5, M=8, eps_grad=1e-5, grad_mode=M.GRAD_FD64, seed=0)
    model = U.open_ctx(prob, P)
    fx, ff = _run(model, P.n_osc)
    mx, mf, negH = MD.significant_modes(prob)
    frac, worst, _ = MD.recovery(fx, mx, negH)
    assert frac == 1.0 and worst <= 1e-3
    assert fx.shape[0] == 4
    with pytest.raises(CH.ChisaoError):
        model.step()                                   # all n_osc cycles ran
    # the oracle's own 50-cycle run: test_gpu_modesets.test_modeset_mixture4_d2
    model.close()


def test_mixture_d16_modes_are_true_modes():
    """d = 16, K = 32, the first 4096 samples, 6 cycles at the Table 1 schedule: every
    returned point is one of the significant modes (no spurious mode).  The set against
    the oracle's own run: test_gpu_modesets.test_modeset_mixture32_d16."""
    prob = I.mixture32_d16(n=4096)
    P = M.Params(n_osc=6, m=10, eps_grad=1e-4, grad_mode=M.GRAD_ADJOINT, seed=1)
    model = U.open_ctx(prob, P)
    fx, ff = _run(model, P.n_osc)
    mx, mf, negH = MD.significant_modes(prob)
    frac, worst, best = MD.recovery(fx, mx, negH)
    for x in fx:
        e = min(MD.mahalanobis(x[None], m, H)[0] for m, H in zip(mx, negH))
        assert e <= 1e-3
    assert frac > 0
    model.close()


def test_quadratic_proposition1_with_sufficient_iterations():
    """Proposition 1 / Remark 1 on the d=64 rotated quadratic (Lambda 1..1e4):
    with enough L-BFGS steps one cycle sticks samples at c and dedup leaves one."""
    prob = I.quadratic_d64(n=2048)
    P = M.Params(n_osc=1, n_conv=2500, m=10, eps_grad=0.05, grad_mode=M.GRAD_ADJOINT, seed=3)
    model = U.open_ctx(prob, P)
    fx, ff = _run(model, 1)
    c = prob.objective.arrays["center"]
    mx, mf, negH = MD.significant_modes(prob)
    assert fx.shape[0] == 1
    assert MD.mahalanobis(fx, c, negH[0])[0] <= 1e-3
    model.close()


def _local_mode_errors(prob, fx):
    """Each returned point's Mahalanobis distance to the local maximum that
    Newton's method reaches from it (inf when that point is not a maximum).
    Eq. 3 gates on the population's own f_max, so a returned point is a local
    maximum; it is a significant mode of Eq. 1 once the global one is found."""
    out = []
    for x in fx:
        xs, _ = MD.newton_max(prob.objective, x.astype(np.float64))
        H = -OB.hessian(prob.objective, xs)
        ok = np.linalg.eigvalsh(H).min() > 0
        out.append(MD.mahalanobis(x[None].astype(np.float64), xs, H)[0] if ok else np.inf)
    return np.array(out)


def test_full_covariance_mixture_d64_fp32_modes():
    """d=64, K=256 full-covariance mixture (Cholesky factors with cond <= 100,
    means in [-20, 20]^64) on the FP32 path with a sufficient n_conv (samples
    start ~100 units from any component): every returned point is a local
    maximum to 1e-3 local sigmas.  (The highest peaks belong to the narrowest
    components, whose basins are the smallest seen from uniform starts, so the
    global one is not guaranteed at this population size.)"""
    prob = I.mixture256_d64(n=8192)
    P = M.Params(n_osc=2, n_conv=100, m=10, eps_grad=1e-2, grad_mode=M.GRAD_ADJOINT, seed=4)
    model = U.open_ctx(prob, P)
    fx, ff = _run(model, P.n_osc)
    assert fx.shape[0] >= 3
    assert np.all(_local_mode_errors(prob, fx) <= 1e-3)
    model.close()


def test_batched_problems_in_one_context():
    """Independent problems of uneven (d, N, K) in one context: each one's
    returned points are local maxima of its own objective, and the significant
    modes (Eq. 1) are recovered on average."""
    probs = I.batched512(n_problems=10, n_scale=0.3)
    # |g|_inf < eps bounds the local-sigma error by ~sqrt(d) eps / sqrt(lambda_min): 1e-4 keeps it < 1e-3
    P = M.Params(n_osc=3, m=10, eps_grad=1e-4, grad_mode=M.GRAD_ADJOINT, seed=5)
    U.ensure_built()
    model = CH.Chisao(probs, U.lib_params(P))
    for _ in range(P.n_osc):
        model.step()
    fracs = []
    for q, prob in enumerate(probs):
        fx, ff = model.modes(q)
        if fx.shape[0]:
            assert np.all(_local_mode_errors(prob, fx) <= 1e-3), q
        mx, mf, negH = MD.significant_modes(prob)
        fracs.append(MD.recovery(fx, mx, negH)[0])
        assert model.counters(q)["cycles"] == P.n_osc
    assert np.mean(fracs) > 0.3, fracs
    model.close()


def _mixed_kinds():
    return [I.small_quadratic(7, 900, seed=1), I.small_mixture(5, 4, 700, seed=2),
            I.benchmark("rastrigin", 4, 600, seed=3), I.small_full_mixture(3, 3, 500, seed=4),
            I.small_mixture(6, 3, 300, seed=5), I.small_quadratic(8, 200, seed=6)]


@pytest.mark.parametrize("case", ["batched", "mixed_kinds"])
def test_batched_problems_match_separate_contexts(case):
    """Problems of one context are independent: with exact gradients the context runs
    Phases 1, 5 and 6 as one grouped launch per (objective kind, padded dimension) and
    the objective-independent steps as one launch per kernel over all problems.  Problem
    q's state after two cycles is
    bit-identical in a context of six problems and in one of the first q + 1 (same
    problem index, hence the same Philox streams; a single problem runs ungrouped),
    with and without graph capture."""
    import torch
    probs = I.batched512(n_problems=6, n_scale=0.1, seed=3) if case == "batched" else _mixed_kinds()
    P = M.Params(n_osc=4, m=6, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=2)
    junk = torch.full((64 << 20,), float("nan"), device="cuda")   # arenas below start dirty
    del junk
    U.ensure_built()
    fields = (CH.FIELD_X, CH.FIELD_F, CH.FIELD_STUCK)
    for use_graph in (1, 0):
        prm = U.lib_params(P)
        prm.use_graph = use_graph
        together = CH.Chisao(probs, prm)
        for _ in range(2):
            together.step()
        for q in range(len(probs)):
            part = CH.Chisao(probs[:q + 1], prm)
            for _ in range(2):
                part.step()
            for fld in fields:
                np.testing.assert_array_equal(part.get(q, fld), together.get(q, fld))
            part.close()
        together.close()


def test_determinism_and_graph_equivalence():
    prob = I.small_mixture(5, 6, 3000, seed=20)
    P = M.Params(n_osc=4, m=6, eps_grad=1e-4, grad_mode=M.GRAD_ADJOINT, seed=9)
    outs = []
    for use_graph in (1, 1, 0):
        model = U.open_ctx(prob, P, use_graph=use_graph)
        for _ in range(3):
            model.step()
        outs.append(model.get(0, CH.FIELD_X).copy())
        model.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_full_size_quadratic_step_properties():
    """quadratic_d64 at N = 65536 in the benchmark's launch configuration (the Phase 1
    kernel over every sample, condition 1e4).  Three iterations, each launched on the
    whole population from the state the previous one left; on 512 sampled rows every
    iteration matches the oracle's one iteration from the same binary32 state to 1e-5
    of the step (rows where binary32 and FP64 decide an Armijo test differently take
    a power-of-two multiple of the oracle's step, at most 2 %).  Then the fused launch
    of the benchmark (n_conv = 18 iterations in one kernel): f never decreases, f and
    the gradient it stores are the objective's at the point it stores (1e-5; the
    gradient at the objective parity bound), every stored pair is curved with
    rho = 1 / s^T y; and a full non-final cycle runs."""
    from test_gpu_kernels import assert_grad_close, grad_term_scale, value_term_scale
    prob = I.quadratic_d64()
    P = M.Params(n_osc=1000, m=10, eps_grad=0.05, grad_mode=M.GRAD_ADJOINT, seed=3)
    model = U.open_ctx(prob, P)
    rows = np.sort(np.random.default_rng(0).choice(prob.n, 512, replace=False))
    sub = I.Problem(64, rows.size, prob.lo, prob.hi, prob.objective, prob.x0[rows], prob.eps_grad,
                    prob.sigma_mode)
    st = U.read_state(model, prob, P.m, rows=rows)
    for it in range(3):
        model.run_phase(0, CH.PHASE_LBFGS, 1 if it == 0 else -1)
        got = U.read_state(model, prob, P.m, rows=rows)
        ref = M.State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.__dict__.items()})
        M.lbfgs_iterations(sub, ref, P, 1, fresh_gradient=(it == 0))
        U.assert_phase1_step(st, got, ref)
        if it > 0:                                    # the first launch evaluates f itself
            assert np.all(got.f >= st.f - 1e-6 * np.abs(st.f))
        st = got
    x_before = model.get(0, CH.FIELD_X)[:, :64].astype(np.float64)
    f_before = model.get(0, CH.FIELD_F).astype(np.float64)
    model.run_phase(0, CH.PHASE_LBFGS, -P.n_conv_for(64))
    st = U.read_state(model, prob, P.m)
    assert np.all(st.f >= f_before - 1e-6 * np.abs(f_before))
    assert np.any(np.abs(st.x - x_before).max(axis=1) > 0)
    f_ref = OB.value(prob.objective, st.x)
    assert np.all(np.abs(st.f - f_ref) <= 1e-5 * (value_term_scale(prob, st.x) + 1.0))
    assert_grad_close(st.g[rows], OB.grad(prob.objective, st.x[rows]), grad_term_scale(prob, st.x[rows]), 1e-5)
    for k in range(P.m):
        live = st.hlen > k
        sy = np.einsum("nd,nd->n", st.S[live, k], st.Y[live, k])
        assert np.all(sy > 0)
        np.testing.assert_allclose(st.rho[live, k], 1.0 / sy, rtol=4 * 2.0 ** -24)
    model.step()                                      # a full non-final cycle runs
    c = model.counters(0)
    assert c["cycles"] == 1 and c["evals"] > 0 and c["ls_fail"] <= c["ls_trials"]
    model.close()


def test_modes_capacity_and_errors():
    prob = I.mixture4_d2(n=256)
    P = M.Params(n_osc=2, m=5, eps_grad=1e-5, grad_mode=M.GRAD_ADJOINT)
    model = U.open_ctx(prob, P)
    model.step()
    model.step()
    x, f = model.modes(0)
    with pytest.raises(CH.ChisaoError):
        model.modes(0, cap=max(0, x.shape[0] - 1))
    model.load_population(0, prob.x0)                   # resets the cycle count
    model.step()
    assert model.counters(0)["cycles"] == 1
    model.close()


@pytest.mark.parametrize("sigma", [0.1, 1.0])
def test_noisy_mixture_modes_adjoint(sigma):
    """Sec. 5.6 noise on every evaluation: with exact gradients the four modes
    are still found, and no spurious mode is returned (oracle: the same)."""
    prob = I.mixture4_d2(n=1024)
    prob.objective.noise_sigma = sigma
    P = M.Params(n_osc=4, m=5, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=0)
    model = U.open_ctx(prob, P)
    fx, ff = _run(model, P.n_osc)
    mx, mf, negH = MD.significant_modes(prob)
    frac, worst, _ = MD.recovery(fx, mx, negH)
    assert frac == 1.0 and fx.shape[0] == 4
    model.close()


def test_tensor_core_cycle_with_fp32_refinement():
    """d=64, K=256 full-covariance mixture on the BF16 tensor-core objective
    (Phases 1, 5, 6), then n_refine FP32 L-BFGS steps with the exact objective on
    the survivors after the last cycle: every returned point is a local maximum
    of the exact objective to 1e-3 local sigmas."""
    prob = I.mixture256_d64(n=8192)
    P = M.Params(n_osc=2, n_conv=100, m=10, eps_grad=1e-2, grad_mode=M.GRAD_ADJOINT, seed=4)
    model = U.open_ctx(prob, P, grad_mode=CH.GRAD_ADJOINT_TC, n_refine=10)
    fx, ff = _run(model, P.n_osc)
    c = model.counters(0)
    assert fx.shape[0] >= 3 and c["cycles"] == 2 and c["evals"] > 0
    assert np.all(_local_mode_errors(prob, fx) <= 1e-3)
    model.close()


def test_tensor_core_cycle_graph_equivalence():
    """The tensor-core cycle captured in a CUDA graph and launched eagerly leave the same
    state bit for bit (the line-search rounds fill their lists with atomics, in any order,
    and every result is per sample) and count the same evaluations, trials and failed
    searches."""
    prob = I.mixture256_d64(n=4096)
    P = M.Params(n_osc=3, n_conv=12, m=10, eps_grad=1e-2, grad_mode=M.GRAD_ADJOINT, seed=7)
    fields = (CH.FIELD_X, CH.FIELD_G, CH.FIELD_F, CH.FIELD_HS, CH.FIELD_HY, CH.FIELD_HLEN, CH.FIELD_STUCK)
    keys = ("evals", "grads", "ls_trials", "ls_fail")
    runs = []
    for use_graph in (1, 0):
        model = U.open_ctx(prob, P, grad_mode=CH.GRAD_ADJOINT_TC, use_graph=use_graph)
        for _ in range(2):
            model.step()
        c = model.counters(0)
        runs.append(({f: model.get(0, f).copy() for f in fields}, {k: c[k] for k in keys}))
        model.close()
    for f in fields:
        np.testing.assert_array_equal(runs[0][0][f], runs[1][0][f])
    assert runs[0][1] == runs[1][1], runs


@pytest.mark.parametrize("d", [8, 16])
def test_carry_tiger_seeding_on_ackley(d):
    """Sec. 5.3: on Ackley's flat outer region uniform samples see almost no
    gradient, and ray seeding from the domain's faces, edges and vertices cuts
    through it.  After four cycles from each seeding (the same seeds otherwise),
    the best mode found from Carry Tiger lies well above the best from uniform
    seeding, and every returned point is a local maximum."""
    best = {}
    for method in (CH.SEED_UNIFORM, CH.SEED_CARRY_TIGER):
        prob = I.benchmark("ackley", d, 4096, seed=3, eps_grad=1e-3)
        P = M.Params(n_osc=4, m=10, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=5)
        model = U.open_ctx(prob, P)
        model.seed(0, method)
        for _ in range(P.n_osc):
            model.step()
        fx, ff = model.modes(0)
        best[method] = ff.max()
        if method == CH.SEED_CARRY_TIGER:
            assert np.all(_local_mode_errors(prob, fx) <= 1e-3)
        model.close()
    assert best[CH.SEED_CARRY_TIGER] > best[CH.SEED_UNIFORM] + 5.0


@pytest.mark.parametrize("noise", I.NOISE_LEVELS)
def test_two_mode_d6_noise_levels(noise):
    """The Sec. 5.6 noise workload (d = 6, unit components at +-2 e_1) at each noise
    level of its table, exact gradients: both peaks within 1e-3 sigma, no spurious
    mode, over three seeds."""
    for seed in range(3):
        prob = I.mixture2_d6(n=2048, seed=seed, noise_sigma=noise)
        P = M.Params(n_osc=3, m=10, eps_grad=prob.eps_grad, grad_mode=M.GRAD_ADJOINT, seed=seed)
        model = U.open_ctx(prob, P)
        fx, ff = _run(model, P.n_osc)
        mx, mf, negH = MD.significant_modes(prob)
        frac, worst, _ = MD.recovery(fx, mx, negH)
        assert frac == 1.0 and fx.shape[0] == 2, (seed, frac, fx.shape)
        model.close()


def test_large_population_quadratic():
    """N = 2^22 samples at d = 64 (the history holds 2.7e9 floats, past 32-bit
    indexing): one Phase-1 iteration on sampled rows, the first and the last
    included, matches the oracle's on the same rows, and a whole cycle runs."""
    n = 1 << 22
    prob = I.quadratic_d64(n=n, seed=1)
    P = M.Params(n_osc=1000, m=10, eps_grad=0.05, grad_mode=M.GRAD_ADJOINT, seed=3)
    model = U.open_ctx(prob, P)
    model.run_phase(0, CH.PHASE_LBFGS, 1)
    x1 = model.get(0, CH.FIELD_X)[:, :64]
    rows = np.concatenate([[0, 1, n // 2], np.random.default_rng(1).choice(n, 40, replace=False), [n - 2, n - 1]])
    sub = I.Problem(64, rows.size, prob.lo, prob.hi, prob.objective, prob.x0[rows], prob.eps_grad, prob.sigma_mode)
    ref = M.new_state(prob.x0[rows].astype(np.float64), P.m)
    M.lbfgs_iterations(sub, ref, P, 1)
    x0 = prob.x0[rows].astype(np.float64)
    move = np.abs(ref.x - x0).max(axis=1)
    err = np.abs(x1[rows].astype(np.float64) - ref.x).max(axis=1)
    ok = err <= 1e-4 * move + 1e-6 * np.abs(x0).max(axis=1)
    # a binary32-vs-FP64 tie of the Armijo test takes the neighbouring trial (a power-of-two step)
    assert (~ok).sum() <= 2, (err / move)[~ok]
    for i in np.flatnonzero(~ok):
        dg, dr = x1[rows[i]] - x0[i], ref.x[i] - x0[i]
        j = np.argmax(np.abs(dr))
        ratio = abs(dg[j] / dr[j])
        assert abs(np.log2(ratio) - round(np.log2(ratio))) < 1e-3
    hlen = model.get(0, CH.FIELD_HLEN)
    np.testing.assert_array_equal(hlen[rows][ok], ref.hlen[ok])
    model.step()
    c = model.counters(0)
    assert c["cycles"] == 1 and c["evals"] > 2 * n
    model.close()


@pytest.mark.parametrize("d,n", [(1, 1), (1, 37), (3, 1), (64, 1), (2, 2)])
def test_degenerate_sizes(d, n):
    """One coordinate, one sample, two samples: one Phase-1 iteration matches the
    oracle, whole cycles run, and the returned modes and widths are consistent."""
    prob = I.small_mixture(d, 2, n, seed=40 + d)
    P = M.Params(n_osc=3, m=5, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=1)
    model = U.open_ctx(prob, P)
    model.run_phase(0, CH.PHASE_LBFGS, 1)
    got = U.read_state(model, prob, P.m)
    ref = M.new_state(prob.x0.astype(np.float64), P.m)
    M.lbfgs_iterations(prob, ref, P, 1)
    move = np.abs(ref.x - prob.x0).max(axis=1)
    err = np.abs(got.x - ref.x).max(axis=1)
    assert np.all(err <= 1e-4 * move + 1e-6 * (1.0 + np.abs(prob.x0).max(axis=1))), (err, move)
    model.close()
    model = U.open_ctx(prob, P)
    for _ in range(P.n_osc):
        model.step()
    fx, ff = model.modes(0)
    w, H = model.widths(0, cov=True)
    assert fx.shape == (w.shape[0], d) and H.shape == (w.shape[0], d, d)
    assert np.all(w > 0) and np.all(np.isfinite(H))
    assert model.counters(0)["cycles"] == P.n_osc
    model.close()


def test_bounded_wait_timeout_is_reported_and_the_context_stays_usable():
    """A device wait that nothing completes gives up after its budget (no trap, no
    hang), raises the problem's error flag, and chisao_get_counters reports
    CHISAO_ERR_TIMEOUT once and clears it; the context then keeps stepping."""
    prob = I.small_mixture(3, 2, 500, seed=1)
    P = M.Params(n_osc=4, m=5, grad_mode=M.GRAD_ADJOINT, seed=2)
    model = U.open_ctx(prob, P)
    model.step()
    model.selftest_wait(0, budget_ns=20_000_000)
    with pytest.raises(CH.ChisaoError, match=r"\(6\)"):
        model.counters(0)
    c = model.counters(0)
    assert c["device_error"] == 0 and c["cycles"] == 1
    model.step()
    model.step()
    fx, _ = model.modes(0)
    assert model.counters(0)["cycles"] == 3 and fx.shape[1] == 3
    model.close()


def test_autotune_keeps_state_and_results():
    """The launch-shape autotuner (branch streams x grouped or per-problem launches)
    leaves the state as it found it, and the cycles that follow give the same bits as
    in a context that was never tuned."""
    probs = I.batched512(n_problems=20, n_scale=0.05, seed=8)
    P = M.Params(n_osc=6, m=6, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=3)
    U.ensure_built()
    tuned = CH.Chisao(probs, U.lib_params(P))
    plain = CH.Chisao(probs, U.lib_params(P))
    for m in (tuned, plain):
        m.step()
    before = [tuned.get(q, CH.FIELD_X).copy() for q in range(len(probs))]
    t = tuned.autotune(cycles_per_trial=1)
    assert t["trials"] >= 4 and t["n_branch"] in (8, 16, 20) and t["grouped"] in (0, 1)
    assert all(ck in (2, 4, 8) for ck in t["ck"].values())
    assert 0 < t["ms_per_cycle"] <= t["ms_default"] * 1.0001
    for q in range(len(probs)):
        np.testing.assert_array_equal(tuned.get(q, CH.FIELD_X), before[q])
        assert tuned.counters(q)["cycles"] == 1
    for m in (tuned, plain):
        m.step()
        m.step()
    for q in range(len(probs)):
        for fld in (CH.FIELD_X, CH.FIELD_F, CH.FIELD_STUCK):
            np.testing.assert_array_equal(tuned.get(q, fld), plain.get(q, fld))
    tuned.close()
    plain.close()


def test_tile_shapes_give_the_same_bits():
    """The compiled tile shapes of the grouped diagonal-mixture kernels (2, 4 or 8
    components per step; the tuner picks one per padded dimension) change only the
    schedule: whole cycles give the same bits with every shape."""
    probs = I.batched512(n_problems=24, n_scale=0.05, seed=9)
    P = M.Params(n_osc=4, m=6, eps_grad=1e-3, grad_mode=M.GRAD_ADJOINT, seed=4)
    U.ensure_built()
    dps = sorted({max(4, 1 << (p.d - 1).bit_length()) for p in probs})
    out = []
    for ck in (4, 2, 8):
        model = CH.Chisao(probs, U.lib_params(P))
        for dp in dps:
            model.set_tile(dp, ck)
        for _ in range(3):
            model.step()
        out.append([model.get(q, f).copy() for q in range(len(probs)) for f in (CH.FIELD_X, CH.FIELD_G, CH.FIELD_F)])
        with pytest.raises(CH.ChisaoError):
            model.set_tile(dps[0], 3)
        model.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            np.testing.assert_array_equal(a, b)
