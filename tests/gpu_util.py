"""Helpers for the GPU parity tests: build the library, open contexts, and move
state between the CUDA library (through the C ABI) and the oracle."""
import numpy as np

from oracle import method as M
from paper_2606_26164_gb300 import build
from paper_2606_26164_gb300 import chisao as CH

_built = False


def ensure_built():
    global _built
    if not _built:
        build.build()
        _built = True


def lib_params(P: M.Params, **over) -> CH.CParams:
    """The C parameter block with the same values as an oracle Params."""
    p = CH.default_params(n_osc=P.n_osc, n_conv=P.n_conv, n_anti=P.n_anti, n_cloud=P.n_cloud, M=P.M, m=P.m,
                          T_ls=P.T_ls, grad_mode=P.grad_mode, eps_grad=P.eps_grad, eps_dup=P.eps_dup,
                          delta=P.delta, mu=P.mu, alpha=P.alpha, sigma=P.sigma, c_sigma=P.c_sigma,
                          alpha_scale=P.alpha_scale, h=P.h, h_rel=P.h_rel, c1=P.c1, curv_eps=P.curv_eps,
                          seed=P.seed, rm_min_unfrozen=P.rm_min_unfrozen, gr_patience=P.gr_patience,
                          hlc_value_only=P.hlc_value_only)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def open_ctx(prob, P: M.Params, **over) -> CH.Chisao:
    ensure_built()
    return CH.Chisao([prob], lib_params(P, **over))


def read_state(model: CH.Chisao, prob, m: int, q: int = 0, rows=None) -> M.State:
    """Oracle State (FP64 copies of the FP32 device values); with `rows`, only those
    samples (the masks stay whole-population)."""
    d = prob.d
    sel = (lambda a: a) if rows is None else (lambda a: a[rows])
    x = sel(model.get(q, CH.FIELD_X))[:, :d].astype(np.float64)
    st = M.new_state(x, m)
    st.g = sel(model.get(q, CH.FIELD_G))[:, :d].astype(np.float64)
    st.f = sel(model.get(q, CH.FIELD_F)).astype(np.float64)
    hs = sel(model.get(q, CH.FIELD_HS))[:, :m, :d].astype(np.float64)
    hy = sel(model.get(q, CH.FIELD_HY))[:, :m, :d].astype(np.float64)
    rho = sel(model.get(q, CH.FIELD_HRHO))[:, :m].copy()
    hlen = sel(model.get(q, CH.FIELD_HLEN)).astype(np.int64)
    for k in range(m):
        live = hlen > k
        hs[~live, k] = 0.0
        hy[~live, k] = 0.0
        rho[~live, k] = 0.0
    st.S, st.Y, st.rho, st.hlen = hs, hy, rho, hlen
    n = prob.n
    st.stuck = sel(CH.unpack_bits(model.get(q, CH.FIELD_STUCK), n))
    st.removed = sel(CH.unpack_bits(model.get(q, CH.FIELD_REMOVED), n))
    return st


def write_state(model: CH.Chisao, prob, st: M.State, q: int = 0):
    """Write FP32-rounded oracle state into the device (rho recomputed from
    the FP32 pairs so the history is self-consistent)."""
    d, n = prob.d, prob.n
    dp, mm = model.layout(q)
    m = st.S.shape[1]
    X = np.zeros((n, dp), np.float32)
    X[:, :d] = st.x
    model.set(q, CH.FIELD_X, X)
    G = np.zeros((n, dp), np.float32)
    G[:, :d] = st.g
    model.set(q, CH.FIELD_G, G)
    model.set(q, CH.FIELD_F, st.f.astype(np.float32))
    HS = np.zeros((n, mm, dp), np.float32)
    HY = np.zeros((n, mm, dp), np.float32)
    HS[:, :m, :d] = st.S
    HY[:, :m, :d] = st.Y
    R = np.zeros((n, mm), np.float32)
    s64, y64 = HS[:, :m, :d].astype(np.float64), HY[:, :m, :d].astype(np.float64)
    sy = np.einsum("nkd,nkd->nk", s64, y64)
    with np.errstate(divide="ignore"):
        R[:, :m] = np.where(np.arange(m)[None, :] < st.hlen[:, None], 1.0 / np.where(sy != 0, sy, 1.0), 0.0)
    model.set(q, CH.FIELD_HS, HS)
    model.set(q, CH.FIELD_HY, HY)
    model.set(q, CH.FIELD_HRHO, R)
    model.set(q, CH.FIELD_HLEN, st.hlen.astype(np.int32))
    model.set(q, CH.FIELD_STUCK, CH.pack_bits(st.stuck))
    model.set(q, CH.FIELD_REMOVED, CH.pack_bits(st.removed))


def rounded(st: M.State) -> M.State:
    """The state with every float rounded through binary32 (what the device holds)."""
    r = M.State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.__dict__.items()})
    for k in ("x", "g", "f", "S", "Y"):
        setattr(r, k, getattr(st, k).astype(np.float32).astype(np.float64))
    m = r.S.shape[1]
    sy = np.einsum("nkd,nkd->nk", r.S, r.Y)
    with np.errstate(divide="ignore"):
        r.rho = np.where(np.arange(m)[None, :] < r.hlen[:, None], 1.0 / np.where(sy != 0, sy, 1.0), 0.0)
    return r


def rel_err_rows(a, b, floor=0.0):
    """Per-row ||a - b||_inf / max(||b||_inf, floor)."""
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), floor)


def assert_phase1_step(st: M.State, got: M.State, ref: M.State, max_tie_frac: float = 0.02):
    """One Phase-1 iteration from the same binary32 state: every row's new position
    within 1e-5 of the oracle's step (plus binary32 rounding of the position), except
    rows where binary32 and FP64 decided an Armijo test differently -- there the
    device's step must be a power-of-two multiple of the oracle's, and at most
    max_tie_frac of the rows may be such ties.  Returns the mask of matching rows."""
    step = np.abs(ref.x - st.x).max(axis=1)
    xerr = np.abs(got.x - ref.x).max(axis=1)
    scale = np.abs(st.x).max(axis=1)
    ok = xerr <= 1e-5 * step + 4e-7 * scale
    bad = np.flatnonzero(~ok)
    assert bad.size <= max_tie_frac * st.x.shape[0], (bad.size, xerr[bad][:5], step[bad][:5])
    for i in bad:
        dg = got.x[i] - st.x[i]
        dr = ref.x[i] - st.x[i]
        j = np.argmax(np.abs(dr))
        ratio = dg[j] / dr[j] if dr[j] != 0 else np.inf
        assert np.isfinite(ratio) and abs(np.log2(abs(ratio)) - round(np.log2(abs(ratio)))) < 1e-3, (i, ratio)
    return ok

