"""ctypes binding of the C ABI in include/chisao.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libchisao.so``; when it is
missing this module raises instead of falling back to anything else.  PyTorch
supplies device memory (the context arena) and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libchisao.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_CAPACITY, ERR_STATE, ERR_TIMEOUT = 0, 1, 2, 3, 4, 5, 6
GRAD_FD64, GRAD_FD32, GRAD_ADJOINT, GRAD_ADJOINT_TC = 0, 1, 2, 3
SEED_UNIFORM, SEED_CARRY_TIGER = 0, 1
FIELD_X, FIELD_G, FIELD_F, FIELD_HS, FIELD_HY, FIELD_HRHO, FIELD_HLEN, FIELD_STUCK, FIELD_REMOVED = range(9)
(PHASE_LBFGS, PHASE_FREEZE, PHASE_DEDUP, PHASE_RESEED, PHASE_HLC, PHASE_ANTI, PHASE_DIRECTION, PHASE_LISTS,
 PHASE_REFINE) = range(1, 10)
MMAX = 10

EXPORTS = ["chisao_default_params", "chisao_arena_bytes", "chisao_create", "chisao_step",
           "chisao_load_population", "chisao_modes", "chisao_get_counters", "chisao_eval",
           "chisao_last_error", "chisao_destroy", "chisao_layout", "chisao_state_get",
           "chisao_state_set", "chisao_run_phase", "chisao_set_gr_state", "chisao_dedup_noalloc", "chisao_seed",
           "chisao_widths", "chisao_selftest_wait", "chisao_autotune", "chisao_measure_fma_peak", "chisao_measure_mma_rate", "chisao_init",
           "chisao_stats", "chisao_set_tile"]


class CParams(C.Structure):
    _fields_ = [("n_osc", C.c_int32), ("n_conv", C.c_int32), ("n_anti", C.c_int32), ("n_cloud", C.c_int32),
                ("M", C.c_int32), ("m", C.c_int32), ("T_ls", C.c_int32), ("grad_mode", C.c_int32),
                ("eps_grad", C.c_double), ("eps_dup", C.c_double), ("delta", C.c_double), ("mu", C.c_double),
                ("alpha", C.c_double), ("sigma", C.c_double), ("c_sigma", C.c_double),
                ("alpha_scale", C.c_double), ("h", C.c_double), ("h_rel", C.c_double), ("c1", C.c_double),
                ("curv_eps", C.c_double), ("seed", C.c_uint64), ("rm_min_unfrozen", C.c_int32),
                ("gr_patience", C.c_int32), ("use_graph", C.c_int32), ("n_refine", C.c_int32),
                ("hlc_value_only", C.c_int32)]


_DP = C.POINTER(C.c_double)


# int32 (*)(user, x, ldx, rows, idx, count, f, g, ldg, stream)
BATCH_EVAL_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p)


class CObjective(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_comp", C.c_int32), ("weights", _DP), ("means", _DP),
                ("sigmas", _DP), ("chol", _DP), ("center", _DP), ("Q", _DP), ("lam", _DP),
                ("noise_sigma", C.c_double), ("eval", BATCH_EVAL_FN), ("user", C.c_void_p)]


class _DevArray:
    """A device buffer seen by torch.as_tensor (CUDA array interface, no copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


def _external_evaluator(fn, d: int, errors: list):
    """The C evaluator of an OBJ_EXTERNAL objective: runs fn on the listed rows on
    the stream the library passes (reading the row count synchronizes that stream,
    so contexts with such objectives run without CUDA graphs)."""
    import torch

    def call(user, x, ldx, rows, idx, count, f, g, ldg, stream):
        try:
            if rows <= 0:
                return 0
            with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
                X = torch.as_tensor(_DevArray(x, (rows, ldx), "<f4"), device="cuda")
                if idx:
                    k = int(torch.as_tensor(_DevArray(count, (1,), "<i4"), device="cuda").item())
                    if k <= 0:
                        return 0
                    sel = torch.as_tensor(_DevArray(idx, (k,), "<i4"), device="cuda").long()
                else:
                    sel = None
                pts = (X[sel] if sel is not None else X)[:, :d].contiguous()
                fv, gv = fn(pts)
                if f:
                    Fo = torch.as_tensor(_DevArray(f, (rows,), "<f4"), device="cuda")
                    if sel is None:
                        Fo.copy_(fv.reshape(-1))
                    else:
                        Fo.index_copy_(0, sel, fv.reshape(-1).to(torch.float32))
                if g:
                    Go = torch.as_tensor(_DevArray(g, (rows, ldg), "<f4"), device="cuda")
                    gv = gv.reshape(-1, d).to(torch.float32)
                    if sel is None:
                        Go[:, :d].copy_(gv)
                    else:
                        Go[sel, :d] = gv
            return 0
        except Exception as e:                 # reported by the next call into the binding
            errors.append(e)
            return ERR_ARG

    return BATCH_EVAL_FN(call)


def autograd_objective(fval):
    """fn for an OBJ_EXTERNAL objective from a value-only torch function
    fval(x [k, d]) -> f [k]: the gradient comes from torch.autograd."""
    import torch

    def fn(x):
        with torch.enable_grad():
            xr = x.detach().requires_grad_(True)
            fv = fval(xr)
            (gv,) = torch.autograd.grad(fv.sum(), xr)
        return fv.detach(), gv
    return fn


class CProblem(C.Structure):
    _fields_ = [("d", C.c_int32), ("n", C.c_int64), ("lo", _DP), ("hi", _DP),
                ("x0", C.POINTER(C.c_float)), ("objective", CObjective)]


class CTuning(C.Structure):
    _fields_ = [("n_branch", C.c_int32), ("grouped", C.c_int32), ("trials", C.c_int32),
                ("ms_per_cycle", C.c_float), ("ms_default", C.c_float), ("ck", C.c_int32 * 5)]


class CCounters(C.Structure):
    _fields_ = [("evals", C.c_uint64), ("grads", C.c_uint64), ("ls_trials", C.c_uint64), ("ls_fail", C.c_uint64),
                ("cycles", C.c_int64), ("n_stuck", C.c_int64), ("k_lost", C.c_int64), ("n_unfrozen", C.c_int64),
                ("last_reseed", C.c_int32), ("gr_enabled", C.c_int32), ("f_max", C.c_float),
                ("sigma", C.c_float), ("alpha_hlc", C.c_float), ("alpha_anti", C.c_float),
                ("device_error", C.c_int32)]


_lib = None


def library() -> C.CDLL:
    """Load the CUDA library; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2606_26164_gb300.build)")
        lib = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        lib.chisao_default_params.argtypes = [C.POINTER(CParams)]
        lib.chisao_default_params.restype = None
        lib.chisao_arena_bytes.argtypes = [C.POINTER(CProblem), C.c_int32, C.POINTER(CParams), C.POINTER(C.c_size_t)]
        lib.chisao_create.argtypes = [C.POINTER(CProblem), C.c_int32, C.POINTER(CParams), vp, C.c_size_t, vp,
                                      C.POINTER(vp)]
        lib.chisao_init.argtypes = [C.POINTER(CProblem), C.c_int32, C.POINTER(CParams), vp, C.POINTER(vp)]
        lib.chisao_stats.argtypes = [vp, C.c_int32, C.POINTER(CCounters)]
        lib.chisao_step.argtypes = [vp]
        lib.chisao_load_population.argtypes = [vp, C.c_int32, C.POINTER(C.c_float)]
        lib.chisao_seed.argtypes = [vp, C.c_int32, C.c_int32]
        lib.chisao_selftest_wait.argtypes = [vp, C.c_int32, C.c_int64]
        lib.chisao_autotune.argtypes = [vp, C.c_int32, C.POINTER(CTuning)]
        lib.chisao_measure_fma_peak.argtypes = [C.c_int32, vp, C.POINTER(C.c_double)]
        lib.chisao_measure_mma_rate.argtypes = [C.c_int32, C.c_int32, C.c_int32, vp, C.POINTER(C.c_double)]
        lib.chisao_widths.argtypes = [vp, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int64,
                                      C.POINTER(C.c_int64)]
        lib.chisao_modes.argtypes = [vp, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int64,
                                     C.POINTER(C.c_int64)]
        lib.chisao_get_counters.argtypes = [vp, C.c_int32, C.POINTER(CCounters)]
        lib.chisao_eval.argtypes = [vp, C.c_int32, vp, C.c_int64, vp, vp, C.c_int32]
        lib.chisao_last_error.argtypes = [vp]
        lib.chisao_last_error.restype = C.c_char_p
        lib.chisao_destroy.argtypes = [vp]
        lib.chisao_destroy.restype = None
        lib.chisao_layout.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        lib.chisao_state_get.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_size_t]
        lib.chisao_state_set.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_size_t]
        lib.chisao_run_phase.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
        lib.chisao_set_gr_state.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        lib.chisao_set_tile.argtypes = [vp, C.c_int32, C.c_int32]
        lib.chisao_dedup_noalloc.argtypes = [vp, C.c_int32, C.c_int64, vp, vp, C.c_double, vp, vp, vp]
        for name in EXPORTS:
            if name not in ("chisao_default_params", "chisao_last_error", "chisao_destroy"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
    return _lib


def measure_mma_rate(n: int, threads: int, tmem_a: int = 0, stream=None) -> float:
    """SM clocks per tcgen05.mma (M = 128, K = 16, width n) with `threads` issuers together."""
    out = C.c_double(0.0)
    ptr = C.c_void_p(stream.cuda_stream) if stream is not None else None
    st = library().chisao_measure_mma_rate(n, threads, tmem_a, ptr, C.byref(out))
    if st != OK:
        raise ChisaoError(f"chisao_measure_mma_rate failed ({st})")
    return out.value


def measure_fma_peak(f64: bool = False, stream=None) -> float:
    """Measured FMA throughput of the current GPU in FLOP/s (binary32 or binary64)."""
    out = C.c_double(0.0)
    ptr = C.c_void_p(stream.cuda_stream) if stream is not None else None
    st = library().chisao_measure_fma_peak(1 if f64 else 0, ptr, C.byref(out))
    if st != OK:
        raise ChisaoError(f"chisao_measure_fma_peak failed ({st})")
    return out.value


def copy_params(p: CParams) -> CParams:
    q = CParams()
    C.memmove(C.byref(q), C.byref(p), C.sizeof(CParams))
    return q


def default_params(**over) -> CParams:
    p = CParams()
    library().chisao_default_params(C.byref(p))
    for k, v in over.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class ChisaoError(RuntimeError):
    pass


def _dptr(a: Optional[np.ndarray]):
    return a.ctypes.data_as(_DP) if a is not None else None


class Chisao:
    """One context over one or more problems (``inputs.Problem``)."""

    def __init__(self, problems: Sequence[I.Problem], params: CParams, use_torch_arena: bool = True,
                 stream=None):
        lib = library()
        self._keep = []
        self._callbacks = []                   # live as long as the context
        self._cb_errors = []
        cprobs = (CProblem * len(problems))()
        for q, pr in enumerate(problems):
            ob = pr.objective
            A = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in ob.arrays.items()}
            lo = np.ascontiguousarray(pr.lo, np.float64)
            hi = np.ascontiguousarray(pr.hi, np.float64)
            x0 = np.ascontiguousarray(pr.x0, np.float32)
            self._keep += [A, lo, hi, x0]
            co = CObjective(kind=ob.kind, n_comp=ob.n_comp, weights=_dptr(A.get("weights")),
                            means=_dptr(A.get("means")), sigmas=_dptr(A.get("sigmas")), chol=_dptr(A.get("chol")),
                            center=_dptr(A.get("center")), Q=_dptr(A.get("Q")), lam=_dptr(A.get("lam")),
                            noise_sigma=float(getattr(ob, "noise_sigma", 0.0)))
            if ob.kind == I.OBJ_EXTERNAL:
                cb = _external_evaluator(ob.fn, pr.d, self._cb_errors)
                self._callbacks.append(cb)
                co.eval = cb
                if params.use_graph:
                    params = copy_params(params)
                    params.use_graph = 0           # the evaluator reads the row count on the host
            cprobs[q] = CProblem(d=pr.d, n=pr.n, lo=_dptr(lo), hi=_dptr(hi),
                                 x0=x0.ctypes.data_as(C.POINTER(C.c_float)), objective=co)
        self.problems = list(problems)
        self.params = params
        nbytes = C.c_size_t(0)
        st = lib.chisao_arena_bytes(cprobs, len(problems), C.byref(params), C.byref(nbytes))
        if st != OK:
            raise ChisaoError(f"chisao_arena_bytes failed ({st})")
        self.arena_bytes = nbytes.value
        arena_ptr = None
        self._arena = None
        self._stream = None
        import torch
        if stream is None:
            self._stream = torch.cuda.Stream()
            stream_ptr = self._stream.cuda_stream
        else:
            self._stream = stream
            stream_ptr = stream.cuda_stream
        if use_torch_arena:
            self._arena = torch.empty(self.arena_bytes + 256, dtype=torch.uint8, device="cuda")
            base = self._arena.data_ptr()
            arena_ptr = (base + 255) // 256 * 256
        ctx = C.c_void_p()
        st = lib.chisao_create(cprobs, len(problems), C.byref(params), arena_ptr, self.arena_bytes,
                               C.c_void_p(stream_ptr), C.byref(ctx))
        if st != OK:
            raise ChisaoError(f"chisao_create failed ({st})")
        self.ctx = ctx
        self._keep = []

    # ------------------------------------------------------------------ core API
    def _check(self, st, what):
        if self._cb_errors:
            e = self._cb_errors[0]
            self._cb_errors.clear()
            raise ChisaoError(f"{what}: the external objective raised {e!r}") from e
        if st != OK:
            msg = library().chisao_last_error(self.ctx).decode()
            raise ChisaoError(f"{what} failed ({st}): {msg}")

    def step(self):
        self._check(library().chisao_step(self.ctx), "chisao_step")

    def load_population(self, prob: int, x: np.ndarray):
        x = np.ascontiguousarray(x, np.float32)
        self._check(library().chisao_load_population(self.ctx, prob, x.ctypes.data_as(C.POINTER(C.c_float))),
                    "chisao_load_population")
        self.synchronize()

    def seed(self, prob: int, method: int = SEED_CARRY_TIGER):
        """Initial population generated on the device (uniform or Carry Tiger)."""
        self._check(library().chisao_seed(self.ctx, prob, method), "chisao_seed")

    def modes(self, prob: int = 0, cap: Optional[int] = None):
        pr = self.problems[prob]
        cap = pr.n if cap is None else cap
        xo = np.empty((max(cap, 1), pr.d), np.float32)
        fo = np.empty(max(cap, 1), np.float32)
        cnt = C.c_int64(0)
        self._check(library().chisao_modes(self.ctx, prob, xo.ctypes.data_as(C.POINTER(C.c_float)),
                                           fo.ctypes.data_as(C.POINTER(C.c_float)), cap, C.byref(cnt)),
                    "chisao_modes")
        k = cnt.value
        return xo[:k].copy(), fo[:k].copy()

    def widths(self, prob: int = 0, cov: bool = False):
        """Laplace widths of the modes (order of `modes`): (w [k, d], H [k, d, d] or None)."""
        d = self.problems[prob].d
        cnt = C.c_int64(0)
        fp = C.POINTER(C.c_float)
        library().chisao_widths(self.ctx, prob, None, None, 0, C.byref(cnt))    # the count only
        k = cnt.value
        wo = np.empty((max(k, 1), d), np.float32)
        co = np.empty((max(k, 1), d, d), np.float32) if cov else None
        if k > 0:
            self._check(library().chisao_widths(self.ctx, prob, wo.ctypes.data_as(fp),
                                                co.ctypes.data_as(fp) if cov else None, k, C.byref(cnt)),
                        "chisao_widths")
        return wo[:k].copy(), (co[:k].copy() if cov else None)

    def autotune(self, cycles_per_trial: int = 2) -> dict:
        """Pick the fastest launch shape for this context (results and state unchanged)."""
        t = CTuning()
        self._check(library().chisao_autotune(self.ctx, cycles_per_trial, C.byref(t)), "chisao_autotune")
        out = {name: getattr(t, name) for name, _ in CTuning._fields_}
        out["ck"] = {4 << k: int(t.ck[k]) for k in range(5) if t.ck[k]}
        return out

    def selftest_wait(self, prob: int = 0, budget_ns: int = 10_000_000):
        """Test hook: a bounded device wait that runs out and raises the problem's error flag."""
        self._check(library().chisao_selftest_wait(self.ctx, prob, budget_ns), "chisao_selftest_wait")

    def counters(self, prob: int = 0) -> dict:
        c = CCounters()
        self._check(library().chisao_get_counters(self.ctx, prob, C.byref(c)), "chisao_get_counters")
        return {name: getattr(c, name) for name, _ in CCounters._fields_}

    def eval(self, prob: int, x, grad_mode: int = GRAD_ADJOINT, want_grad: bool = True):
        """f (and grad f) at device points x (a CUDA float32 tensor [n, d], d = the
        problem's dimension; non-contiguous inputs are copied).  Raises ChisaoError,
        launching nothing, for any other dtype, device or shape."""
        import torch
        self._check_points(prob, x)
        x = x.detach().contiguous()
        n = x.shape[0]
        f = torch.empty(n, dtype=torch.float32, device=x.device)
        g = torch.empty_like(x) if want_grad else None
        self._stream.wait_stream(torch.cuda.current_stream())
        self._check(library().chisao_eval(self.ctx, prob, x.data_ptr(), n, f.data_ptr(),
                                          g.data_ptr() if g is not None else None, grad_mode), "chisao_eval")
        torch.cuda.current_stream().wait_stream(self._stream)
        return f, g

    def _check_points(self, prob: int, x):
        """The kernels read and write rows of exactly d binary32 values on the device."""
        import torch
        if not 0 <= prob < len(self.problems):
            raise ChisaoError(f"problem index {prob} out of range")
        d = self.problems[prob].d
        if not isinstance(x, torch.Tensor):
            raise ChisaoError("points must be a torch tensor")
        if not x.is_cuda:
            raise ChisaoError("points must be on the CUDA device")
        if x.dtype != torch.float32:
            raise ChisaoError(f"points must be float32, got {x.dtype}")
        if x.dim() != 2 or x.shape[1] != d:
            raise ChisaoError(f"points must have shape [n, {d}], got {tuple(x.shape)}")

    def synchronize(self):
        self._stream.synchronize()

    # ------------------------------------------------------------------ test hooks
    def layout(self, prob: int = 0):
        dp, mm = C.c_int32(0), C.c_int32(0)
        self._check(library().chisao_layout(self.ctx, prob, C.byref(dp), C.byref(mm)), "chisao_layout")
        return dp.value, mm.value

    def _field_shape(self, prob, field):
        pr = self.problems[prob]
        dp, mm = self.layout(prob)
        n = pr.n
        return {FIELD_X: ((n, dp), np.float32), FIELD_G: ((n, dp), np.float32), FIELD_F: ((n,), np.float32),
                FIELD_HS: ((n, mm, dp), np.float32), FIELD_HY: ((n, mm, dp), np.float32),
                FIELD_HRHO: ((n, mm), np.float32), FIELD_HLEN: ((n,), np.int32),
                FIELD_STUCK: (((n + 31) // 32,), np.uint32), FIELD_REMOVED: (((n + 31) // 32,), np.uint32)}[field]

    def get(self, prob: int, field: int) -> np.ndarray:
        shape, dt = self._field_shape(prob, field)
        a = np.empty(shape, dt)
        self._check(library().chisao_state_get(self.ctx, prob, field, a.ctypes.data, a.nbytes), "chisao_state_get")
        return a

    def set(self, prob: int, field: int, value: np.ndarray):
        shape, dt = self._field_shape(prob, field)
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(value, dtype=dt), shape))
        self._check(library().chisao_state_set(self.ctx, prob, field, a.ctypes.data, a.nbytes), "chisao_state_set")

    def run_phase(self, prob: int, phase: int, arg: int = 0):
        self._check(library().chisao_run_phase(self.ctx, prob, phase, arg), "chisao_run_phase")

    def set_gr_state(self, prob: int, enabled: int, noprog: int, prev_surv: int):
        self._check(library().chisao_set_gr_state(self.ctx, prob, enabled, noprog, prev_surv),
                    "chisao_set_gr_state")

    def set_tile(self, dp: int, ck: int):
        """Test hook: the components per step (2, 4, 8) of the grouped diagonal-mixture
        kernels of padded dimension dp."""
        self._check(library().chisao_set_tile(self.ctx, dp, ck), "chisao_set_tile")

    def close(self):
        if getattr(self, "ctx", None):
            library().chisao_destroy(self.ctx)
            self.ctx = None
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    b = np.unpackbits(words.view(np.uint8), bitorder="little")
    return b[:n].astype(bool)


def pack_bits(mask: np.ndarray) -> np.ndarray:
    n = mask.shape[0]
    nw = (n + 31) // 32
    b = np.zeros(nw * 32, np.uint8)
    b[:n] = mask.astype(np.uint8)
    return np.packbits(b, bitorder="little").view(np.uint32)


def _objective_function():
    """The torch.autograd.Function over the library's objective (built once)."""
    import torch

    class _ChisaoObjectiveFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, model, prob, xin):
            f, g = model.eval(prob, xin, GRAD_ADJOINT, want_grad=True)
            ctx.save_for_backward(g)
            return f

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return None, None, gout[:, None] * g

    return _ChisaoObjectiveFn


_OBJECTIVE_FN = None


class ChisaoObjective:
    """torch.autograd.Function over the library's objective: forward = the value
    f(x) of problem `prob` at the rows of x ([n, d] float32 on the device), backward =
    grad_output times the hand-written adjoint gradient (exact; the analytic-gradient
    alternative to finite differences of Sec. 3.1), both from one chisao_eval call."""

    @staticmethod
    def apply(model: Chisao, prob: int, x):
        global _OBJECTIVE_FN
        if _OBJECTIVE_FN is None:
            _OBJECTIVE_FN = _objective_function()
        model._check_points(prob, x)
        return _OBJECTIVE_FN.apply(model, prob, x)
