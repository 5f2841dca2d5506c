"""The C-ABI library builds for sm_103a, loads, and exports every function
include/chisao.h declares (no GPU needed: only host-side calls are made)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2606_26164_gb300 import build
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "chisao.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chisao_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return CH.library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(CH.EXPORTS) == names


def test_default_params_follow_table1(lib):
    p = CH.default_params()
    assert (p.n_osc, p.n_anti, p.n_cloud, p.m) == (3, 5, 3, 10)
    assert (p.eps_grad, p.eps_dup, p.delta, p.mu) == (1e-6, 1e-3, 0.1, 0.9)
    assert p.alpha == 0.0 and p.sigma == 0.0 and p.c_sigma == 0.1


def _cproblem(pr, keep):
    A = {k: np.ascontiguousarray(v, np.float64) for k, v in pr.objective.arrays.items()}
    lo, hi = np.ascontiguousarray(pr.lo), np.ascontiguousarray(pr.hi)
    x0 = np.ascontiguousarray(pr.x0)
    keep += [A, lo, hi, x0]
    dp = CH._dptr
    co = CH.CObjective(kind=pr.objective.kind, n_comp=pr.objective.n_comp, weights=dp(A.get("weights")),
                       means=dp(A.get("means")), sigmas=dp(A.get("sigmas")), chol=dp(A.get("chol")),
                       center=dp(A.get("center")), Q=dp(A.get("Q")), lam=dp(A.get("lam")))
    return CH.CProblem(d=pr.d, n=pr.n, lo=dp(lo), hi=dp(hi), x0=x0.ctypes.data_as(C.POINTER(C.c_float)), objective=co)


def test_arena_bytes_and_argument_checks(lib):
    keep = []
    pr = I.small_mixture(5, 3, 100, seed=0)
    probs = (CH.CProblem * 1)(_cproblem(pr, keep))
    p = CH.default_params()
    nb = C.c_size_t(0)
    assert lib.chisao_arena_bytes(probs, 1, C.byref(p), C.byref(nb)) == CH.OK
    # x, g (100 x 8 floats), histories (2 x 100 x 10 x 8 floats) dominate
    assert nb.value >= 4 * (2 * 100 * 8 + 2 * 100 * 10 * 8)
    bad = CH.default_params(m=11)
    assert lib.chisao_arena_bytes(probs, 1, C.byref(bad), C.byref(nb)) == CH.ERR_ARG
    bad = CH.default_params(delta=1.5)
    assert lib.chisao_arena_bytes(probs, 1, C.byref(bad), C.byref(nb)) == CH.ERR_ARG
    probs[0].d = 65
    assert lib.chisao_arena_bytes(probs, 1, C.byref(p), C.byref(nb)) == CH.ERR_ARG
    ctx = C.c_void_p()
    assert lib.chisao_create(probs, 1, C.byref(p), None, 0, None, C.byref(ctx)) == CH.ERR_ARG
    assert lib.chisao_init(probs, 1, C.byref(p), None, C.byref(ctx)) == CH.ERR_ARG
    assert lib.chisao_step(None) == CH.ERR_ARG
    assert lib.chisao_stats(None, 0, None) == CH.ERR_ARG


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the CUDA library absent the binding raises instead of
    computing anything another way."""
    monkeypatch.setattr(CH, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(CH, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        CH.library()
    with pytest.raises(RuntimeError):
        CH.default_params()


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "chisao.h"

int main(void) {
  chisao_params p;
  chisao_problem pr;
  double lo[3] = {-1, -1, -1}, hi[3] = {1, 1, 1};
  double center[3] = {0, 0, 0}, Q[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, lam[3] = {1, 2, 3};
  float x0[4 * 3] = {0};
  size_t nb = 0;
  chisao_status status;
  chisao_default_params(&p);
  memset(&pr, 0, sizeof pr);
  pr.d = 3;
  pr.n = 4;
  pr.lo = lo;
  pr.hi = hi;
  pr.x0 = x0;
  pr.objective.kind = CHISAO_OBJ_QUADRATIC;
  pr.objective.center = center;
  pr.objective.Q = Q;
  pr.objective.lam = lam;
  status = chisao_arena_bytes(&pr, 1, &p, &nb);
  printf("%d %d %d %zu\n", (int)status, p.n_osc, p.m, nb);
  p.m = CHISAO_MAX_MEMORY + 1;
  printf("%d\n", (int)chisao_arena_bytes(&pr, 1, &p, &nb));
  printf("%d\n", (int)chisao_step(NULL));
  return 0;
}
"""


def test_header_is_plain_c_and_the_library_links_from_c(lib, tmp_path):
    """The boundary is usable without Python or C++: the header compiles as strict
    C11 and a C program linked against the library makes host-side calls."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use_chisao.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_chisao"
    libdir = os.path.dirname(CH.LIB_PATH)
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-L", libdir, "-lchisao", f"-Wl,-rpath,{libdir}", "-Wl,--allow-shlib-undefined",
           "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split()
    status, n_osc, m, nbytes = (int(v) for v in lines[:4])
    assert (status, n_osc, m) == (CH.OK, 3, 10)
    # x, g (4 x 4 floats) and the histories (2 x 4 x 10 x 4 floats) at least
    assert nbytes >= 4 * (2 * 4 * 4 + 2 * 4 * 10 * 4)
    assert int(lines[4]) == CH.ERR_ARG and int(lines[5]) == CH.ERR_ARG


def test_eval_rejects_bad_points_before_any_launch(lib):
    """Chisao.eval / ChisaoObjective check dtype, device and shape on the host (the
    kernels read and write rows of exactly d binary32 values): a wrong input raises
    ChisaoError before the library is called."""
    import torch
    model = CH.Chisao.__new__(CH.Chisao)           # no device context needed for the checks
    model.problems = [I.small_mixture(5, 3, 10, seed=0)]
    calls = []

    class _Spy:
        def __getattr__(self, name):
            calls.append(name)
            raise AssertionError("the library must not be called")

    good = torch.zeros(4, 5, dtype=torch.float32)
    bad = [torch.zeros(4, 5, dtype=torch.float64), torch.zeros(4, 5, dtype=torch.bfloat16),
           torch.zeros(4, 4), torch.zeros(20), torch.zeros(4, 6), good, np.zeros((4, 5), np.float32)]
    orig = CH.library
    CH.library = lambda: _Spy()
    try:
        for x in bad:                                # CPU tensors fail the device test too
            with pytest.raises(CH.ChisaoError):
                model.eval(0, x)
            with pytest.raises(CH.ChisaoError):
                CH.ChisaoObjective.apply(model, 0, x)
        with pytest.raises(CH.ChisaoError):
            model.eval(3, good)
    finally:
        CH.library = orig
    assert calls == []
    model.ctx = None


def test_mma_rate_rejects_bad_arguments_before_any_launch(lib):
    """The tensor-core rate measurement checks its shape arguments on the host (no GPU
    needed to get CHISAO_ERR_ARG)."""
    out = C.c_double(0.0)
    for n, thr, ta in ((8, 1, 0), (272, 1, 0), (144, 2, 0), (80, 3, 0), (24, 1, 0), (16, 0, 0), (16, 5, 0),
                      (16, 2, 3), (16, 2, -1)):
        assert lib.chisao_measure_mma_rate(n, thr, ta, None, C.byref(out)) == CH.ERR_ARG, (n, thr, ta)
    assert lib.chisao_measure_mma_rate(16, 1, 0, None, None) == CH.ERR_ARG
