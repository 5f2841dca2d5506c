"""Strength of the oracle's pins: a single mistake planted in a scratch copy of the
oracle (on the CPU, never in the oracle itself) must make the pin suite
(tests/test_oracle_*.py) fail.  Each mutant is a plausible slip in one step of
Algorithm 1 -- a sign, a comparison, a wrong slot or divisor, a dropped factor --
and the unmutated copy must pass, so a failure is the mutant's doing."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name -> [(exact text, replacement), ...] in oracle/method.py, or in the module the
# name starts with ("objectives.py: ...")
MUTANTS = {
    "momentum sign (Eq. 6)": [("V = P.mu * V - alpha * G", "V = P.mu * V + alpha * G")],
    "dedup distance <= instead of < (Eq. 4)": [("close = D < eps", "close = D <= eps")],
    "gamma from the oldest slot instead of the newest pair": [
        ('sy = np.einsum("nd,nd->n", S[:, 0], Y[:, 0])', 'sy = np.einsum("nd,nd->n", S[:, -1], Y[:, -1])'),
        ('yy = np.einsum("nd,nd->n", Y[:, 0], Y[:, 0])', 'yy = np.einsum("nd,nd->n", Y[:, -1], Y[:, -1])')],
    "Hands Like Clouds step sign (Eq. 5)": [("X = np.clip(X + alpha * (acc / P.M)", "X = np.clip(X - alpha * (acc / P.M)")],
    "quality gate > instead of >= (Eq. 3)": [("(f >= thr)", "(f > thr)")],
    "Repulse Monkey ray twice as long": [("t = PX.u01(w[:, 1]) * ray_exit(", "t = PX.u01(w[:, 1]) * 2.0 * ray_exit(")],
    "Golden Rooster ray half as long": [("t = PX.u01(w[:, 0]) * ray_exit(", "t = PX.u01(w[:, 0]) * 0.5 * ray_exit(")],
    "Armijo sufficient-decrease sign": [("ok = Ft <= F[idx] + P.c1 *", "ok = Ft <= F[idx] - P.c1 *")],
    "sample instead of population variance in sigma": [
        ("var = ((X - mean[None, :]) ** 2).mean(axis=0)",
         "var = ((X - mean[None, :]) ** 2).sum(axis=0) / max(X.shape[0] - 1, 1)")],
    "g_rms over U instead of U d": [("float((G * G).sum()) / (U * prob.d))", "float((G * G).sum()) / U)")],
    "sigma without c_sigma": [("else P.c_sigma * s", "else s")],
    "Repulse Monkey only above five unfrozen": [("if U >= P.rm_min_unfrozen:", "if U > P.rm_min_unfrozen:")],
    "Golden Rooster sign never alternates": [
        ("sgn = np.where(((r // (S * d)) % 2) == 0, 1.0, -1.0)", "sgn = np.ones(K)")],
    "Hands Like Clouds reuses one draw in every step": [
        ("PX.TAG_HLC, cycle, t, prob_index, k)", "PX.TAG_HLC, cycle, 0, prob_index, k)")],
    "velocity kept on clamped coordinates": [("V = np.where(Xc != Xn, 0.0, V)", "V = V")],
    "curvature test sign": [("ok = (sy > P.curv_eps * nrm)", "ok = (sy > -P.curv_eps * nrm)")],
    "two-loop first recursion sign": [("q = q - ai[:, None] * Y[:, i]", "q = q + ai[:, None] * Y[:, i]")],
    "dedup tie-break to the higher index": [
        ("(idx[None, :] < idx[j0:j1, None])", "(idx[None, :] > idx[j0:j1, None])")],
    "rho = s^T y instead of its reciprocal": [("st.rho[j, 0] = 1.0 / sy[ok]", "st.rho[j, 0] = sy[ok]")],
    "trial points not projected onto the box": [
        ("Xt = np.clip(X[idx] + a[:, None] * Pd[idx], lo, hi)", "Xt = X[idx] + a[:, None] * Pd[idx]")],
    "refinement clears the kept history": [
        ("lbfgs_iterations(prob, sub, P, n_refine, fresh_gradient=True)",
         "sub.hlen[:] = 0\n    lbfgs_iterations(prob, sub, P, n_refine, fresh_gradient=True)")],
    "refinement moves every sample, not only the survivors": [
        ("idx = np.flatnonzero(st.stuck & ~st.removed)", "idx = np.arange(st.x.shape[0])")],
    "refinement keeps the stale gradient of the lower-precision objective": [
        ("lbfgs_iterations(prob, sub, P, n_refine, fresh_gradient=True)",
         "lbfgs_iterations(prob, sub, P, n_refine, fresh_gradient=False)")],
    "objectives.py: diagonal score without the square of sigma": [
        ("score = -R / (sig[None] ** 2)", "score = -R / sig[None]")],
    "objectives.py: Hessian without the mean-score term": [("return H - np.outer(gbar, gbar)", "return H")],
    "seeding.py: Carry Tiger face signs swapped": [
        ("np.where(q % 2 == 1, 1.0, -1.0)", "np.where(q % 2 == 1, -1.0, 1.0)")],
    "seeding.py: Carry Tiger edge frees the next axis": [
        ("E[edge, j[edge] % d] = 0.0", "E[edge, (j[edge] + 1) % d] = 0.0")],
    "philox.py: the two Box-Muller pairs share a word": [
        ("a01 = 2.0 * np.pi * u[..., 1]", "a01 = 2.0 * np.pi * u[..., 2]")],
    "philox.py: Philox multiplier": [("MUL0, MUL1 = 0xD2511F53, 0xCD9E8D57", "MUL0, MUL1 = 0xD2511F53, 0xCD9E8D55")],
    "modes.py: quality gate on delta instead of log delta": [
        ("if c[1] >= fmax + np.log(delta)]", "if c[1] >= fmax + delta]")],
    "benchmarks.py: Trid neighbour term sign": [
        ("+ (X[:, 1:] * X[:, :-1]).sum(axis=1)", "- (X[:, 1:] * X[:, :-1]).sum(axis=1)")],
}


def _scratch_copy(dst):
    ign = shutil.ignore_patterns("__pycache__", "*.pyc")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"), ignore=ign)
    pkg = os.path.join(dst, "paper_2606_26164_gb300")
    os.makedirs(pkg)
    for f in ("__init__.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, "paper_2606_26164_gb300", f), pkg)


def _plant(dst, name, edits):
    module = name.split(": ")[0] if ": " in name else "method.py"
    path = os.path.join(dst, "oracle", module)
    src = open(path).read()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation site not unique or missing: {old!r}"
        src = src.replace(old, new)
    open(path, "w").write(src)


def _pin_suite(dst):
    # the pins (the stored-values check in test_oracle_golden.py tests staleness, not arithmetic)
    tests = sorted(f for f in os.listdir(os.path.join(dst, "tests"))
                   if f.startswith("test_oracle_") and f.endswith(".py")
                   and f not in (os.path.basename(__file__), "test_oracle_golden.py"))
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    r = subprocess.run([sys.executable, "-m", "pytest", *[os.path.join("tests", t) for t in tests], "-x", "-q",
                        "-m", "not gpu", "-p", "no:cacheprovider"], cwd=dst, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_unmutated_copy_passes(tmp_path):
    _scratch_copy(str(tmp_path))
    rc, out = _pin_suite(str(tmp_path))
    assert rc == 0, out


@pytest.mark.parametrize("name", list(MUTANTS))
def test_each_planted_mistake_fails_a_pin(name, tmp_path):
    _scratch_copy(str(tmp_path))
    _plant(str(tmp_path), name, MUTANTS[name])
    rc, out = _pin_suite(str(tmp_path))
    assert rc == 1, f"mutant survived the pins ({name}):\n{out}"
