#!/usr/bin/env python
"""Benchmark of the ChiSao population step (one oscillation cycle = one step).

Default workload: the d=64 rotated ill-conditioned quadratic (Lambda from 1 to
1e4, c uniform in [-5, 5]^64) over N=65536 samples, FP32 state, m=10,
n_conv = max(10, 3 log2 d) = 18, exact (adjoint) gradients; every timed step
is a non-final cycle (Phases 1-6).  The same workload with central FD
gradients (FP64 stencil at h=1e-5) is timed beside it.

Prints one JSON line.  Under torchrun every rank runs an independent replica
population (its own seed): the work per GPU is fixed (weak scaling) and the
reported value is the sum over ranks of samples x cycles divided by the
slowest rank's time.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KERNELS_PER_STEP = 22   # kernel launches in one non-final cycle of one problem
FP32_LANES_PER_SM = 128
N_SM = 152
SM_MHZ_NOMINAL = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="quadratic_d64")
    ap.add_argument("--grad", default="adjoint", choices=["adjoint", "fd64", "fd32", "adjoint_tc"])
    ap.add_argument("--fd-steps", type=int, default=2)
    ap.add_argument("--n", type=int, default=0, help="override the population size (profiling cases)")
    ap.add_argument("--tc-steps", type=int, default=2, help="cycles of the full-covariance tensor-core leg")
    ap.add_argument("--batched-steps", type=int, default=3, help="cycles of the 512-problem leg")
    ap.add_argument("--bench-fn-steps", type=int, default=3, help="cycles of each benchmark-function leg")
    ap.add_argument("--noise-trials", type=int, default=10, help="trials per level of the noise-table leg")
    ap.add_argument("--leg", default=None, choices=["batched512", "noise_d6", "benchmark_functions", "mixture4_d2",
                                                    "mixture32_d16", "mixture256_d64"],
                    help="run only this leg (one JSON line; for profiling one workload)")
    ap.add_argument("--no-extras", action="store_true", help="skip the FD, e2e, kernel and CPU legs")
    ap.add_argument("--no-small-legs", dest="small_legs", action="store_false",
                    help="skip the d = 2 and d = 16 workload legs")
    ap.add_argument("--cpu-leg", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


GRAD = {"fd64": 0, "fd32": 1, "adjoint": 2, "adjoint_tc": 3}


def launches_per_step(params, tc, d):
    """Kernel launches in one non-final cycle of one problem."""
    if not tc:
        return KERNELS_PER_STEP
    n_conv = params.n_conv or max(10, int(np.ceil(3 * np.log2(d))))
    rounds = 1 + -(-(params.T_ls - 1) // 4)          # line-search rounds: 1 trial, then 4 at a time
    # cycle begin + first evaluation, per L-BFGS iteration one direction kernel and one
    # (evaluation, acceptance) pair per round, the history rotation, freeze (3) / dedup (6) /
    # reseed (4), HLC and anti with their scale passes, cycle end
    return (2 + n_conv * (1 + 2 * rounds) + 1 + 13 + (3 + 3 * params.n_cloud)
            + (2 + 2 * params.n_anti) + 1)


def make_problem(name, seed):
    from paper_2606_26164_gb300 import inputs as I
    return I.WORKLOADS[name](seed=seed)


# --------------------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- helpers

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


GOLDEN = os.path.join(ROOT, "tests", "golden")


def stored_modes(workload):
    """The significant modes of a workload's objective and -Hess f there, as stored by
    tests/golden/make_modes.py (FP64 Newton from every component mean; read here, not
    computed)."""
    p = os.path.join(GOLDEN, f"modes_{workload}.npz")
    if not os.path.exists(p):
        return None
    z = np.load(p)
    return z["x"], z["neg_hess"]


def recovery_of(found, workload, rel=1e-3):
    """Recovered fraction of the stored significant modes (a returned point within
    `rel` of the mode's local sigma: Mahalanobis distance under -Hess f at the mode) and
    the worst matched error in local sigmas."""
    m = stored_modes(workload)
    if m is None:
        return None
    mx, negH = m
    found = np.asarray(found, np.float64).reshape(-1, mx.shape[1])
    best = np.full(mx.shape[0], np.inf)
    for k, (x, H) in enumerate(zip(mx, negH)):
        if found.shape[0]:
            D = found - x[None, :]
            best[k] = float(np.sqrt(np.maximum(np.einsum("nd,de,ne->n", D, H, D), 0.0)).min())
    hit = best <= rel
    return {"significant_modes": int(mx.shape[0]), "recovered": float(hit.mean()),
            "worst_error_sigma": float(best[hit].max()) if hit.any() else None, "returned": int(found.shape[0])}


def kernel_source_hash():
    h = hashlib.sha1()
    for f in ("obj_kernels.cuh", "objectives.cuh", "dev_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2606_26164_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` recorded in profiles/*.md, if the
    recorded source hash matches the current kernel source."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    cur = kernel_source_hash()
    for f in sorted(os.listdir(pdir)):
        if not f.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, f)).read()
        m = re.search(r"traffic_bytes_per_launch\[%s\]:\s*([0-9.eE+]+)\s+source_hash:\s*(\w+)" % kernel, txt)
        if m and m.group(2) == cur:
            return float(m.group(1))
    return None


def dist_setup():
    """Ranks from the torchrun environment; NCCL when there is a GPU, gloo otherwise."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def allmax(v, world):
    """The largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank, steps, world, t_max):
    """Whole-job throughput of independent replicas (weak scaling): every rank's
    samples x cycles over the slowest rank's time."""
    return n_per_rank * steps * world / t_max


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- CPU oracle leg

def cpu_leg(spec):
    """Time the FP64 oracle on a bounded sample of the workload (run in a child
    process with single-threaded BLAS so `cores` is exact)."""
    a = json.loads(spec)
    from oracle import method as M
    prob = make_problem(a["workload"], a["seed"])
    from paper_2606_26164_gb300 import inputs as I
    rows = np.arange(a.get("offset", 0), a.get("offset", 0) + a["sample_n"]) % prob.n
    sub = I.Problem(prob.d, rows.size, prob.lo, prob.hi, prob.objective, prob.x0[rows], prob.eps_grad,
                    prob.sigma_mode)
    P = M.Params(n_osc=10 ** 6, m=10, eps_grad=prob.eps_grad, grad_mode=GRAD[a["grad"]], seed=a["seed"])
    st = M.new_state(sub.x0, P.m)
    t0 = time.perf_counter()
    cycles = 0
    times = []
    while True:
        c0 = time.perf_counter()
        M.cycle(sub, st, P, last=False)
        times.append(time.perf_counter() - c0)
        cycles += 1
        if time.perf_counter() - t0 >= a["budget_s"] or cycles >= a.get("max_cycles", 10 ** 6):
            break
    el = time.perf_counter() - t0
    return {"value": rows.size * cycles / el, "cycles": cycles, "seconds": el, "evals": st.evals,
            "evals_per_s": st.evals / el, "step_times": times}


def run_cpu_leg(workload, grad, seed, sample_n, budget_s, max_cycles=10 ** 6):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    spec = json.dumps({"workload": workload, "grad": grad, "seed": seed, "sample_n": sample_n,
                       "budget_s": budget_s, "max_cycles": max_cycles})
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", spec], env=env,
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_cpu_legs_all_cores(workload, grad, sample_n, budget_s):
    """The oracle on every host core at once: one single-threaded process per core,
    each on its own slice of the same workload; aggregate samples x cycles / the
    longest process's time."""
    n = os.cpu_count() or 1
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = []
    for k in range(n):
        spec = json.dumps({"workload": workload, "grad": grad, "seed": 0, "sample_n": sample_n,
                           "offset": k * sample_n, "budget_s": budget_s})
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-leg", spec], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    res = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    t = max(r["seconds"] for r in res)
    work = sum(sample_n * r["cycles"] for r in res)
    return {"value": work / t, "cores": n, "cycles_per_process": [r["cycles"] for r in res], "seconds": t,
            "evals_per_s": sum(r["evals"] for r in res) / t}


# --------------------------------------------------------------------------- GPU legs

def gpu_timed(model, steps, warmup):
    import torch
    for _ in range(warmup):
        model.step()
    model.synchronize()
    c0 = model.counters(0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(model._stream)
    ranged = nvtx_push("timed")                        # a profiler can select the timed launches
    for _ in range(steps):
        model.step()
    e1.record(model._stream)
    if ranged:
        torch.cuda.nvtx.range_pop()
    e1.synchronize()
    c1 = model.counters(0)
    return e0.elapsed_time(e1) / 1e3, c0, c1


def nvtx_push(name):
    """Open an NVTX range (no-op where the profiler markers are unavailable)."""
    import torch
    try:
        torch.cuda.nvtx.range_push(name)
        return True
    except Exception:
        return False


def tc_executed_flop_per_point(d, K):
    """Tensor-core flop the kernel issues per point (2 per multiply-add), per group of
    two components over the padded dimension 64 in four 16-wide slabs: Z over the split
    input, input K-chunk c meeting the rows of slabs >= c (N = 32 (4 - c)), twice; the
    bias block (K = 16, N = 128); G = Y V, y K-chunk c meeting the outputs of slabs <= c
    (N = 16 (c + 1)), per component."""
    z = 2 * sum(32 * (4 - c) * 16 for c in range(4)) + 128 * 16
    gr = 2 * sum(16 * (c + 1) * 16 for c in range(4))
    return 2 * (z + gr) * ((K + 1) // 2)


def events_time(stream, fn):
    """Device time of fn()'s work on `stream` (CUDA events on that stream)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_and_score(CH, prob, workload, prm, cycles, warm=True):
    """A whole run of `cycles` cycles (the last one final) from the workload's population:
    device time of the non-final cycles and of the final one, evaluations, and the
    recovery of the stored significant modes.  With `warm`, a first run captures the
    cycle graphs so the timed run replays them."""
    model = CH.Chisao([prob], prm)
    if warm:
        for _ in range(cycles):
            model.step()
        model.modes(0)
        model.load_population(0, prob.x0)
    c0 = model.counters(0)
    t_nf = events_time(model._stream, lambda: [model.step() for _ in range(cycles - 1)]) if cycles > 1 else 0.0
    c1 = model.counters(0)
    t_last = events_time(model._stream, model.step)
    c2 = model.counters(0)
    fx, _ = model.modes(0)
    model.close()
    nf = max(cycles - 1, 1)
    return {"value": prob.n * (cycles - 1) / t_nf if cycles > 1 else None, "unit": "sample-cycles/s",
            "ms_per_step": 1e3 * t_nf / nf if cycles > 1 else None, "final_cycle_ms": 1e3 * t_last,
            "evals_per_s": (c1["evals"] - c0["evals"]) / t_nf if cycles > 1 else None,
            "run_ms": 1e3 * (t_nf + t_last), "run_evals": int(c2["evals"] - c0["evals"]),
            "stuck_last_cycle": int(c2["n_stuck"]), "k_lost_last_cycle": int(c2["k_lost"]),
            "recovery": recovery_of(fx, workload)}


def full_covariance_leg(CH, steps, n_osc, fp32_peak_tf):
    """cfg 4, d = 64, K = 256 full-covariance mixture: throughput of the BF16 tensor-core
    cycle and of the FP32 (SIMT adjoint) cycle at N = 65536, the tensor-core objective
    against the measured BF16 peak and against the exact FP64 mixture, and the three
    forms (tensor cores + FP32 refinement, FP32 adjoint, FP32 central differences) at
    matched mode-location error on the same 1024 rows."""
    import torch
    prob = make_problem("mixture256_d64", 0)
    N, d, K = prob.n, prob.d, prob.objective.n_comp
    res = {"N": N, "d": d, "K": K}
    for mode, label, nsteps in ((CH.GRAD_ADJOINT_TC, "bf16_tensor_core", steps), (CH.GRAD_ADJOINT, "fp32", 1)):
        prm = CH.default_params(n_osc=n_osc, m=10, eps_grad=prob.eps_grad, grad_mode=mode, seed=0)
        m4 = CH.Chisao([prob], prm)
        t, c0, c1 = gpu_timed(m4, nsteps, 1)
        ev = (c1["evals"] - c0["evals"]) / t
        res[label] = {"value": N * nsteps / t, "unit": "sample-cycles/s", "ms_per_step": 1e3 * t / nsteps,
                      "evals_per_s": ev, "steps": nsteps, "stuck_last_cycle": int(c1["n_stuck"]),
                      "k_lost_last_cycle": int(c1["k_lost"])}
        if mode == CH.GRAD_ADJOINT:
            # every evaluation of the SIMT adjoint path is a value and a gradient: two
            # triangular contractions d (d + 1) K each (the dense rows it walks: 4 d^2 K)
            alg = ev * 2 * d * (d + 1) * K / 1e12
            res[label]["roofline"] = {"bound": "alu", "achieved": alg, "peak": fp32_peak_tf, "unit": "TFLOP/s",
                                      "frac": alg / fp32_peak_tf if fp32_peak_tf else None,
                                      "executed_tflops": ev * 4 * d * d * K / 1e12,
                                      "peak_source": "measured FP32 FMA throughput"}
        if mode == CH.GRAD_ADJOINT_TC:
            x = torch.from_numpy(prob.x0).cuda()
            m4.eval(0, x, mode)
            reps = 5
            tk = events_time(m4._stream, lambda: [m4.eval(0, x, mode) for _ in range(reps)]) / reps
            # algorithmic work (triangular factors): d (d + 1) K for the value's contraction
            # and the same again for the adjoint's, 2 flop per multiply-add
            flop = N * 2 * d * (d + 1) * K
            dense = N * (2 * d * (d * K) + 2 * (d * K) * d)
            executed = N * tc_executed_flop_per_point(d, K)
            _, bf16_peak, src = peaks()
            res["roofline_tc"] = {"kernel": "k_tc_mixfull<true>", "bound": "tensor", "achieved": flop / tk / 1e12,
                                  "peak": bf16_peak, "unit": "TFLOP/s", "frac": flop / tk / 1e12 / bf16_peak,
                                  "count": "triangular: 2 d (d + 1) K flop per value and gradient",
                                  "dense_tflops": dense / tk / 1e12, "dense_frac": dense / tk / 1e12 / bf16_peak,
                                  "executed_tflops": executed / tk / 1e12,
                                  "peak_source": f"{src} bf16 dense (MEASURED_PEAKS.json burst)",
                                  "launch_ms": 1e3 * tk, "points_per_launch": N}
            # the instruction-rate floor: a group of two components issues 17 small MMAs
            # (M = 128, K = 16: nine for Z, eight for the gradient), which the tensor core takes
            # at a measured rate whatever their width; one CTA per SM, waves of whole tiles
            clk4 = CH.measure_mma_rate(64, 4, 2)
            clk1 = CH.measure_mma_rate(64, 1, 0)
            waves = -(-(-(-N // 128)) // N_SM)
            floor_ms = waves * ((K + 1) // 2) * 17 * clk4 / (SM_MHZ_NOMINAL * 1e3)
            res["roofline_tc"]["mma_rate_floor"] = {
                "clk_per_mma_4_issuers": clk4, "clk_per_mma_1_issuer": clk1, "mmas_per_group": 17,
                "waves": waves, "floor_ms": floor_ms, "frac": floor_ms / (1e3 * tk),
                "basis": "measured clocks per tcgen05.mma (N = 64, four issuers, two reading A from TMEM) "
                         "x 17 per group x groups x waves at the nominal 2070 MHz"}
            res["tc_error_vs_exact"] = tc_error_vs_exact(CH, m4)
        m4.close()
    res["matched_error"] = matched_error_forms(CH)
    return res


def tc_error_vs_exact(CH, model):
    """The tensor-core objective (BF16 factors, split input) and the FP32 SIMT adjoint
    against the exact FP64 mixture at 256 stored rows of the population
    (tests/golden/exact_mixture256_d64.npz): value error |f - f*| and gradient error
    |g - g*|_inf / |g*|_inf, max and median over the points."""
    import torch
    p = os.path.join(GOLDEN, "exact_mixture256_d64.npz")
    if not os.path.exists(p):
        return None
    z = np.load(p)
    x = torch.from_numpy(z["x"].astype(np.float32)).cuda()
    out = {"points": int(z["x"].shape[0])}
    for mode, label in ((CH.GRAD_ADJOINT_TC, "bf16_tensor_core"), (CH.GRAD_ADJOINT, "fp32_adjoint")):
        f, g = model.eval(0, x, mode)
        f = f.cpu().numpy().astype(np.float64)
        g = g.cpu().numpy().astype(np.float64)
        fe = np.abs(f - z["f"])
        ge = np.abs(g - z["g"]).max(axis=1) / np.maximum(np.abs(z["g"]).max(axis=1), 1e-300)
        out[label] = {"value_abs_max": float(fe.max()), "value_abs_median": float(np.median(fe)),
                      "grad_rel_max": float(ge.max()), "grad_rel_median": float(np.median(ge))}
    return out


def matched_error_forms(CH, n_rows=1024, n_conv=100, cycles=2):
    """cfg 4's forms on the same first n_rows samples, n_conv = 100 and 2 cycles (enough
    for every significant mode to stick): each form's whole-run device time and the
    recovery (fraction of significant modes within 1e-3 local sigma, worst error)."""
    from paper_2606_26164_gb300 import inputs as I
    prob = I.mixture256_d64(n=n_rows)
    out = {"N": n_rows, "n_conv": n_conv, "cycles": cycles}
    forms = (("bf16_tensor_core_refined", CH.GRAD_ADJOINT_TC, 10, True),
             ("fp32_adjoint", CH.GRAD_ADJOINT, 0, True),
             ("fp32_central_differences", CH.GRAD_FD32, 0, False))
    for label, mode, n_refine, warm in forms:
        prm = CH.default_params(n_osc=cycles, n_conv=n_conv, m=10, eps_grad=prob.eps_grad, grad_mode=mode,
                                seed=4, n_refine=n_refine)
        r = run_and_score(CH, prob, "mixture256_d64", prm, cycles, warm=warm)
        out[label] = {"run_ms": r["run_ms"], "run_evals": r["run_evals"], "recovery": r["recovery"]}
    return out


def mixture4_d2_leg(CH):
    """cfg 1, the plain method at d = 2: K = 4 isotropic mixture, N = 1024, FD64
    (h = 1e-5), m = 5, 50 cycles.  The state is L2-resident and each cycle is a few
    dozen short kernels, so the leg reports microseconds per cycle with the per-cycle
    CUDA graph and without it (every kernel launched from the host), the host time of
    one chisao_step call, and the recovery after the 50 cycles."""
    from paper_2606_26164_gb300 import inputs as I
    prob = I.mixture4_d2()
    out = {"N": prob.n, "d": 2, "K": 4, "grad": "fd64", "m": 5, "cycles": 50}
    for use_graph in (1, 0):
        prm = CH.default_params(n_osc=50, m=5, eps_grad=1e-5, grad_mode=GRAD["fd64"], seed=0, use_graph=use_graph)
        model = CH.Chisao([prob], prm)
        for _ in range(50):
            model.step()
        model.modes(0)
        model.load_population(0, prob.x0)
        model.synchronize()
        host = []

        def run():
            for _ in range(50):
                h0 = time.perf_counter()
                model.step()
                host.append(time.perf_counter() - h0)
        t = events_time(model._stream, run)
        fx, _ = model.modes(0)
        c = model.counters(0)
        model.close()
        out["graph" if use_graph else "no_graph"] = {
            "us_per_cycle": 1e6 * t / 50, "value": prob.n * 50 / t, "unit": "sample-cycles/s",
            "host_us_per_step_call": 1e6 * float(np.median(host)), "recovery": recovery_of(fx, "mixture4_d2"),
            "stuck_last_cycle": int(c["n_stuck"]), "k_lost_last_cycle": int(c["k_lost"])}
    return out


def mixture32_d16_leg(CH):
    """cfg 2, d = 16, K = 32 diagonal mixture, N = 16384, the Table 1 schedule (3 cycles,
    n_conv = 12): central differences (FP64 stencil, h = 1e-5) against exact gradients,
    each without noise and with N(0, sigma_noise^2) added to every evaluation
    (sigma_noise = 0.1, 1.0).  Throughput of the two non-final cycles, the final cycle's
    time, and the recovery of the run."""
    from paper_2606_26164_gb300 import inputs as I
    out = {"N": 16384, "d": 16, "K": 32, "cycles": 3, "eps_grad": 1e-4}
    for grad in ("adjoint", "fd64"):
        for noise in (0.0, 0.1, 1.0):
            prob = I.mixture32_d16(noise_sigma=noise)
            prm = CH.default_params(n_osc=3, m=10, eps_grad=1e-4, grad_mode=GRAD[grad], seed=2)
            out[f"{grad}_noise{noise:g}"] = run_and_score(CH, prob, "mixture32_d16", prm, 3)
    return out


def batched_leg(CH, steps):
    """512 independent diagonal-mixture problems (d in {2..64}, N log-uniform in
    [256, 16384], K in [4, 128]) in one context: one step = one non-final cycle of all."""
    from paper_2606_26164_gb300 import inputs as I
    probs = I.batched512()
    prm = CH.default_params(n_osc=10 ** 6, m=10, eps_grad=1e-3, grad_mode=GRAD["adjoint"], seed=0)
    model = CH.Chisao(probs, prm)
    model.step()                                       # a first cycle, then the launch shape is tuned on it
    tune = model.autotune(cycles_per_trial=1)
    t, _, _ = gpu_timed(model, steps, 1)
    n_total = sum(p.n for p in probs)
    model.close()
    # kernel launches of one non-final cycle: grouped, the objective-independent steps of all
    # problems are one launch per kernel (begin 1, freeze 3, dedup 5 + one per padded
    # dimension, reseed 3 + one per padded dimension, end 1) and each (kind, padded dimension)
    # group runs Phase 1 (1) and Phases 5-6 with their scale passes (6); per problem, every
    # problem launches the single-problem cycle
    pads = {max(4, 1 << (p.d - 1).bit_length()) for p in probs}
    launches = (13 + 7 * len(pads) + 2 * len(pads)) if tune["grouped"] else KERNELS_PER_STEP * len(probs)
    return {"problems": len(probs), "samples": n_total, "value": n_total * steps / t, "unit": "sample-cycles/s",
            "ms_per_step": 1e3 * t / steps, "steps": steps, "grad": "adjoint", "autotune": tune,
            "launches_per_cycle": launches}


def benchmark_functions_leg(CH, steps, n_osc):
    """The Appendix D benchmark functions at d = 64 (Bukin N.6: d = 2), N = 65536,
    exact gradients: samples x cycles per second and evaluations per second."""
    from paper_2606_26164_gb300 import inputs as I
    res = {}
    for name in I.BENCHMARK_KINDS:
        d = 2 if name == "bukin6" else 64
        prob = I.benchmark(name, d, 65536, seed=0)
        prm = CH.default_params(n_osc=n_osc, m=10, eps_grad=prob.eps_grad, grad_mode=GRAD["adjoint"], seed=0)
        model = CH.Chisao([prob], prm)
        t, c0, c1 = gpu_timed(model, steps, 2)
        res[f"{name}_d{d}"] = {"value": prob.n * steps / t, "unit": "sample-cycles/s", "ms_per_step": 1e3 * t / steps,
                               "evals_per_s": (c1["evals"] - c0["evals"]) / t}
        model.close()
    return res


def noise_table_leg(CH, trials):
    """The Sec. 5.6 noise workload (d = 6, unit components at +-2 e_1, N = 2048) at
    each noise level of its table, exact gradients, 3 cycles per trial: how often both
    peaks are returned, the mean L2 error of the returned peaks, spurious returns and
    the device time of a whole run (its three cycles, the first one's graph capture
    included; context creation excluded).  The true peaks are
    +-x* e_1 with x* = 2 tanh(2 x*) (the stationarity condition along e_1)."""
    import torch
    from paper_2606_26164_gb300 import inputs as I
    xs = 2.0
    for _ in range(50):                                    # Newton on x - 2 tanh(2x) = 0
        t = np.tanh(2 * xs)
        xs -= (xs - 2 * t) / (1 - 4 * (1 - t * t))
    peaks_true = np.zeros((2, 6))
    peaks_true[0, 0], peaks_true[1, 0] = xs, -xs
    rows = []
    for noise in I.NOISE_LEVELS:
        both = spurious = 0
        errs, ms = [], []
        for seed in range(trials):
            prob = I.mixture2_d6(n=2048, seed=seed, noise_sigma=noise)
            prm = CH.default_params(n_osc=3, m=10, eps_grad=prob.eps_grad, grad_mode=GRAD["adjoint"], seed=seed)
            model = CH.Chisao([prob], prm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(model._stream)
            for _ in range(3):
                model.step()
            e1.record(model._stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            fx, _ = model.modes(0)
            model.close()
            dist = np.abs(fx[:, None, :].astype(np.float64) - peaks_true[None]).max(axis=2)   # L-inf
            hit = dist.min(axis=0) <= 1e-3
            both += int(hit.all())
            matched = dist.min(axis=1) <= 1e-3
            spurious += int((~matched).sum())
            for k in range(2):
                if hit[k]:
                    errs.append(float(np.linalg.norm(fx[dist[:, k].argmin()] - peaks_true[k])))
        rows.append({"sigma_noise": noise, "both_found": f"{both}/{trials}", "spurious": spurious,
                     "mean_peak_error_l2": float(np.mean(errs)) if errs else None,
                     "ms_per_run": float(np.median(ms))})
    return {"d": 6, "N": 2048, "cycles": 3, "grad": "adjoint", "trials": trials, "levels": rows}


def main():
    args = parse()
    if args.cpu_leg:
        print(json.dumps(cpu_leg(args.cpu_leg)))
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import torch
    torch.cuda.set_device(local)
    from paper_2606_26164_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    barrier(world)
    from paper_2606_26164_gb300 import chisao as CH

    if args.leg:
        legs = {"batched512": lambda: batched_leg(CH, args.batched_steps),
                "noise_d6": lambda: noise_table_leg(CH, args.noise_trials),
                "benchmark_functions": lambda: benchmark_functions_leg(CH, args.bench_fn_steps, 2),
                "mixture4_d2": lambda: mixture4_d2_leg(CH),
                "mixture32_d16": lambda: mixture32_d16_leg(CH),
                "mixture256_d64": lambda: full_covariance_leg(CH, args.tc_steps, 10 ** 6,
                                                              CH.measure_fma_peak(False) / 1e12)}
        print(json.dumps({"leg": args.leg, **legs[args.leg]()}))
        return
    prob = make_problem(args.workload, seed=rank)
    if args.n:
        from paper_2606_26164_gb300 import inputs as I
        prob = I.Problem(prob.d, args.n, prob.lo, prob.hi, prob.objective, prob.x0[:args.n], prob.eps_grad,
                         prob.sigma_mode)
    N, d = prob.n, prob.d
    gm = GRAD[args.grad]
    n_osc = 10 ** 6                      # every timed cycle is a non-final cycle
    params = CH.default_params(n_osc=n_osc, m=10, eps_grad=prob.eps_grad, grad_mode=gm, seed=rank)
    model = CH.Chisao([prob], params)
    n_conv = max(10, int(np.ceil(3 * np.log2(d))))

    barrier(world)
    clk = Clocks(local)
    clk.start()
    t, c0, c1 = gpu_timed(model, args.steps, args.warmup)
    clocks = clk.stop()
    t_max = allmax(t, world)
    value = job_value(N, args.steps, world, t_max)
    evals = (c1["evals"] - c0["evals"]) * world / t_max
    grads = (c1["grads"] - c0["grads"]) * world / t_max

    out = {"metric": f"sample-cycles/s ({args.grad} gradients) at N={N}, d={d}", "value": value,
           "unit": "sample-cycles/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "N": N, "d": d, "m": 10, "n_conv": n_conv,
                      "objective": "rotated quadratic, Lambda 1..1e4" if args.workload == "quadratic_d64" else args.workload,
                      "grad": args.grad, "parallelism": f"replicas x{world}",
                      "l2": "inputs larger than L2: per-step state (x, g, m=10 history) "
                            f"{(2 * N * d * 4 + 2 * N * 10 * d * 4 + N * 80) / 1e6:.0f} MB > 129 MB"},
           "evals_per_s": evals, "grads_per_s": grads,
           "gpu_launches": launches_per_step(params, gm == GRAD["adjoint_tc"], d) * args.steps,
           "clocks": clocks,
           # what the timed cycles left: samples stuck after the last dedup, and removed by it
           "stuck_last_cycle": int(c1["n_stuck"]), "k_lost_last_cycle": int(c1["k_lost"]),
           "n_unfrozen_last_cycle": int(c1["n_unfrozen"])}
    if rank == 0:
        out["recovery"] = {"timed_schedule": recovery_of(model.modes(0)[0], args.workload)}

    if gm == GRAD["adjoint_tc"]:
        args.no_extras = True            # the kernel, FD, e2e and CPU legs time the FP32 path
    if not args.no_extras and rank == 0:
        # --- dominant kernel: Phase 1 (fused L-BFGS) alone, CUDA events on the context stream
        reps = 5
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        model.load_population(0, prob.x0)
        k0 = model.counters(0)
        e0.record(model._stream)
        for _ in range(reps):
            model.run_phase(0, CH.PHASE_LBFGS, n_conv)
        e1.record(model._stream)
        e1.synchronize()
        k1 = model.counters(0)
        t_k = e0.elapsed_time(e1) / 1e3 / reps
        ev_k = (k1["evals"] - k0["evals"]) / reps
        # FLOPs per objective evaluation of the quadratic (value and gradient from one
        # d x d matrix-vector product): 2 d^2 + 4 d; per L-BFGS iteration the two-loop
        # and the update take 8 m d + 8 d.
        flop = ev_k * (2 * d * d + 4 * d) + N * n_conv * (8 * 10 * d + 8 * d)
        mhz = clocks.get("sm_mhz") or 1900.0
        nominal_tf = N_SM * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        # the denominator: FMA throughput measured on this GPU now (packed binary32 FMAs,
        # independent chains on every SM), the nominal unit count x clock beside it
        measured_tf = CH.measure_fma_peak(False, model._stream) / 1e12
        peak_tf = measured_tf
        achieved_tf = flop / t_k / 1e12
        out["roofline"] = {"kernel": "k_phase1", "bound": "alu", "achieved": achieved_tf, "peak": peak_tf,
                           "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                           "traffic": profiled_traffic("k_phase1"),
                           "peak_source": "measured FP32 FMA throughput (chisao_measure_fma_peak: packed FMAs, "
                                          "8 independent chains per thread, 8 blocks of 256 per SM)",
                           "peak_nominal": nominal_tf,
                           "peak_nominal_source": f"{N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 x {mhz:.0f} MHz "
                                                  "(sampled clock)",
                           "fp64_peak_measured": CH.measure_fma_peak(True, model._stream) / 1e12,
                           "launch_ms": 1e3 * t_k, "evals_per_launch": ev_k,
                           "limiter": "the latency of each warp's serial chain (20 dependent group reductions per "
                                      "two-loop recursion, the line search's reductions) at the 20 warps per SM "
                                      "that 96 registers and the 45 KB shared-memory history ring allow: issue "
                                      "54 %, the L1 / shared-memory path 74 % busy under ncu; moving the history "
                                      "into tensor memory took that path to 46 % but the launch got slower (16 "
                                      "warps per SM); profiles/k_phase1_quadratic_d64.md"}
        # --- recovery at a schedule long enough to converge (Prop. 1): one cycle of
        #     n_conv = 2500 on the whole population (the quadratic's mode is its centre)
        if args.workload == "quadratic_d64":
            pc = CH.default_params(n_osc=1, n_conv=2500, m=10, eps_grad=1e-2, grad_mode=gm, seed=3)
            r = run_and_score(CH, prob, args.workload, pc, 1, warm=False)
            out["recovery"]["n_conv_2500_one_cycle"] = {**r["recovery"], "run_ms": r["run_ms"],
                                                        "eps_grad": 1e-2}
        # --- FD leg: the plain form (central differences, FP64 stencil, h = 1e-5)
        fd = CH.default_params(n_osc=n_osc, m=10, eps_grad=prob.eps_grad, grad_mode=CH.GRAD_FD64, seed=rank)
        mfd = CH.Chisao([prob], fd)
        tf, f0, f1 = gpu_timed(mfd, args.fd_steps, 1)
        out["fd64"] = {"value": N * args.fd_steps / tf, "unit": "sample-cycles/s",
                       "evals_per_s": (f1["evals"] - f0["evals"]) / tf, "ms_per_step": 1e3 * tf / args.fd_steps,
                       "steps": args.fd_steps, "stuck_last_cycle": int(f1["n_stuck"]),
                       "k_lost_last_cycle": int(f1["k_lost"]),
                       "recovery_timed_schedule": recovery_of(mfd.modes(0)[0], args.workload)}
        if args.workload == "quadratic_d64":
            # every evaluation of the FD64 cycle is one binary64 value of the quadratic: u = A r
            # and r^T u, 2 d^2 + 2 d FLOP; against the measured binary64 FMA throughput
            fp64_peak = out["roofline"]["fp64_peak_measured"]
            ach = out["fd64"]["evals_per_s"] * (2 * d * d + 2 * d) / 1e12
            out["fd64"]["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                       "frac": ach / fp64_peak, "peak_source": "measured FP64 FMA throughput"}
        mfd.close()
        # --- the same FD cycle with the value-only smoothing estimator in Phase 5 (a variant:
        #     M + 1 evaluations per smoothing step instead of M central-difference gradients)
        fd.hlc_value_only = 1
        mfv = CH.Chisao([prob], fd)
        tv, v0, v1 = gpu_timed(mfv, args.fd_steps, 1)
        out["fd64_value_only_hlc"] = {"value": N * args.fd_steps / tv, "unit": "sample-cycles/s",
                                      "evals_per_s": (v1["evals"] - v0["evals"]) / tv,
                                      "ms_per_step": 1e3 * tv / args.fd_steps, "steps": args.fd_steps}
        mfv.close()
        # --- the d=64, K=256 full-covariance mixture at N=65536: BF16 tensor-core cycle vs FP32 cycle,
        #     and the tensor-core objective kernel against the measured BF16 peak
        if args.workload == "quadratic_d64" and args.tc_steps > 0:
            out["mixture256_d64"] = full_covariance_leg(CH, args.tc_steps, n_osc, peak_tf)
        # --- cfg 1 (d = 2, the plain method, 50 cycles) and cfg 2 (d = 16, FD vs adjoint, noise)
        if args.workload == "quadratic_d64" and args.small_legs:
            out["mixture4_d2"] = mixture4_d2_leg(CH)
            out["mixture32_d16"] = mixture32_d16_leg(CH)
        # --- 512 problems of uneven size in one context (cycle graph with one branch per stream)
        if args.workload == "quadratic_d64" and args.batched_steps > 0:
            out["batched512"] = batched_leg(CH, args.batched_steps)
        # --- the Appendix D benchmark functions
        if args.workload == "quadratic_d64" and args.bench_fn_steps > 0:
            out["benchmark_functions"] = benchmark_functions_leg(CH, args.bench_fn_steps, n_osc)
        # --- the Sec. 5.6 noise table workload
        if args.workload == "quadratic_d64" and args.noise_trials > 0:
            out["noise_d6"] = noise_table_leg(CH, args.noise_trials)
        # --- end to end through the C ABI: pinned host population in, modes out, every step
        xh = torch.empty((N, d), dtype=torch.float32, pin_memory=True)
        xh.copy_(torch.from_numpy(prob.x0))
        xh_np = xh.numpy()
        for _ in range(2):
            model.load_population(0, xh_np)
            model.step()
            model.modes(0)
        ts = time.perf_counter()
        mode_rows = 0
        for _ in range(args.steps):
            model.load_population(0, xh_np)
            model.step()
            xm, fm = model.modes(0)
            mode_rows += xm.shape[0]
        te = time.perf_counter() - ts
        out["e2e"] = {"value": N * args.steps / te, "unit": "sample-cycles/s",
                      "h2d_bytes_per_step": N * d * 4,
                      "d2h_bytes_per_step": int(112 + 4 * (d + 1) * mode_rows / args.steps)}
        # --- CPU oracle on a bounded sample of the same workload
        try:
            cpu = run_cpu_leg(args.workload, args.grad, 0, sample_n=512, budget_s=12.0)
            out["cpu_baseline"] = {"value": cpu["value"], "unit": "sample-cycles/s", "cores": 1, "kind": "oracle",
                                   "sample": f"{512} of {N} samples, {cpu['cycles']} non-final cycles, "
                                             f"{args.grad} gradients, FP64 NumPy, single-threaded BLAS",
                                   "evals_per_s": cpu["evals_per_s"]}
        except Exception as e:  # report, do not hide
            out["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
        try:
            cpa = run_cpu_legs_all_cores(args.workload, args.grad, sample_n=512, budget_s=12.0)
            out["cpu_baseline_all_cores"] = {
                "value": cpa["value"], "unit": "sample-cycles/s", "cores": cpa["cores"], "kind": "oracle",
                "sample": f"{cpa['cores']} processes x 512 samples (disjoint slices of the {N}), non-final cycles "
                          f"for {cpa['seconds']:.1f} s, {args.grad} gradients, FP64 NumPy, one BLAS thread each",
                "evals_per_s": cpa["evals_per_s"]}
        except Exception as e:
            out["cpu_baseline_all_cores"] = {"value": None, "error": str(e)[:200]}
    model.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def reference_arm(args, world, rank):
    """The oracle as it stands on the host cores, same workload/metric/unit;
    each step a bounded sample (512 samples, one non-final cycle)."""
    if rank != 0:
        return
    prob = make_problem(args.workload, 0)
    sample_n = 512
    cpu = run_cpu_leg(args.workload, args.grad, 0, sample_n=sample_n, budget_s=1e9,
                      max_cycles=args.warmup + args.steps)
    ts = cpu["step_times"][args.warmup:]
    el = float(np.sum(ts))
    value = sample_n * len(ts) / el
    out = {"impl": "reference", "metric": f"sample-cycles/s ({args.grad} gradients) at N={prob.n}, d={prob.d}",
           "value": value, "unit": "sample-cycles/s", "n_gpus": world, "steps": len(ts), "warmup": args.warmup,
           "ms_per_step": 1e3 * el / max(1, len(ts)), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "N": prob.n, "d": prob.d, "grad": args.grad,
                      "sample": f"{sample_n} samples per step"},
           "cpu_baseline": {"value": value, "unit": "sample-cycles/s", "cores": 1, "kind": "oracle",
                            "sample": f"{sample_n} of {prob.n} samples per step, FP64 NumPy, single-threaded"},
           "e2e": {"value": value, "unit": "sample-cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
