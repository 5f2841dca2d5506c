"""Writes the stored expected values the benchmark reads (it may not run the oracle):

  modes_<workload>.npz  the significant modes of each workload's objective (Eq. 1:
                        Newton in FP64 from every component mean, kept when
                        f >= f_max + log delta; the quadratic's centre), their f
                        values and -Hess f there -- oracle.modes.significant_modes;
  exact_mixture256_d64.npz  the exact FP64 value and gradient of the d = 64, K = 256
                        full-covariance mixture (oracle.objectives) at 256 sampled
                        rows of the workload's population, the points where the
                        benchmark reports the tensor-core objective's error.

Only oracle/ and the seeded input module are called.  Run from the repository root:
``python tests/golden/make_modes.py``; tests/test_oracle_golden.py checks that the
stored files equal a fresh computation.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import modes as MD  # noqa: E402
from oracle import objectives as OB  # noqa: E402
from paper_2606_26164_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
MODE_WORKLOADS = ("mixture4_d2", "mixture32_d16", "quadratic_d64", "mixture256_d64")
EXACT_ROWS = np.arange(0, 65536, 256)            # 256 rows spread over the population


def modes_of(name):
    prob = I.WORKLOADS[name](n=16)                 # the objective does not depend on N
    x, f, negH = MD.significant_modes(prob)
    return {"x": x, "f": f, "neg_hess": negH}


def exact_mixture256():
    prob = I.mixture256_d64()
    X = prob.x0[EXACT_ROWS].astype(np.float64)
    return {"rows": EXACT_ROWS, "x": X, "f": OB.value(prob.objective, X), "g": OB.grad(prob.objective, X)}


def path(name):
    return os.path.join(HERE, name + ".npz")


def main():
    for name in MODE_WORKLOADS:
        np.savez_compressed(path("modes_" + name), **modes_of(name))
    np.savez_compressed(path("exact_mixture256_d64"), **exact_mixture256())


if __name__ == "__main__":
    main()
