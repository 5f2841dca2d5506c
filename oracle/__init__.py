"""CPU oracle for the ChiSao population step -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 NumPy implementation of Algorithm 1 (Section 3.4) and its
phases (Sections 3.2.1-3.2.6), written from the paper.  It shares no code with
the CUDA library: it has its own Philox generator, its own Householder QR and
its own objectives.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path never does.

Modules
-------
philox      Philox4x32-10 and the stream layout both sides implement.
objectives  value / analytic gradient / Hessian of the objective families.
method      the phases of one oscillation cycle and the cycle driver.
modes       ground-truth significant-mode sets (Eq. 1) by Newton's method.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, library routines, published test vectors or brute
force (see tests/test_oracle_*.py).  Functions whose results the paper does
not fix numerically (the noise experiment of Section 5.6) are marked
"parity unpinned" where they are defined.
"""
