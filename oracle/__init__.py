"""Plain FP64 CPU oracle of the adaptive randomized butterfly factorization.

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may use it.  It shares no code with the
CUDA path (``paper_2002_03400_gb300/csrc``); the two meet only on the seeded
inputs of ``paper_2002_03400_gb300.inputs`` (which the oracle does not
import either: callers pass arrays in).

Modules, each following the paper step by step in complex128:

* ``rng``        Philox-4x32-10 counter-based generator + Box-Muller normals
                 (the random matrices of Alg. 1 step 1 and Sec. 4.1).
* ``tree``       bisection trees T_S, T_T (Sec. 3.1).
* ``qr``         column-pivoted Householder QR with truncation (Alg. 1 step 3).
* ``operators``  black-box products with A and A^T (dense, kernel, butterfly,
                 composition) (Alg. 2 input, Sec. 4.1).
* ``butterfly``  Alg. 2 (adaptive hybrid butterfly), its apply
                 (eq. hybrid_butterfly_mat) and the error metric (Sec. 7, eq. error).

Parity status per function is listed in each module header; every function
here is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
