"""FP64 CPU oracle for the QTT fractional-step hot path (arXiv:2507.05222).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call, link or
execute anything under ``oracle/``.  The CUDA library never does, and this package never
imports the CUDA library.

* ``fd``      -- L0: full-grid finite-difference fractional step (the definition).
* ``tt``      -- L1: plain TT algebra (TT-SVD, rounding, sums, mat-vec, Hadamard, fit, ALS).
* ``qtt_ops`` -- L1: analytic QTT grid fields, metric terms, FD operators, boundary vectors.
* ``step``    -- L1: the QTT fractional step built from the above.
* ``nn``      -- the learned Poisson warm start: network, loss, Adam step, grid transfers.

Parity status: every function is pinned by a ``-m "not gpu"`` test (tests/test_oracle_*.py)
against the paper's worked example, closed forms, brute force or L0.
"""
