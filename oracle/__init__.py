"""Plain, slow FP64 CPU oracle of the wavelet multilevel l1 deblurring method.

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports, links or
calls this package; only the test-suite, the smoke check and the benchmark's
CPU-baseline leg do. It shares no code with the CUDA path.

Every function follows a passage of the paper (section / equation /
algorithm cited in its docstring) step by step, in float64, using numpy and
scipy primitives (sparse and dense matrix products, a dense generalized
symmetric eigensolver) with no blocking, fusion or reordering beyond what the
definition states.

Parity status of each part (what pins it is in tests/test_oracle_*.py):
  operators  -- pinned (explicit-loop definitions, transpose identities,
                filter orthonormality, Galerkin identity against dense W)
  lsqr       -- pinned (dense least-squares solve)
  gcv        -- exact mode pinned (dense solves + explicit trace + brute grid);
                projected mode pinned to exact mode at full subspace dimension
  solvers    -- pinned by majorisation invariants (MM, IRLS), the l1 KKT
                conditions (SB) and Tikhonov special cases
  mgm        -- levels = 1 reduces to Approach I; the end-to-end result has no
                printed example to compare with ("parity unpinned" against the
                paper's numbers, which need its test images)
"""
