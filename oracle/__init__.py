"""FP64 CPU oracle for the nested MLMC hot path (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference arm may import anything under ``oracle/``.  The product path (the
CUDA library and its Python binding) never does.

Modules:
  build   -- gcc build of mlmc_oracle.c
  core    -- ctypes wrapper: Philox4x32-10, exact inverse CDF, the level simulation
  tables  -- Method-1 / Method-3 approximate inverse-CDF tables (mpmath)
  driver  -- the MLMC sample-size formulas and the adaptive MLMC algorithm
"""
