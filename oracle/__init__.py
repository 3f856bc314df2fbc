"""FP64 CPU oracle for the FDLBM of Gan et al. (arXiv 0801.4169).

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA product path never does, and shares no code with it.

Modules:
  fdlbm      -- ctypes wrapper over fdlbm_oracle.c (the scheme itself, Eqs. 1-17)
  fdlbm_mp   -- a second, independent reading of the step in mpmath at 40+ digits (small grids),
                which decides whether a rejected run fails in exact arithmetic or only in FP64
  riemann    -- exact Riemann solver for the model's gamma = 2 (Sec. 5.1 reference curves)
  shocks     -- Rankine-Hugoniot and oblique-shock relations (Sec. 5.2 states)
  vonneumann -- amplification matrix G of Eqs. 18-20
"""
