"""FP64 CPU oracle for the FDLBM of Gan et al. (arXiv 0801.4169).

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA product path never does, and shares no code with it.

Modules:
  fdlbm      -- ctypes wrapper over fdlbm_oracle.c (the scheme itself, Eqs. 1-17)
  riemann    -- exact Riemann solver for the model's gamma = 2 (Sec. 5.1 reference curves)
  shocks     -- Rankine-Hugoniot and oblique-shock relations (Sec. 5.2 states)
  vonneumann -- amplification matrix G of Eqs. 18-20
"""
