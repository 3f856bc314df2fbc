"""GB300-native FDLBM for compressible flow with high Mach number (Gan et al., arXiv 0801.4169).

The compute path is hand-written sm_103a CUDA behind the C ABI of include/fdlbm.h
(libfdlbm_gb300.so). ``paper_0801_4169_gb300.fdlbm`` is the thin ctypes binding with
the same names; ``workloads`` builds seeded synthetic inputs.
"""
__all__ = ["fdlbm", "workloads"]
