"""GB300 (sm_103a) implementation of RLOBPCG's data-parallel hot path.

RLOBPCG (Epperly, Park & Nakatsukasa, arXiv 2602.16797): sketch-preconditioned block LOBPCG for
the few smallest singular triplets (or the nullspace) of a tall matrix. The compute runs in the
CUDA library built from ``csrc/`` (C ABI in ``include/rlobpcg.h``); ``rlobpcg`` is its Python
binding and ``workloads`` draws seeded synthetic test matrices.
"""
__all__ = ["rlobpcg", "workloads", "build"]
