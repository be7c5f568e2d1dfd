"""GB300 (sm_103a) FFT-preconditioned Schur-complement GMRES for the 5-point
Helmholtz-Poisson equation on L, T and cross block domains.

The solver is the CUDA library libfpg.so behind the C ABI of include/fpg.h;
`binding` is its thin ctypes wrapper and `build` compiles it in-tree.
"""
__all__ = ["binding", "build"]
