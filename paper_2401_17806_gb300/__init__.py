"""GB300-native Schur-complement / Helmholtz CG solver for the staggered
semi-Lagrangian IMEX DG method (Tavelli & Boscheri, Sec. 2-3).

Importing the package loads nothing compiled.  ``paper_2401_17806_gb300.dgsl``
is the ctypes binding of the C-ABI library ``libdgsl.so``; it raises if the
library has not been built.
"""
__all__ = ["synth", "dgsl"]
