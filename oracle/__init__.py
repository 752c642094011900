"""FP64 CPU oracle for the fast Fourier spectral collision operator (test infrastructure).

This package is test infrastructure.  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the product library never
does.  It shares no code with the CUDA path: its quadrature rules, kernel
constants, F table (``ftable.c``), DFT and operator are written independently
from the paper.

Modules
-------
quadrature   radial Gauss-Legendre rule and sphere rules (Sec. 4, eq. approxG)
kernels      angular kernels b(cos theta), their normalisation and Taylor moments
             (Sec. 2.1, Sec. 4.1, Sec. 5.1, eqs. b5-b8)
ftable       F(k, |q|, qhat) by the split of Sec. 4.1 (C, OpenMP), plus an exact
             Funk-Hecke series used only as an independent pin
spectral     DFT by definition, the operator of eq. realQ, the direct weighted
             sum of eq. sum (small N), BKW closed forms (Sec. 5.1), moments, RK4

Every function cites the passage it follows.  Parity-unpinned parts: none (see
the pins in tests/test_oracle_*.py).
"""
from . import quadrature, kernels, ftable, spectral  # noqa: F401
