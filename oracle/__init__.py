"""CPU oracle for multigrid waveform relaxation (MGWR) on the time-fractional
heat equation -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, FP64 restatement of what the GPU path
computes, written from the paper's equations.  Only the test suite, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product
path (the CUDA library and its Python binding) never does, and shares no code
with it apart from the seeded input generators in
``paper_1608_05400_gb300.inputs``.

Modules
  l1         L1 weights d_k, Toeplitz column r_i (Sec. 2 L1 scheme; Sec. 5 T_M)
  toeplitz   first column of (T_M + sigma I)^{-1} by forward substitution (Sec. 5)
  direct     the discrete solution by L1 time stepping (Sec. 2 / Sec. 6 discrete
             models) and by a dense all-at-once solve of T_M (x) I + A_h (Sec. 5)
  separable  exact discrete solution for separable sources (sine eigenvector)
  mgwr       Algorithm 1 (WRMG) in 1-D and 2-D: red-black waveform smoother,
             defect, full weighting, linear / bilinear interpolation, V/W cycles
  mittag_leffler  E_alpha(z) by its power series: the exact solution of the
             Sec. 7 experiment with initial value sin x
  fas        waveform relaxation FAS for the 1-D nonlinear problem of Sec. 7
             (conservative flux, upwind convection) and a time-marching Newton
             solver of the same discrete problem
  sama       semi-algebraic mode analysis of the 1-D two-grid cycle (Sec. 4):
             predicted smoothing and two-grid factors; a CPU tool as well
             (python -m oracle.sama)

Pin status: every function above is pinned by a CPU test against something
other than itself (closed forms, a dense solve, brute force, special cases);
see tests/test_oracle_*.py.
"""
