"""CPU FP64 oracle for the condensed interior-point method (test infrastructure).

This package is test infrastructure.  Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it;
the library itself never does, and it shares no code with the CUDA path
(only the seeded networks of ``gridgen`` serve both).

Contents
--------
model   polar AC-OPF in state-control form (Sec. 2.1, Eq. 2-3): residuals,
        hand-derived Jacobians and Lagrangian Hessian.
kkt     the augmented KKT matrix (Eq. kktmatrix:normal), its dense full-space
        solve, the condensed matrix by definition (Theorems 1-2 and
        Eq. algo:reduction), the condensed step with recovery, and inertia
        (Theorem 3).
ipm     the primal-dual barrier loop around it, linearize-then-reduce
        (Algorithm 1) and reduce-then-linearize (Algorithm 2) with the
        Newton-Raphson projection.
sens    derivative of the optimal dispatch with respect to the bus loads.

Every floating-point quantity is float64.  Pins (tests under ``-m "not gpu"``)
tie each function to something other than itself: complex-step and
finite-difference derivatives, the complex-matrix power-injection form, the
full-space LDL^T step, Sylvester inertia, the lossless economic-dispatch closed
form, an independent SciPy optimiser on a 3-bus case, and the reduced-derivative
theorem through the Newton-Raphson projection.
"""
