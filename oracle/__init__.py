"""RIDG oracle: a plain, slow, FP64 CPU implementation of the regionally-implicit DG step.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import it; the product library never does, and it shares no
code, tables or helpers with the CUDA path.

Modules
-------
basis      1D orthonormal Legendre basis, Gauss rules, derivative / trace / triple-product
           tables (Sec. 2.1; Sec. 3 triple-product integrals).
linear     Linear-flux prediction by solving every region system (eq. pred_full_system)
           and keeping the centre element; explicit correction (Sec. 2.3).
nonlinear  Residual of eq. pred_full_system by Gauss quadrature, quasi-quadrature-free
           Jacobian (eqs. Jacproj, Jacobian2), quadrature Jacobian (eq. Jacobian),
           Newton iteration (Sec. 3) and the nonlinear correction (Sec. 2.3).
error      Approximate relative L2 error (eq. l2relerror) and observed order (eq. Mratio).
"""
