"""Plain FP64 CPU oracle for the semi-implicit multilevel SDC method (SI-MLSDC).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
reference that the CUDA path is checked against.  Only the test suite, the
``smoke()`` check and the CPU-baseline leg of the benchmark may import it.
The product path (the C-ABI library and its Python binding) never imports,
links or executes anything in here, and this package imports nothing from
the product path.

Modules
-------
tables     collocation nodes, node-to-node weights, GLL tables, Lagrange
           transfer matrices (Sec. 3.1-3.2, Sec. 4.2, Sec. 6.2)
dg         DG-SEM operators on periodic uniform 1D/2D meshes: strong-form
           convective operator with a Rusanov flux, SIPG diffusion operator,
           GLL mass (Sec. 6; the flux details follow the stated readings)
solver     Jacobi-preconditioned CG for (M + c A) x = M r
sdc        SI(1)/SI(2) predictor and incremental corrector sweep, collocation
           residual (Sec. 3.3, Sec. 4.3, Algorithm 1)
mlsdc      space-time transfers, FAS right-hand side, V-cycle, Cascade and
           FMG starts, one time step (Sec. 4.1-4.7, Algorithms 2-4)
dahlquist  the scalar Fourier-mode problem of Sec. 5 driven through the same
           sdc/mlsdc code (stability function R(z))
mlp        FP64 reference of the element-patch MLP (forward/backward)
fds        element-wise fast-diagonalisation preconditioner (Sec. 8's fast
           diagonalisation solver, element-local reading)
av         Persson-Peraire artificial viscosity added to f (Sec. 6; the form
           follows the stated readings)

Parity status of every function is listed in the module docstrings.
"""
