"""Plain, slow FP64 CPU oracle for the space-angle DG transport method of
Lathouwers & Perko, "An Angular Multigrid Preconditioner for the Radiation
Transport Equation with Forward-Peaked Scatter" (arXiv 2010.04559).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  The CUDA library in
``paper_2010_04559_gb300`` never calls it and shares no code with it: every
table (angular mesh, bases, quadrature, spherical harmonics, spatial Q1
matrices) is rebuilt here from the paper's definitions.

Modules
-------
harmonics  real orthonormal spherical harmonics Y_{n,o} (Sec. 4.2, flux moments)
angular    spherical patch hierarchy, Const/Lin bases, patch quadrature and the
           angular matrices M, A^xi, X, the prolongation P (Sec. 2.1-2.3, 4.1)
spatial    DG-Q1 spatial matrices N, V_xi and face traces (Sec. 2.3)
transport  the discrete operators L, S, the source f, the sweep L^-1 and the
           scalar flux (Eq. complete, Sec. 3, Sec. 4.2)
multigrid  restriction/prolongation, source-iteration smoother, the linear
           V-cycle of Fig. lmg and the coarse block Gauss-Seidel solver (Sec. 4)
gmres      right-preconditioned restarted GMRES with CGS2 orthogonalisation

Every function is written from the defining formula; where the paper is silent
the reading taken is stated in the function's docstring.
"""
