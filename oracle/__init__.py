"""FP64 CPU oracle for the IgA Helmholtz solver of arXiv 2010.10232.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm) may
import or call anything in this package.  The product path (the CUDA library
and its Python binding) never imports it and shares no code with it.

Every function is a plain, slow, obviously-correct restatement of the paper:

* ``bspline``    knot vectors and the Cox-de Boor recursion (Section 2.3.1)
* ``assembly``   Gauss-quadrature assembly of S, M, M_{k^2} (Section 2.3, Eq. linearsystem1)
* ``multigrid``  knot-insertion transfers, rediscretised CSLP levels, damped
                 Jacobi, V-cycle (Section 3, CSLP paragraph; Section 4.2)
* ``deflation``  ADP deflation matrix Z, E = Z^T A Z, P = I - A Q (Section 3, Eq. adef1 and the Z stencils)
* ``krylov``     GMRES (left preconditioned, MGS Arnoldi, Givens) and FGMRES
* ``solver``     end-to-end deflated, preconditioned solve and direct solve
* ``cnn``        NumPy reference 3x3 convolution network (forward/backward)

Parity status of each function is stated in its docstring; functions with no
independent pin say "parity unpinned".
"""
