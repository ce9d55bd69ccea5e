"""Plain CPU FP64 oracle of the hybrid-spectral free-surface Navier-Stokes hot path.

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` (to check one small GPU result) and by the CPU
baseline / reference leg of ``bench.py``.  The product path (the CUDA library
and its Python binding) never imports, links or executes anything here, and
nothing here imports the product package.

Everything is numpy float64, written to be read against the paper
(Melander, Bitsch, Chen, Engsig-Karup, "A High-Order Hybrid-Spectral
Incompressible Navier-Stokes Model For Nonlinear Water Waves"):

* ``spectral``  - Fourier and Chebyshev-Gauss-Lobatto grids, differentiation,
                  modal transforms, the exponential cut-off filter (Sec. 3.4-3.6).
* ``operator``  - sigma-transform metric (Eq. 1_Scoef), transformed gradient and
                  divergence (Eq. 1_chain), the mixed-stage Poisson operator with
                  its Dirichlet / Neumann rows (Eq. poissonp, bcpd, bcpdneu).
* ``pmg``       - geometric p-multigrid: coarsening (Sec. 4.1), spectral
                  transfers (Sec. 4.2), block smoothers (Sec. 4.3), V-cycle
                  (Algorithm 1), FMG (Algorithm 2), dense coarsest solve.
* ``krylov``    - restarted GMRES with right preconditioning (Sec. 4.4).
* ``rk``        - low-storage explicit Runge-Kutta (Eq. LSERK) with the
                  pressure projection at every stage (Sec. 3.2-3.3) and the
                  kinematic free-surface update (Eq. kinematicFS).
* ``adjoint``   - exact derivative of the 2D time step and of a gauge loss
                  (the paper has no adjoint): the step restated in plain
                  PyTorch CPU float64 with a dense operator and LU solve,
                  differentiated by torch.autograd; pinned against the numpy
                  step and by central finite differences.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test unless it says "parity unpinned".
"""

from . import spectral, operator, pmg, krylov, rk  # noqa: F401
