"""FP64 CPU oracle for the circle-cover interfacial system (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, obviously correct restatement of the method of
"An explicit substructuring method for overlapping domain decomposition based
on stochastic calculus" (Moron-Vidal, Bernal, Suzuki): the circle cover
(Eqs. 4-7), interfaces, knots and stencils (Eqs. 8-12), the Fourier and IMQ
cardinal functions (Eqs. 14-22), the interfacial system (Eqs. 28-30), the
pseudospectral floating rows (Eqs. 31-35, 40-41), the Feynman-Kac
Euler-Maruyama perimeter rows (Eqs. 25-30, 53, 56) with the optional
Gobet-Menozzi boundary shift, averaged multi-subdomain rows (Eqs. 38-39), the
global solve (direct, GMRES, RAS-preconditioned, Eqs. 42-45), the Poisson test
of Eq. 46 and an adjoint gradient.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or link anything in
this package.  It shares no code with the CUDA library and never imports it.

Parity status per module (what pins each one is listed in its docstring):
  problem    pinned (closed forms of the manufactured solutions; u46 at the origin, its
             symmetry, central differences of its derivatives)
  cover      pinned (hand counts, coverage/stencil invariants, brute force, incl. Pi_i)
  spectral   pinned (textbook differentiation matrices, Poisson kernel, mean exit time)
  imq        pinned (Kronecker property, exactness on the IMQ span, 50-digit solve)
  mc         pinned (Philox against a library implementation, Brownian exit
             laws on a disk, Poisson-kernel harmonic measure, the boundary shift's
             exit-time bias, Feynman-Kac for Eq. 46 on a disk)
  system     pinned (constant data, harmonic rows with averaged subdomains, Table 1
             statistics of the Eq. 46 system)
  krylov     pinned (residual of the direct sparse solve, dense LU, RAS special cases)
  adjoint    pinned (central finite differences with common random numbers)
"""
